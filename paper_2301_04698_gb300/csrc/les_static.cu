// les_static.cu -- a Poisson solve that allocates nothing, for callers that
// cannot allocate device memory themselves.
//
// Every other entry point works on a handle whose workspace the caller
// allocates.  Some callers cannot do that: a plug-in living inside a host
// application whose device memory is owned entirely by the host's own pool
// allocator (a third-party cudaMalloc would bypass the pool's budget and
// fragment it), or a latency-bound loop that must not call cudaMalloc /
// cudaFree because those calls can synchronise the whole device and stall
// other streams.  les_poisson_solve_static() serves them: the caller passes
// only the right-hand side and the solution array, and the solver's work
// vectors, control block and reduction partials live in one file-scope
// __device__ array that every GPU loading this library holds until the
// process exits.  The paper has no counterpart; the solve itself is the same
// CG / weighted-Jacobi code as les_poisson_solve().
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>

#include "les_internal.h"

namespace {

// Layout of the static scratch: [control block | reduction partials | 4 vectors]
constexpr size_t kCtlBytes = 256;
constexpr int kMaxBlocks = 2048;                                   // grid cap
constexpr size_t kPartialBytes = (size_t)16 * kMaxBlocks * sizeof(double);  // 256 KiB
constexpr size_t kVecBytes = (size_t)16 << 20;                     // 16 MiB for r, p_a, p_b, q
constexpr size_t kScratchBytes = kCtlBytes + kPartialBytes + kVecBytes;
static_assert(sizeof(les::SolverCtl) <= kCtlBytes, "control block does not fit");

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// device address of g_scratch in the current device's context, looked up on
// every call (no allocation): a cached address would go stale if the
// context were torn down and created again in the same process
int scratch_address(void** out, std::string* err) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
  if (e != cudaSuccess || !p) {
    *err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
    return LES_ERR_CUDA;
  }
  *out = p;
  return LES_OK;
}

template <typename T>
int solve_static(const les_config& c, const void* rho0, const void* rhs, void* x, double rtol, int maxit,
                 cudaStream_t st, char* base, int* iters, double* rel, std::string* err) {
  using namespace les;
  const size_t n = (size_t)c.nx * c.ny * c.nz;
  int nsm = 148, dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  SolverArgs<T> s;
  s.g = make_grid<T>(c, 8);
  s.lc = tile_launch(s.g, std::min(kMaxBlocks, std::max(1, nsm) * 8));
  s.st = st;
  s.op = c.poisson_op;
  s.solver = c.solver;
  s.omega = c.jacobi_omega;
  s.rho0 = (const T*)rho0;
  s.ctl = (SolverCtl*)base;
  SolverCtl host_ctl{};
  s.ctl_host = &host_ctl;
  s.partials = (double*)(base + kCtlBytes);
  T* vec = (T*)(base + kCtlBytes + kPartialBytes);
  s.r = vec;
  s.p0 = vec + n;
  s.p1 = vec + 2 * n;
  s.q = vec + 3 * n;
  s.prof = nullptr;
  // the array keeps the previous call's contents: the control block (with
  // the reduction tickets) must start at zero; the vectors are written
  // before they are read.
  cudaError_t e = cudaMemsetAsync(base, 0, kCtlBytes, st);
  if (e != cudaSuccess) {
    *err = std::string("clearing the control block: ") + cudaGetErrorString(e);
    return LES_ERR_CUDA;
  }
  return poisson_solve<T>(s, (const T*)rhs, (T*)x, rtol, maxit, iters, rel, err);
}

void put_err(char* buf, size_t len, const std::string& m) {
  if (buf && len) std::snprintf(buf, len, "%s", m.c_str());
}

}  // namespace

extern "C" int les_poisson_solve_static(const les_config* cfg, const void* d_rho0, const void* d_rhs,
                                        void* d_x, double rtol, int32_t maxit, void* stream, int32_t* iters,
                                        double* rel_res, char* err, size_t err_len) {
  put_err(err, err_len, "");
  auto bad = [&](const std::string& m) {
    put_err(err, err_len, m);
    return LES_ERR_INVALID_ARG;
  };
  if (!cfg || cfg->struct_size != sizeof(les_config)) return bad("config is NULL or has the wrong struct_size");
  if (cfg->precision != 32 && cfg->precision != 64) return bad("precision must be 32 or 64");
  if (cfg->nx < 3 || cfg->ny < 3 || cfg->nz < 2) return bad("grid must be at least 3 x 3 x 2");
  if (!(cfg->dx > 0 && cfg->dy > 0 && cfg->dz > 0)) return bad("spacings must be positive");
  if (cfg->bc_z != LES_BC_PERIODIC && cfg->bc_z != LES_BC_WALLS) return bad("bc_z invalid");
  if (cfg->solver != LES_SOLVER_CG && cfg->solver != LES_SOLVER_JACOBI) return bad("solver invalid");
  if (cfg->poisson_op != LES_OP_COMPACT && cfg->poisson_op != LES_OP_WIDE) return bad("poisson_op invalid");
  if (cfg->solver == LES_SOLVER_JACOBI && cfg->poisson_op != LES_OP_COMPACT)
    return bad("weighted Jacobi is defined for the compact operator only");
  if (cfg->poisson_op == LES_OP_WIDE && !d_rho0) return bad("the wide operator needs d_rho0");
  if (!d_rhs || !d_x || !(rtol > 0) || maxit < 0) return bad("NULL array, rtol <= 0 or maxit < 0");
  const size_t es = cfg->precision == 64 ? 8 : 4;
  const size_t n = (size_t)cfg->nx * cfg->ny * cfg->nz;
  const size_t max_cells = kVecBytes / (4 * es);
  if (n > max_cells) {
    char m[160];
    std::snprintf(m, sizeof(m), "grid of %zu cells exceeds the static scratch limit of %zu cells at precision %d",
                  n, max_cells, cfg->precision);
    return bad(m);
  }
  void* base = nullptr;
  std::string msg;
  int rc = scratch_address(&base, &msg);
  if (rc != LES_OK) {
    put_err(err, err_len, msg);
    return rc;
  }
  int it = 0;
  double rel = 0;
  if (cfg->precision == 64)
    rc = solve_static<double>(*cfg, d_rho0, d_rhs, d_x, rtol, maxit, (cudaStream_t)stream, (char*)base, &it, &rel,
                              &msg);
  else
    rc = solve_static<float>(*cfg, d_rho0, d_rhs, d_x, rtol, maxit, (cudaStream_t)stream, (char*)base, &it, &rel,
                             &msg);
  if (iters) *iters = it;
  if (rel_res) *rel_res = rel;
  if (rc != LES_OK) put_err(err, err_len, msg.empty() ? "Poisson solve reached maxit" : msg);
  return rc;
}
