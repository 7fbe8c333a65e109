// les_internal.h -- host-side declarations shared by the translation units of
// libles.so (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "les.h"
#include "les_common.cuh"

namespace les {

// Physical constants of Table 1 (and the reading of the saturation vapour
// pressure: Clausius-Clapeyron with constant L_v0 from the triple point).
constexpr double kRd = 287.0;
constexpr double kRv = 461.89;
constexpr double kCpd = 1004.5;
constexpr double kCpv = 1859.5;
constexpr double kCl = 4181.0;
constexpr double kLv0 = 2.47e6;
constexpr double kGrav = 9.81;
constexpr double kTtr = 273.16;
constexpr double kEtr = 611.657;

// Per-launch physics parameters (passed by value).
template <typename T>
struct Phys {
  uint32_t flags;
  T dt;
  T cs2d2;            // (c_s Delta)^2
  T inv_pr, inv_sc;
  T nu_const;
  T f_cor, ug, vg;
  T sponge_rate, sponge_zs, sponge_h;
  T subs_div;
  T sflux_th, sflux_qt;  // rho0 (w' phi')_s: SHF / c_pd, LHF / L_v0
  T rad_f0, rad_f1, rad_kappa;
  T p00;
  T sat_tol;
  int sat_maxit;
  int advection;      // LES_ADV_*
  const T* rho0;      // nz
  const T* alpha0;    // nz
  const T* p0;        // nz
};

// Device-side solver control block (lives in the workspace).
// Algorithmic traffic of a CG solve in fields per node, the same for every
// CG kernel whatever it moves: the set-up (mean of b: 1; r = b - L_c x0:
// b, x in, r out: 3; the gauge: x twice in, x out: 3) and, per iteration,
// the matvec with its dot product (p in, q out: 2) and the update (x, p, r,
// q in; x, r out: 6).  A kernel's DRAM traffic is measured separately.
constexpr double kCgSetupFields = 7.0;
constexpr double kCgIterFields = 8.0;

struct SolverCtl {
  double sum;       // result of the last mean reduction
  double bn2;       // ||b - mean(b)||^2
  double rr;        // r.r
  double pq;        // p.Ap
  double alpha, beta;
  double rel;       // current relative residual
  double tol;
  int iter, maxit;
  int done;         // 0 running, 1 converged, 2 maxit, 3 breakdown, 4 zero rhs
  int first;        // next CG iteration is the first one
  int answer;       // Jacobi: buffer holding the answer (0 = x, 1 = scratch)
  int pad;
  double scal;      // misc scalar (CFL max)
  unsigned tickets[8];
};

enum Ticket { TK_SUM = 0, TK_INIT, TK_MATVEC, TK_UPDATE, TK_JACOBI, TK_DIAG, TK_MAX, TK_SPARE };

// Grid barrier of the persistent solver (lives in the workspace, cleared
// before every launch).
// Grid barrier of the persistent solver (lives in the workspace, cleared
// before every launch).  The arrival counter, the generation and the fail
// flag each sit in their own 128-byte line so that polling does not contend
// with the arrivals.
struct alignas(128) BarLine {
  unsigned v;
  unsigned pad[31];
};
struct FusedBar {
  BarLine count;                 // blocks arrived at the current barrier
  BarLine gen;                   // barrier generation
  BarLine fail;                  // a wait timed out
  alignas(128) double value[4];  // totals published by the last block to arrive
};

// Tile shape and limits of the persistent solver.
struct FusedCfg {
  int ty = 2;                           // thread rows per block (block = 32 x ty)
  int zc = 8;                           // z-planes per tile (2 x 8: fastest of a sweep at 1024^2 x 128
                                        // and 1536^2 x 256, FP32)
  int max_blocks = 1 << 30;             // cap on the cooperative grid
  long long spin_cycles = 4000000000LL; // barrier wait limit (~2 s at 2 GHz)
  double timeout_ms = 2000.0;
  int missing = 0;                      // test hook: arrivals that never come
  int stencil_path = 0;                 // 0 column marches where eligible (else rolling), 1 rolling z-march
  int variant = 0;                      // 0 standard iterates (resident, else FP32 columns, else
                                        // two-phase streaming when tile-aligned, else one-pass),
                                        // 2 two-phase streaming, 3 one-pass one-reduction, 4 columns
  int resident = 0;                     // 0 on-chip CG when the grid fits (p, r, q in registers where
                                        // the grid allows), 1 never, 2 on chip with every vector in
                                        // shared memory
};

struct LaunchCfg {
  dim3 grid, block;
};

// Kernel classes for launch counting and the optional event profiler.
enum KernelId : int {
  KI_THERMO = 0, KI_RADIATION, KI_SCALAR, KI_MOMENTUM, KI_RHS, KI_CORRECT,
  KI_DIAG, KI_CFL, KI_APPLY, KI_SUM, KI_CG_INIT, KI_CG_MATVEC, KI_CG_UPDATE, KI_JACOBI, KI_FINISH,
  KI_CTL, KI_CG_FUSED, KI_UNET_CONV, KI_UNET_WGRAD, KI_UNET_ADAM, KI_CG_RESIDENT, KI_CG_ROLL, KI_CG_WAVE, KI_CG_REGS, KI_COUNT
};
extern const char* const kKernelNames[KI_COUNT];

// Counts every launch; when enabled, brackets each launch with a pair of
// CUDA events on the launching stream and accumulates the elapsed times.
struct Profiler {
  bool on = false;
  long long launches[KI_COUNT] = {};
  long long timed[KI_COUNT] = {};
  double ms[KI_COUNT] = {};
  double bytes[KI_COUNT] = {};  // algorithmic bytes of launches whose size varies
  struct Rec {
    int id;
    cudaEvent_t a, b;
  };
  std::vector<Rec> pending;
  std::vector<cudaEvent_t> pool;

  cudaEvent_t take() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  void begin(int id, cudaStream_t st) {
    launches[id] += 1;
    if (!on) return;
    Rec r{id, take(), take()};
    cudaEventRecord(r.a, st);
    pending.push_back(r);
  }
  void end(cudaStream_t st) {
    if (!on || pending.empty()) return;
    cudaEventRecord(pending.back().b, st);
  }
  // fold the finished records into the totals (synchronises on the last one)
  cudaError_t collect() {
    if (pending.empty()) return cudaSuccess;
    cudaError_t e = cudaEventSynchronize(pending.back().b);
    if (e != cudaSuccess) return e;
    for (auto& r : pending) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
        ms[r.id] += t;
        timed[r.id] += 1;
      }
      pool.push_back(r.a);
      pool.push_back(r.b);
    }
    pending.clear();
    return cudaSuccess;
  }
  void reset() {
    collect();
    for (int i = 0; i < KI_COUNT; ++i) launches[i] = timed[i] = 0, ms[i] = bytes[i] = 0.0;
  }
  ~Profiler() {
    for (auto& r : pending) {
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
    for (auto e : pool) cudaEventDestroy(e);
  }
};

// launch bracket: counts (and optionally times) one kernel launch
struct ProfScope {
  Profiler* p;
  cudaStream_t st;
  ProfScope(Profiler* prof, int id, cudaStream_t s) : p(prof), st(s) {
    if (p) p->begin(id, st);
  }
  ~ProfScope() {
    if (p) p->end(st);
  }
};

template <typename T>
Grid<T> make_grid(const les_config& c, int zc);

template <typename T>
LaunchCfg tile_launch(const Grid<T>& g, int max_blocks);

// ---- stencil stage launchers (les_stencil.cu) ------------------------------
template <typename T>
struct StageArgs {
  Grid<T> g;
  Phys<T> ph;
  LaunchCfg lc;
  cudaStream_t st;
  Profiler* prof;
};

template <typename T>
cudaError_t launch_thermo(const StageArgs<T>& a, const T* th, const T* qt, T* temp, T* ql, T* b,
                          T* srad);
// rolling-window predictors and Poisson right side (les_stencil_roll.cu)
template <typename T>
cudaError_t launch_rhs_roll(const StageArgs<T>& a, int max_blocks, int op, const T* ou, const T* ov, const T* ow,
                            const T* psi, T* rhs);
template <typename T>
cudaError_t launch_scalar_roll(const StageArgs<T>& a, int max_blocks, const T* u, const T* v, const T* w,
                               const T* b, const T* thk, const T* qtk, const T* thh, const T* qth, const T* srad,
                               T* th_out, T* qt_out);
template <typename T>
cudaError_t launch_momentum_roll(const StageArgs<T>& a, int max_blocks, const T* uk, const T* vk, const T* wk,
                                 const T* un, const T* vn, const T* wn, const T* p, const T* b, T* ou, T* ov,
                                 T* ow);
// column marches over 16-byte lanes (les_stencil_col.cu): nx a multiple of
// 32 lanes x (16 bytes / element size), ny a multiple of 8
template <typename T>
bool col_eligible(const Grid<T>& g);
template <typename T>
cudaError_t launch_correct_col(const StageArgs<T>& a, int max_blocks, const T* ou, const T* ov, const T* ow,
                               const T* psi, T* u, T* v, T* w, T* p);
template <typename T>
cudaError_t launch_rhs_col(const StageArgs<T>& a, int max_blocks, int op, const T* ou, const T* ov, const T* ow,
                           const T* psi, T* rhs);
// predictors as column marches with staged shared-memory planes
// (les_predict_col.cu): nx a multiple of 32 lanes x (16 bytes / element
// size), ny a multiple of 8
template <typename T>
bool pcol_eligible(const Grid<T>& g);
template <typename T>
cudaError_t launch_scalar_col(const StageArgs<T>& a, int nsm, const T* u, const T* v, const T* w, const T* b,
                              const T* thk, const T* qtk, const T* thh, const T* qth, const T* srad, T* th_out,
                              T* qt_out);
template <typename T>
cudaError_t launch_momentum_col(const StageArgs<T>& a, int nsm, const T* uk, const T* vk, const T* wk, const T* un,
                                const T* vn, const T* wn, const T* p, const T* b, T* ou, T* ov, T* ow);
template <typename T>
cudaError_t launch_correct(const StageArgs<T>& a, const T* ou, const T* ov, const T* ow,
                           const T* psi, T* u, T* v, T* w, T* p);
template <typename T>
cudaError_t launch_diag(const StageArgs<T>& a, const T* u, const T* v, const T* w, const T* p,
                        const T* th, const T* qt, const T* ql, double* partials, SolverCtl* ctl,
                        double* out_dev /* LES_NDIAG */);
template <typename T>
cudaError_t launch_cfl_max(const StageArgs<T>& a, const T* u, const T* v, const T* w,
                           double* partials, SolverCtl* ctl);

// ---- Poisson solver (les_solver.cu) ----------------------------------------
template <typename T>
struct SolverArgs {
  Grid<T> g;
  LaunchCfg lc;
  cudaStream_t st;
  int op;            // LES_OP_*
  int solver;        // LES_SOLVER_*
  double omega;
  const T* rho0;
  SolverCtl* ctl;    // device
  SolverCtl* ctl_host;  // pinned host mirror
  double* partials;  // device
  T* r;              // work vectors (n each)
  T* p0;
  T* p1;
  T* q;
  Profiler* prof;
  FusedBar* bar = nullptr;          // persistent-solver barrier (workspace)
  int nsm = 0;                      // SMs of the device (the persistent solves' budget)
  int guard = 0;                    // restart from x = 0 if ||b - A x0|| > ||b|| (learned guesses)
  T* e0 = nullptr;                  // two spare vectors (the flexible CG's z and b)
  T* e1 = nullptr;
  const FusedCfg* fused = nullptr;  // enables the persistent CG when eligible
};

template <typename T>
cudaError_t launch_apply(const SolverArgs<T>& a, int op, const T* x, T* y);

// Persistent single-launch CG (les_cg_fused.cu): compact operator, nx a
// multiple of the 16-byte tile width (128 floats / 64 doubles), ny a multiple
// of cfg.ty.
template <typename T>
bool fused_cg_eligible(const Grid<T>& g, int op, int solver, int ty);
template <typename T>
int poisson_solve_fused(const SolverArgs<T>& a, const FusedCfg& fc, const T* b, T* x, double tol, int maxit,
                        int* iters, double* rel, std::string* err);
// Persistent one-reduction CG, one pass per iteration (les_cg_roll.cu): any
// grid, compact operator.
template <typename T>
int poisson_solve_roll(const SolverArgs<T>& a, const FusedCfg& fc, const T* b, T* x, double tol, int maxit,
                       int* iters, double* rel, std::string* err);
// one pass and one grid sum per iteration, 64 x 16 or 32 x 32 columns with z
// windows in registers (nx % 64 == 0 and ny % 16 == 0, or both % 32 == 0)
bool wave_cg_eligible(int nx, int ny, int nz);
template <typename T>
int poisson_solve_wave(const SolverArgs<T>& a, const FusedCfg& fc, const T* b, T* x, double tol, int maxit,
                       int* iters, double* rel, std::string* err);
// Persistent CG with its vectors in shared memory (les_cg_resident.cu).
// Sets *used = false and returns LES_OK without launching when the grid has
// no brick decomposition that fits on chip; the caller then streams.
template <typename T>
int poisson_solve_resident(const SolverArgs<T>& a, const FusedCfg& fc, const T* b, T* x, double tol, int maxit,
                           int* iters, double* rel, std::string* err, bool* used);
// The same iterates with p, r and q in registers (les_cg_regs.cu): FP32
// grids with nx = 128; *used as above.
int poisson_solve_regs(const SolverArgs<float>& a, const FusedCfg& fc, const float* b, float* x, double tol,
                       int maxit, int* iters, double* rel, std::string* err, bool* used);

}  // namespace les
struct les_unet;
namespace les {
// learned warm start (les_unet.cu): psi_0 from b on the model's cubic grid
int unet_predict(les_unet* u, int precision, const void* b, void* psi0, cudaStream_t st, std::string* err);
int unet_grid(const les_unet* u);

// Flexible CG with the learned network as the preconditioner (les_fcg.cu);
// *fallbacks counts the iterations that took z = -r.
template <typename T>
int poisson_solve_fcg(const SolverArgs<T>& a, les_unet* model, const T* b, T* x, double tol, int maxit, int* iters,
                      double* rel, int* fallbacks, std::string* err);

// Solve A x = b; returns LES_OK / LES_ERR_NOT_CONVERGED / LES_ERR_CUDA.
template <typename T>
int poisson_solve(const SolverArgs<T>& a, const T* b, T* x, double tol, int maxit, int* iters,
                  double* rel, std::string* err);

// Domain decomposition (les_dd.cu).  A local array as the dd solve reads
// and writes it: node (i, j, k) of the sub-domain at off + k sxy + j sx + i.
struct DdLayout {
  long long off, sxy;
  int sx;
};
template <typename T>
int dd_solve(les_dd* d, const les_dd_ops* ops, const T* rhs, T* x, const DdLayout& lay, double tol, int maxit,
             int* iters, double* rel, std::string* err);
// fill the LES_DD_HALO-deep x-y halos of nf fields of the widened sub-domain
int dd_halo_exchange(les_dd* d, const les_dd_ops* ops, void* const* fields, int nf, cudaStream_t st,
                     std::string* err);
void dd_widened_shape(const les_dd* d, int* nxe, int* nye, int* nz);
const les_config& dd_config(const les_dd* d);

}  // namespace les
