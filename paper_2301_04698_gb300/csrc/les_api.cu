// les_api.cu -- the C ABI of libles.so (declared in include/les.h): handle
// life cycle, workspace layout, state transfer and the stage sequence of one
// time step of the iterative predictor-corrector scheme (Sec. 2.4).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "les_internal.h"

using namespace les;

namespace {

// device buffers carved from the caller's workspace
enum Buf : int {
  B_U = 0, B_V, B_W, B_UN, B_VN, B_WN, B_P,
  B_THA, B_QTA, B_THB, B_QTB, B_THH, B_QTH,
  B_UHAT, B_VHAT, B_WHAT, B_RHS, B_PSI,
  B_B, B_QL, B_T, B_SRAD, B_E0, B_E1,  // B_E*: spare vectors of the flexible CG
  B_R, B_PA, B_PB, B_Q,
  B_NFIXED
};

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

const char* kStatus[] = {"ok", "invalid argument", "CUDA error", "Poisson solve did not converge",
                         "non-finite value", "device wait timed out", "call out of order",
                         "no warm-start model set"};

struct Layout {
  size_t field_bytes = 0;
  size_t off_fixed[B_NFIXED] = {};
  std::vector<size_t> off_prev;
  size_t off_prof = 0, off_ctl = 0, off_partials = 0, off_diag = 0, off_bar = 0;
  size_t total = 0;
  int max_blocks = 0;
};

int validate(const les_config* c, std::string* why) {
  auto bad = [&](const char* m) {
    if (why) *why = m;
    return LES_ERR_INVALID_ARG;
  };
  if (!c) return bad("config is NULL");
  if (c->struct_size != sizeof(les_config)) return bad("les_config.struct_size mismatch (ABI)");
  if (c->precision != 32 && c->precision != 64) return bad("precision must be 32 or 64");
  if (c->nx < 3 || c->ny < 3 || c->nz < 2) return bad("grid must be at least 3 x 3 x 2");
  if ((double)c->nx * c->ny * c->nz > 4.0e9) return bad("grid too large");
  if (!(c->dx > 0 && c->dy > 0 && c->dz > 0)) return bad("spacings must be positive");
  if (c->bc_z != LES_BC_PERIODIC && c->bc_z != LES_BC_WALLS) return bad("bc_z invalid");
  if (c->n_subiter < 1 || c->n_subiter > 64) return bad("n_subiter must be in [1, 64]");
  if (c->solver != LES_SOLVER_CG && c->solver != LES_SOLVER_JACOBI) return bad("solver invalid");
  if (c->poisson_op != LES_OP_COMPACT && c->poisson_op != LES_OP_WIDE) return bad("poisson_op invalid");
  if (c->solver == LES_SOLVER_JACOBI && c->poisson_op != LES_OP_COMPACT)
    return bad("weighted Jacobi is defined for the compact operator only");
  if (c->warm_start < LES_WARM_ZERO || c->warm_start > LES_WARM_LEARNED) return bad("warm_start invalid");
  if (!(c->poisson_tol > 0)) return bad("poisson_tol must be positive");
  if (c->poisson_maxit < 0) return bad("poisson_maxit must be >= 0");
  if (!(c->dt >= 0)) return bad("dt must be >= 0");
  if (c->dt == 0 && !(c->cfl > 0)) return bad("dt = 0 needs cfl > 0");
  if (c->sat_maxit < 0 || c->sat_maxit > 1000) return bad("sat_maxit out of range");
  if (c->solver_path != 0 && c->solver_path != 1) return bad("solver_path must be 0 or 1");
  if (c->advection != LES_ADV_QUICK && c->advection != LES_ADV_WENO3) return bad("unknown advection scheme");
  if (c->precond != LES_PRECOND_NONE && c->precond != LES_PRECOND_LEARNED) return bad("unknown preconditioner");
  if (c->precond == LES_PRECOND_LEARNED && (c->solver != LES_SOLVER_CG || c->poisson_op != LES_OP_COMPACT))
    return bad("the learned preconditioner needs the CG solver and the compact operator");
  return LES_OK;
}

Layout make_layout(const les_config& c, int nsm) {
  Layout L;
  const size_t n = (size_t)c.nx * c.ny * c.nz;
  const size_t es = c.precision == 64 ? 8 : 4;
  L.field_bytes = align_up(n * es);
  size_t off = 0;
  for (int b = 0; b < B_NFIXED; ++b) {
    L.off_fixed[b] = off;
    off += L.field_bytes;
  }
  if (c.warm_start != LES_WARM_ZERO) {
    for (int k = 0; k < c.n_subiter; ++k) {
      L.off_prev.push_back(off);
      off += L.field_bytes;
    }
  }
  L.off_prof = off;
  off += align_up(3 * (size_t)c.nz * es);
  L.off_ctl = off;
  off += align_up(sizeof(SolverCtl));
  L.max_blocks = std::max(1, nsm) * 8;
  L.off_partials = off;
  off += align_up((size_t)16 * L.max_blocks * sizeof(double));
  L.off_diag = off;
  off += align_up(LES_NDIAG * sizeof(double));
  L.off_bar = off;
  off += align_up(sizeof(FusedBar));
  L.total = off;
  return L;
}

int device_sms() {
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 148;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 148;
  return nsm;
}

}  // namespace

struct les_handle {
  les_config cfg;
  int dev = 0;  // the device current at les_init
  cudaStream_t st = nullptr;
  char* ws = nullptr;
  Layout L;
  size_t n = 0;
  int es = 4;
  void* fixed[B_NFIXED] = {};
  std::vector<void*> prev;
  void* profiles = nullptr;  // rho0, alpha0, p0 (nz each, precision T)
  SolverCtl* ctl = nullptr;
  SolverCtl ctl_host{};
  double* partials = nullptr;
  double* diag = nullptr;
  FusedBar* bar = nullptr;
  FusedCfg fused;
  les_unet* model = nullptr;
  int learned_fallbacks = 0;
  int cur = 0;           // scalar ping-pong: 0 -> A holds phi^k, 1 -> B
  int next_stage = LES_STAGE_BEGIN;
  int sub = 0;
  double dt = 0;
  std::string err;
  les_step_stats acc{};
  Profiler prof;
  // states uploaded ahead (les_prefetch_states), consumed in order at BEGIN
  struct Prefetch {
    const char* staging = nullptr;
    int count = 0;
    int fields[8] = {};
    cudaEvent_t ready = nullptr;
  };
  Prefetch pf[2];
  int pf_head = 0, pf_n = 0;
  cudaEvent_t pf_consumed = nullptr;  // recorded after the last consumption

  ~les_handle() {
    for (auto& p : pf)
      if (p.ready) cudaEventDestroy(p.ready);
    if (pf_consumed) cudaEventDestroy(pf_consumed);
  }

  void* field_ptr(int f) {
    switch (f) {
      case LES_U: return fixed[B_U];
      case LES_V: return fixed[B_V];
      case LES_W: return fixed[B_W];
      case LES_P: return fixed[B_P];
      case LES_THETA_L: return fixed[cur ? B_THB : B_THA];
      case LES_QT: return fixed[cur ? B_QTB : B_QTA];
      case LES_UN: return fixed[B_UN];
      case LES_VN: return fixed[B_VN];
      case LES_WN: return fixed[B_WN];
      case LES_THETA_L_HALF: return fixed[B_THH];
      case LES_QT_HALF: return fixed[B_QTH];
      case LES_UHAT: return fixed[B_UHAT];
      case LES_VHAT: return fixed[B_VHAT];
      case LES_WHAT: return fixed[B_WHAT];
      case LES_RHS: return fixed[B_RHS];
      case LES_PSI: return fixed[B_PSI];
      case LES_B: return fixed[B_B];
      case LES_QL: return fixed[B_QL];
      case LES_T: return fixed[B_T];
      case LES_SRAD: return fixed[B_SRAD];
      default: return nullptr;
    }
  }
  int fail(int status, const std::string& m) {
    err = m;
    return status;
  }
  int cuda_fail(cudaError_t e, const char* where) {
    err = std::string(where) + ": " + cudaGetErrorString(e);
    return LES_ERR_CUDA;
  }
};

namespace {

template <typename T>
Phys<T> make_phys(const les_handle* h) {
  const les_config& c = h->cfg;
  Phys<T> ph{};
  ph.flags = c.physics;
  ph.dt = (T)h->dt;
  const double delta = std::cbrt(c.dx * c.dy * c.dz);
  ph.cs2d2 = (T)((c.cs * delta) * (c.cs * delta));
  ph.inv_pr = (T)(1.0 / c.pr);
  ph.inv_sc = (T)(1.0 / c.sc);
  ph.nu_const = (T)c.const_nu;
  ph.f_cor = (T)c.f_cor;
  ph.ug = (T)c.ug;
  ph.vg = (T)c.vg;
  const double H = c.nz * c.dz;
  ph.sponge_rate = (T)c.sponge_rate;
  ph.sponge_zs = (T)((1.0 - c.sponge_frac) * H);
  ph.sponge_h = (T)H;
  ph.subs_div = (T)c.subs_div;
  ph.sflux_th = (T)(c.shf / kCpd);
  ph.sflux_qt = (T)(c.lhf / kLv0);
  ph.rad_f0 = (T)c.rad_f0;
  ph.rad_f1 = (T)c.rad_f1;
  ph.rad_kappa = (T)c.rad_kappa;
  ph.p00 = (T)c.p00;
  ph.sat_tol = (T)c.sat_tol;
  ph.sat_maxit = c.sat_maxit;
  ph.advection = c.advection;
  const T* pr = (const T*)h->profiles;
  ph.rho0 = pr;
  ph.alpha0 = pr + c.nz;
  ph.p0 = pr + 2 * c.nz;
  return ph;
}

template <typename T>
StageArgs<T> stage_args(const les_handle* h) {
  StageArgs<T> a;
  a.g = make_grid<T>(h->cfg, 8);
  a.ph = make_phys<T>(h);
  a.lc = tile_launch(a.g, h->L.max_blocks);
  a.st = h->st;
  a.prof = const_cast<Profiler*>(&h->prof);
  return a;
}

template <typename T>
SolverArgs<T> solver_args(les_handle* h) {
  SolverArgs<T> s;
  s.g = make_grid<T>(h->cfg, 8);
  s.lc = tile_launch(s.g, h->L.max_blocks);
  s.nsm = h->L.max_blocks / 8;
  s.st = h->st;
  s.op = h->cfg.poisson_op;
  s.solver = h->cfg.solver;
  s.omega = h->cfg.jacobi_omega;
  s.rho0 = (const T*)h->profiles;
  s.ctl = h->ctl;
  s.ctl_host = &h->ctl_host;
  s.partials = h->partials;
  s.r = (T*)h->fixed[B_R];
  s.p0 = (T*)h->fixed[B_PA];
  s.p1 = (T*)h->fixed[B_PB];
  s.q = (T*)h->fixed[B_Q];
  s.prof = &h->prof;
  s.bar = h->bar;
  s.fused = h->cfg.solver_path == 0 ? &h->fused : nullptr;
  s.e0 = (T*)h->fixed[B_E0];
  s.e1 = (T*)h->fixed[B_E1];
  return s;
}

// algorithmic fields read + written once per cell by one launch of each class
int fields_per_cell(const les_config& c, int id) {
  const bool fb = c.physics & LES_PHYS_FB;
  switch (id) {
    case KI_THERMO: return 6;
    case KI_RADIATION: return 3;
    // predictors (nu_t in place): scalar reads u, v, w, phi^k (2),
    // phi^{n+1/2} (2) [+ b for f_B, + radiative source], writes 2; momentum
    // reads u^k (3), u^n (3), p [+ b for buoyancy or f_B] and writes 3
    case KI_SCALAR: return 9 + (fb ? 1 : 0) + ((c.physics & LES_PHYS_RAD) ? 1 : 0);
    case KI_MOMENTUM: return 10 + ((c.physics & (LES_PHYS_BUOY | LES_PHYS_FB)) ? 1 : 0);
    case KI_RHS: return c.poisson_op == LES_OP_COMPACT ? 5 : 4;
    case KI_CORRECT: return 9;
    case KI_DIAG: return 7;
    case KI_CFL: return 3;
    case KI_APPLY: return 2;
    case KI_SUM: return 1;
    case KI_CG_INIT: return 3;
    case KI_CG_MATVEC: return 4;
    case KI_CG_UPDATE: return 6;
    case KI_JACOBI: return 3;
    case KI_FINISH: return 2;
    case KI_CG_FUSED: return 0;  // varies with the iteration count
    case KI_CG_RESIDENT: return 0;
    case KI_CG_ROLL: return 0;
    default: return 0;
  }
}

// Sec. 2.1, Eqs. 2-4: hydrostatic adiabatic reference state at the nodes
void reference_profiles(const les_config& c, const double* rho0_z, std::vector<double>& rho0,
                        std::vector<double>& p0) {
  rho0.resize(c.nz);
  p0.resize(c.nz);
  for (int k = 0; k < c.nz; ++k) {
    const double z = (k + 0.5) * c.dz;
    p0[k] = c.p00 * std::pow(1.0 - kGrav * z / (kCpd * c.theta0), kCpd / kRd);
    const double T0 = c.theta0 * std::pow(p0[k] / c.p00, kRd / kCpd);
    rho0[k] = rho0_z ? rho0_z[k] : p0[k] / (kRd * T0);
  }
}

// the oldest prefetched state becomes the state (after its copies land)
int take_prefetch(les_handle* h) {
  les_handle::Prefetch& p = h->pf[h->pf_head];
  const size_t bytes = h->n * h->es;
  cudaError_t e = cudaStreamWaitEvent(h->st, p.ready, 0);
  for (int q = 0; q < p.count && e == cudaSuccess; ++q)
    e = cudaMemcpyAsync(h->field_ptr(p.fields[q]), p.staging + (size_t)q * bytes, bytes, cudaMemcpyDeviceToDevice,
                        h->st);
  if (e == cudaSuccess) e = cudaEventRecord(h->pf_consumed, h->st);
  h->pf_head ^= 1;
  h->pf_n -= 1;
  return e == cudaSuccess ? LES_OK : h->cuda_fail(e, "prefetched state");
}

template <typename T>
int stage_begin(les_handle* h) {
  const size_t bytes = h->n * sizeof(T);
  cudaError_t e;
  if (h->pf_n > 0 && take_prefetch(h) != LES_OK) return LES_ERR_CUDA;
  auto a = stage_args<T>(h);
  if (h->dt <= 0) {
    if ((e = launch_cfl_max<T>(a, (T*)h->fixed[B_U], (T*)h->fixed[B_V], (T*)h->fixed[B_W], h->partials,
                               h->ctl)) != cudaSuccess)
      return h->cuda_fail(e, "cfl");
    if ((e = cudaMemcpyAsync(&h->ctl_host, h->ctl, sizeof(SolverCtl), cudaMemcpyDeviceToHost, h->st)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(h->st)) != cudaSuccess)
      return h->cuda_fail(e, "cfl readback");
    const double cmax = h->ctl_host.scal;
    if (!(cmax > 0) || !std::isfinite(cmax))
      return h->fail(LES_ERR_INVALID_ARG, "dt = 0 and the Courant number of the state is 0 or not finite");
    h->dt = h->cfg.cfl / cmax;
    a = stage_args<T>(h);
  }
  // u^n, phi^{n+1/2}; dp^(0) = 0
  const int thk = h->cur ? B_THB : B_THA, qtk = h->cur ? B_QTB : B_QTA;
  const int src[5] = {B_U, B_V, B_W, thk, qtk};
  const int dst[5] = {B_UN, B_VN, B_WN, B_THH, B_QTH};
  for (int q = 0; q < 5; ++q)
    if ((e = cudaMemcpyAsync(h->fixed[dst[q]], h->fixed[src[q]], bytes, cudaMemcpyDeviceToDevice, h->st)) !=
        cudaSuccess)
      return h->cuda_fail(e, "begin copy");
  if ((e = cudaMemsetAsync(h->fixed[B_PSI], 0, bytes, h->st)) != cudaSuccess) return h->cuda_fail(e, "memset");
  if ((e = launch_thermo<T>(a, (T*)h->fixed[B_THH], (T*)h->fixed[B_QTH], (T*)h->fixed[B_T],
                            (T*)h->fixed[B_QL], (T*)h->fixed[B_B], (T*)h->fixed[B_SRAD])) != cudaSuccess)
    return h->cuda_fail(e, "thermo");
  h->sub = 0;
  return LES_OK;
}

template <typename T>
int stage_scalar(les_handle* h) {
  auto a = stage_args<T>(h);
  cudaError_t e;
  T* const* F = (T* const*)h->fixed;
  const int ti = h->cur ? B_THB : B_THA, qi = h->cur ? B_QTB : B_QTA;
  const int to = h->cur ? B_THA : B_THB, qo = h->cur ? B_QTA : B_QTB;
  if (h->fused.stencil_path == 0 && pcol_eligible<T>(a.g)) {
    if ((e = launch_scalar_col<T>(a, h->L.max_blocks / 8, F[B_U], F[B_V], F[B_W], F[B_B], F[ti], F[qi], F[B_THH],
                                  F[B_QTH], F[B_SRAD], F[to], F[qo])) != cudaSuccess)
      return h->cuda_fail(e, "scalar predictor");
  } else if ((e = launch_scalar_roll<T>(a, h->L.max_blocks, F[B_U], F[B_V], F[B_W], F[B_B], F[ti], F[qi], F[B_THH],
                                        F[B_QTH], F[B_SRAD], F[to], F[qo])) != cudaSuccess) {
    return h->cuda_fail(e, "scalar predictor");
  }
  h->cur ^= 1;
  return LES_OK;
}

// the Poisson right side (Eq. pressure_correction with App. A) from u^ and psi
template <typename T>
cudaError_t launch_stage_rhs(les_handle* h, const StageArgs<T>& a) {
  T* const* F = (T* const*)h->fixed;
  if (h->fused.stencil_path == 0 && col_eligible<T>(a.g))
    return launch_rhs_col<T>(a, h->L.max_blocks, h->cfg.poisson_op, F[B_UHAT], F[B_VHAT], F[B_WHAT], F[B_PSI],
                             F[B_RHS]);
  return launch_rhs_roll<T>(a, h->L.max_blocks, h->cfg.poisson_op, F[B_UHAT], F[B_VHAT], F[B_WHAT], F[B_PSI],
                            F[B_RHS]);
}

template <typename T>
int stage_momentum(les_handle* h) {
  auto a = stage_args<T>(h);
  cudaError_t e;
  T* const* F = (T* const*)h->fixed;
  if (h->fused.stencil_path == 0 && pcol_eligible<T>(a.g)) {
    if ((e = launch_momentum_col<T>(a, h->L.max_blocks / 8, F[B_U], F[B_V], F[B_W], F[B_UN], F[B_VN], F[B_WN],
                                    F[B_P], F[B_B], F[B_UHAT], F[B_VHAT], F[B_WHAT])) != cudaSuccess)
      return h->cuda_fail(e, "momentum predictor");
  } else if ((e = launch_momentum_roll<T>(a, h->L.max_blocks, F[B_U], F[B_V], F[B_W], F[B_UN], F[B_VN], F[B_WN],
                                          F[B_P], F[B_B], F[B_UHAT], F[B_VHAT], F[B_WHAT])) != cudaSuccess) {
    return h->cuda_fail(e, "momentum predictor");
  }
  if ((e = launch_stage_rhs<T>(h, a)) != cudaSuccess) return h->cuda_fail(e, "poisson rhs");
  return LES_OK;
}

template <typename T>
int stage_solve(les_handle* h, les_step_stats* st) {
  const size_t bytes = h->n * sizeof(T);
  cudaError_t e;
  T* psi = (T*)h->fixed[B_PSI];
  const int k = std::min(h->sub, h->cfg.n_subiter - 1);
  if (h->cfg.warm_start == LES_WARM_PREV) {
    if ((e = cudaMemcpyAsync(psi, h->prev[k], bytes, cudaMemcpyDeviceToDevice, h->st)) != cudaSuccess)
      return h->cuda_fail(e, "warm start");
  } else if (h->cfg.warm_start == LES_WARM_LEARNED) {
    if (!h->model) return h->fail(LES_ERR_NO_MODEL, "learned warm start requested but no model is attached");
    std::string merr;
    const int mrc = unet_predict(h->model, h->cfg.precision, h->fixed[B_RHS], psi, h->st, &merr);
    if (mrc != LES_OK) {
      // the plain solver is the fallback: start from zero
      h->learned_fallbacks += 1;
      h->err = "learned warm start failed (" + merr + "); solved from a zero first guess";
      if ((e = cudaMemsetAsync(psi, 0, bytes, h->st)) != cudaSuccess) return h->cuda_fail(e, "memset");
    }
  } else {
    if ((e = cudaMemsetAsync(psi, 0, bytes, h->st)) != cudaSuccess) return h->cuda_fail(e, "memset");
  }
  auto s = solver_args<T>(h);
  s.guard = h->cfg.warm_start == LES_WARM_LEARNED ? 1 : 0;
  int iters = 0;
  double rel = 0;
  std::string err;
  int rc;
  if (h->cfg.precond == LES_PRECOND_LEARNED) {
    if (!h->model) return h->fail(LES_ERR_NO_MODEL, "learned preconditioner requested but no model is attached");
    int fb = 0;
    rc = poisson_solve_fcg<T>(s, h->model, (const T*)h->fixed[B_RHS], psi, h->cfg.poisson_tol, h->cfg.poisson_maxit,
                              &iters, &rel, &fb, &err);
  } else {
    rc = poisson_solve<T>(s, (const T*)h->fixed[B_RHS], psi, h->cfg.poisson_tol, h->cfg.poisson_maxit, &iters, &rel,
                          &err);
  }
  if (rc == LES_ERR_CUDA || rc == LES_ERR_NONFINITE) return h->fail(rc, err);
  if (h->cfg.warm_start == LES_WARM_PREV) {
    if ((e = cudaMemcpyAsync(h->prev[k], psi, bytes, cudaMemcpyDeviceToDevice, h->st)) != cudaSuccess)
      return h->cuda_fail(e, "warm start save");
  }
  if (st) {
    st->solves += 1;
    st->iters_total += iters;
    st->iters_max = std::max(st->iters_max, iters);
    st->res_max = std::max(st->res_max, rel);
    if (rc == LES_ERR_NOT_CONVERGED) st->not_converged += 1;
  }
  if (rc == LES_ERR_NOT_CONVERGED) h->err = "Poisson solve reached maxit";
  return rc;
}

// The solve stage over a domain decomposition: h holds the widened
// sub-domain of d (LES_DD_HALO nodes on each side in x and y).
template <typename T>
int stage_solve_dd(les_handle* h, les_dd* d, const les_dd_ops* ops, les_step_stats* st) {
  const size_t bytes = h->n * sizeof(T);
  cudaError_t e;
  auto a = stage_args<T>(h);
  // the halo of u^ is fresh now; the momentum stage's right side was not
  if ((e = launch_stage_rhs<T>(h, a)) != cudaSuccess) return h->cuda_fail(e, "poisson rhs");
  T* psi = (T*)h->fixed[B_PSI];
  const int k = std::min(h->sub, h->cfg.n_subiter - 1);
  if (h->cfg.warm_start == LES_WARM_PREV) {
    if ((e = cudaMemcpyAsync(psi, h->prev[k], bytes, cudaMemcpyDeviceToDevice, h->st)) != cudaSuccess)
      return h->cuda_fail(e, "warm start");
  } else if ((e = cudaMemsetAsync(psi, 0, bytes, h->st)) != cudaSuccess) {
    return h->cuda_fail(e, "memset");
  }
  // the decomposed CG runs on the sub-domain's own stream
  if ((e = cudaStreamSynchronize(h->st)) != cudaSuccess) return h->cuda_fail(e, "solve set-up");
  const int H = LES_DD_HALO;
  const les::DdLayout lay{(long long)H * h->cfg.nx + H, (long long)h->cfg.nx * h->cfg.ny, h->cfg.nx};
  int iters = 0;
  double rel = 0;
  std::string err;
  const int rc = les::dd_solve<T>(d, ops, (const T*)h->fixed[B_RHS], psi, lay, h->cfg.poisson_tol,
                                  h->cfg.poisson_maxit, &iters, &rel, &err);
  if (rc != LES_OK && rc != LES_ERR_NOT_CONVERGED) return h->fail(rc, err);
  if (h->cfg.warm_start == LES_WARM_PREV) {
    if ((e = cudaMemcpyAsync(h->prev[k], psi, bytes, cudaMemcpyDeviceToDevice, h->st)) != cudaSuccess)
      return h->cuda_fail(e, "warm start save");
  }
  if (st) {
    st->solves += 1;
    st->iters_total += iters;
    st->iters_max = std::max(st->iters_max, iters);
    st->res_max = std::max(st->res_max, rel);
    if (rc == LES_ERR_NOT_CONVERGED) st->not_converged += 1;
  }
  if (rc == LES_ERR_NOT_CONVERGED) h->err = "Poisson solve reached maxit";
  return rc;
}

// h is the widened sub-domain of d
bool dd_matches(const les_dd* d, const les_handle* h) {
  int nxe, nye, nz;
  les::dd_widened_shape(d, &nxe, &nye, &nz);
  const les_config& g = les::dd_config(d);
  const les_config& c = h->cfg;
  return c.nx == nxe && c.ny == nye && c.nz == nz && c.precision == g.precision && c.bc_z == g.bc_z &&
         c.dx == g.dx && c.dy == g.dy && c.dz == g.dz && c.poisson_op == LES_OP_COMPACT;
}

template <typename T>
int stage_correct(les_handle* h) {
  auto a = stage_args<T>(h);
  T* const* F = (T* const*)h->fixed;
  cudaError_t e =
      h->fused.stencil_path == 0 && col_eligible<T>(a.g)
          ? launch_correct_col<T>(a, h->L.max_blocks, F[B_UHAT], F[B_VHAT], F[B_WHAT], F[B_PSI], F[B_U], F[B_V],
                                  F[B_W], F[B_P])
          : launch_correct<T>(a, F[B_UHAT], F[B_VHAT], F[B_WHAT], F[B_PSI], F[B_U], F[B_V], F[B_W], F[B_P]);
  if (e != cudaSuccess) return h->cuda_fail(e, "correction");
  h->sub += 1;
  return LES_OK;
}

template <typename T>
int run_stage(les_handle* h, int stage, les_step_stats* st) {
  switch (stage) {
    case LES_STAGE_BEGIN: return stage_begin<T>(h);
    case LES_STAGE_SCALAR: return stage_scalar<T>(h);
    case LES_STAGE_MOMENTUM: return stage_momentum<T>(h);
    case LES_STAGE_SOLVE: return stage_solve<T>(h, st);
    case LES_STAGE_CORRECT: return stage_correct<T>(h);
    case LES_STAGE_END: return LES_OK;
    default: return h->fail(LES_ERR_INVALID_ARG, "unknown stage");
  }
}

int expected_after(const les_handle* h, int stage) {
  switch (stage) {
    case LES_STAGE_BEGIN: return LES_STAGE_SCALAR;
    case LES_STAGE_SCALAR: return LES_STAGE_MOMENTUM;
    case LES_STAGE_MOMENTUM: return LES_STAGE_SOLVE;
    case LES_STAGE_SOLVE: return LES_STAGE_CORRECT;
    case LES_STAGE_CORRECT: return h->sub >= h->cfg.n_subiter ? LES_STAGE_END : LES_STAGE_SCALAR;
    default: return LES_STAGE_BEGIN;
  }
}

int do_stage(les_handle* h, int stage, les_step_stats* st) {
  if (stage != h->next_stage)
    return h->fail(LES_ERR_STATE, "stage " + std::to_string(stage) + " called, expected " +
                                      std::to_string(h->next_stage));
  int rc = h->cfg.precision == 64 ? run_stage<double>(h, stage, st) : run_stage<float>(h, stage, st);
  if (rc == LES_OK || rc == LES_ERR_NOT_CONVERGED) h->next_stage = expected_after(h, stage);
  if (stage == LES_STAGE_END && st) st->steps += 1;
  if (st) st->dt = h->dt;
  return rc;
}

}  // namespace

namespace les {

const char* const kKernelNames[KI_COUNT] = {
    "thermo", "radiation", "scalar", "momentum", "rhs", "correct", "diag",
    "cfl", "apply", "sum", "cg_init", "cg_matvec", "cg_update", "jacobi", "finish", "ctl", "cg_fused",
    "unet_conv", "unet_wgrad", "unet_adam", "cg_resident", "cg_roll", "cg_wave", "cg_regs"};

template <typename T>
Grid<T> make_grid(const les_config& c, int zc) {
  Grid<T> g;
  g.nx = c.nx;
  g.ny = c.ny;
  g.nz = c.nz;
  g.walls = c.bc_z == LES_BC_WALLS;
  g.dx = (T)c.dx;
  g.dy = (T)c.dy;
  g.dz = (T)c.dz;
  g.idx = (T)(1.0 / c.dx);
  g.idy = (T)(1.0 / c.dy);
  g.idz = (T)(1.0 / c.dz);
  g.zc = std::max(1, std::min(zc, c.nz));
  g.ntx = (c.nx + TX - 1) / TX;
  g.nty = (c.ny + TY - 1) / TY;
  g.ntz = (c.nz + g.zc - 1) / g.zc;
  g.ntiles = (long long)g.ntx * g.nty * g.ntz;
  return g;
}

template <typename T>
LaunchCfg tile_launch(const Grid<T>& g, int max_blocks) {
  LaunchCfg lc;
  lc.block = dim3(TX, TY, 1);
  lc.grid = dim3((unsigned)std::min<long long>(g.ntiles, max_blocks), 1, 1);
  return lc;
}

template Grid<float> make_grid<float>(const les_config&, int);
template Grid<double> make_grid<double>(const les_config&, int);
template LaunchCfg tile_launch<float>(const Grid<float>&, int);
template LaunchCfg tile_launch<double>(const Grid<double>&, int);

}  // namespace les

// ============================================================================
// C ABI
// ============================================================================
extern "C" {

void les_config_default(les_config* c, int32_t nx, int32_t ny, int32_t nz) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->struct_size = sizeof(les_config);
  c->precision = 64;
  c->nx = nx;
  c->ny = ny;
  c->nz = nz;
  c->bc_z = LES_BC_PERIODIC;
  c->dx = c->dy = c->dz = 1.0;
  c->dt = 0.0;
  c->cfl = 0.3;
  c->n_subiter = 3;
  c->solver = LES_SOLVER_CG;
  c->poisson_op = LES_OP_COMPACT;
  c->warm_start = LES_WARM_ZERO;
  c->poisson_tol = 1e-10;
  c->poisson_maxit = 5000;
  c->physics = LES_PHYS_ADV | LES_PHYS_SGS;
  c->jacobi_omega = 2.0 / 3.0;
  c->cs = 0.18;  // Table 1
  c->pr = 0.4;
  c->sc = 0.4;
  c->f_cor = 7.62e-5;
  c->sponge_frac = 0.05;
  c->sponge_rate = 0.25;
  c->theta0 = 290.0;
  c->p00 = 1.0e5;
  c->sat_tol = 1e-10;
  c->sat_maxit = 20;
}

int les_workspace_bytes(const les_config* cfg, size_t* bytes) {
  std::string why;
  int rc = validate(cfg, &why);
  if (rc != LES_OK) return rc;
  if (!bytes) return LES_ERR_INVALID_ARG;
  *bytes = make_layout(*cfg, device_sms()).total;
  return LES_OK;
}

int les_init(const les_config* cfg, const double* rho0_z, void* workspace, size_t workspace_bytes, void* stream,
             les_handle** out) {
  if (!out) return LES_ERR_INVALID_ARG;
  *out = nullptr;
  std::string why;
  int rc = validate(cfg, &why);
  if (rc != LES_OK) return rc;
  if (!workspace || ((uintptr_t)workspace % kAlign) != 0) return LES_ERR_INVALID_ARG;
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, workspace) != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
    cudaGetLastError();
    return LES_ERR_INVALID_ARG;
  }
  Layout L = make_layout(*cfg, device_sms());
  if (workspace_bytes < L.total) return LES_ERR_INVALID_ARG;
  if (rho0_z) {
    for (int k = 0; k < cfg->nz; ++k)
      if (!(rho0_z[k] > 0) || !std::isfinite(rho0_z[k])) return LES_ERR_INVALID_ARG;
  }
  les_handle* h = new (std::nothrow) les_handle();
  if (h) cudaGetDevice(&h->dev);
  if (!h) return LES_ERR_INVALID_ARG;
  h->cfg = *cfg;
  h->st = (cudaStream_t)stream;
  h->ws = (char*)workspace;
  h->L = L;
  h->n = (size_t)cfg->nx * cfg->ny * cfg->nz;
  h->es = cfg->precision == 64 ? 8 : 4;
  for (int b = 0; b < B_NFIXED; ++b) h->fixed[b] = h->ws + L.off_fixed[b];
  for (size_t k = 0; k < L.off_prev.size(); ++k) h->prev.push_back(h->ws + L.off_prev[k]);
  h->profiles = h->ws + L.off_prof;
  h->ctl = (SolverCtl*)(h->ws + L.off_ctl);
  h->partials = (double*)(h->ws + L.off_partials);
  h->diag = (double*)(h->ws + L.off_diag);
  h->bar = (FusedBar*)(h->ws + L.off_bar);
  // tile shape of the persistent solver: short z runs on mid-size grids (more
  // tiles than SM slots), longer runs once the grid is large
  {
    const double cells = (double)cfg->nx * cfg->ny * cfg->nz;
    h->fused.ty = (cfg->ny % 8 == 0 && cells > 2.0e7) ? 8 : 4;
    h->fused.zc = cells > 2.0e7 ? 16 : 4;
    int dev = 0, khz = 2000000;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
    h->fused.spin_cycles = (long long)(h->fused.timeout_ms * (double)khz);
  }
  h->dt = cfg->dt;
  // reference profiles, in the field precision
  std::vector<double> rho0, p0;
  reference_profiles(*cfg, rho0_z, rho0, p0);
  std::vector<char> host(3 * (size_t)cfg->nz * h->es);
  for (int k = 0; k < cfg->nz; ++k) {
    const double v[3] = {rho0[k], 1.0 / rho0[k], p0[k]};
    for (int q = 0; q < 3; ++q) {
      if (h->es == 8) ((double*)host.data())[q * cfg->nz + k] = v[q];
      else ((float*)host.data())[q * cfg->nz + k] = (float)v[q];
    }
  }
  // no handle survives a failure here, so only the status reports it
  if (cudaMemsetAsync(h->ws, 0, L.total, h->st) != cudaSuccess ||
      cudaMemcpyAsync(h->profiles, host.data(), host.size(), cudaMemcpyHostToDevice, h->st) != cudaSuccess ||
      cudaStreamSynchronize(h->st) != cudaSuccess) {
    delete h;
    return LES_ERR_CUDA;
  }
  *out = h;
  return LES_OK;
}

void les_destroy(les_handle* h) { delete h; }

int les_set_stream(les_handle* h, void* stream) {
  if (!h) return LES_ERR_INVALID_ARG;
  h->st = (cudaStream_t)stream;
  return LES_OK;
}

int les_set_state(les_handle* h, int32_t field, const void* src, int32_t on_device) {
  if (!h) return LES_ERR_INVALID_ARG;
  void* dst = h->field_ptr(field);
  if (!dst || !src) return h->fail(LES_ERR_INVALID_ARG, "bad field id or NULL source");
  cudaError_t e = cudaMemcpyAsync(dst, src, h->n * h->es,
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->st);
  if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(h->st);
  return e == cudaSuccess ? LES_OK : h->cuda_fail(e, "set_state");
}

int les_set_states(les_handle* h, int32_t count, const int32_t* fields, const void* const* srcs,
                   int32_t on_device) {
  if (!h) return LES_ERR_INVALID_ARG;
  if (count < 0 || (count > 0 && (!fields || !srcs))) return h->fail(LES_ERR_INVALID_ARG, "bad field list");
  for (int q = 0; q < count; ++q)
    if (!h->field_ptr(fields[q]) || !srcs[q]) return h->fail(LES_ERR_INVALID_ARG, "bad field id or NULL source");
  cudaError_t e = cudaSuccess;
  for (int q = 0; q < count && e == cudaSuccess; ++q)
    e = cudaMemcpyAsync(h->field_ptr(fields[q]), srcs[q], h->n * h->es,
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->st);
  if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(h->st);
  return e == cudaSuccess ? LES_OK : h->cuda_fail(e, "set_states");
}

int les_prefetch_states(les_handle* h, int32_t count, const int32_t* fields, const void* const* srcs, void* staging,
                        void* copy_stream) {
  if (!h) return LES_ERR_INVALID_ARG;
  if (count < 1 || count > 8 || !fields || !srcs || !staging || ((uintptr_t)staging % 16) != 0)
    return h->fail(LES_ERR_INVALID_ARG, "bad prefetch arguments");
  for (int q = 0; q < count; ++q) {
    if (!h->field_ptr(fields[q]) || !srcs[q]) return h->fail(LES_ERR_INVALID_ARG, "bad field id or NULL source");
    for (int r = 0; r < q; ++r)
      if (fields[r] == fields[q]) return h->fail(LES_ERR_INVALID_ARG, "repeated field");
  }
  if (h->pf_n >= 2) return h->fail(LES_ERR_STATE, "two prefetched states are pending");
  cudaError_t e = cudaSuccess;
  if (!h->pf_consumed) e = cudaEventCreateWithFlags(&h->pf_consumed, cudaEventDisableTiming);
  les_handle::Prefetch& p = h->pf[(h->pf_head + h->pf_n) & 1];
  if (e == cudaSuccess && !p.ready) e = cudaEventCreateWithFlags(&p.ready, cudaEventDisableTiming);
  cudaStream_t cs = (cudaStream_t)copy_stream;
  // the staging buffer may be the one the last BEGIN read: wait for that read
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, h->pf_consumed, 0);
  const size_t bytes = h->n * h->es;
  for (int q = 0; q < count && e == cudaSuccess; ++q)
    e = cudaMemcpyAsync((char*)staging + (size_t)q * bytes, srcs[q], bytes, cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess) e = cudaEventRecord(p.ready, cs);
  if (e != cudaSuccess) return h->cuda_fail(e, "prefetch");
  p.staging = (const char*)staging;
  p.count = count;
  for (int q = 0; q < count; ++q) p.fields[q] = fields[q];
  h->pf_n += 1;
  return LES_OK;
}

int les_get_state(les_handle* h, int32_t field, void* dst, int32_t on_device) {
  if (!h) return LES_ERR_INVALID_ARG;
  void* src = h->field_ptr(field);
  if (!src || !dst) return h->fail(LES_ERR_INVALID_ARG, "bad field id or NULL destination");
  cudaError_t e = cudaMemcpyAsync(dst, src, h->n * h->es,
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->st);
  if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(h->st);
  return e == cudaSuccess ? LES_OK : h->cuda_fail(e, "get_state");
}

int les_field_offset(les_handle* h, int32_t field, size_t* offset) {
  if (!h || !offset) return LES_ERR_INVALID_ARG;
  void* p = h->field_ptr(field);
  if (!p) return h->fail(LES_ERR_INVALID_ARG, "bad field id");
  *offset = (size_t)((char*)p - h->ws);
  return LES_OK;
}

int les_stage(les_handle* h, int32_t stage, les_step_stats* stats) {
  if (!h) return LES_ERR_INVALID_ARG;
  return do_stage(h, stage, stats);
}

int les_step(les_handle* h, int32_t nsteps, les_step_stats* stats) {
  if (!h || nsteps < 0) return LES_ERR_INVALID_ARG;
  if (h->next_stage != LES_STAGE_BEGIN) return h->fail(LES_ERR_STATE, "a step is in progress (les_stage)");
  les_step_stats local{};
  les_step_stats* st = stats ? stats : &local;
  std::memset(st, 0, sizeof(*st));
  int worst = LES_OK;
  for (int s = 0; s < nsteps; ++s) {
    int rc = do_stage(h, LES_STAGE_BEGIN, st);
    if (rc != LES_OK) return rc;
    for (int k = 0; k < h->cfg.n_subiter; ++k) {
      const int seq[4] = {LES_STAGE_SCALAR, LES_STAGE_MOMENTUM, LES_STAGE_SOLVE, LES_STAGE_CORRECT};
      for (int q = 0; q < 4; ++q) {
        rc = do_stage(h, seq[q], st);
        if (rc == LES_ERR_NOT_CONVERGED) worst = rc;
        else if (rc != LES_OK) return rc;
      }
    }
    rc = do_stage(h, LES_STAGE_END, st);
    if (rc != LES_OK) return rc;
  }
  st->dt = h->dt;
  return worst;
}

int les_dd_step_config(const les_dd* d, les_config* out) {
  if (!d || !out) return LES_ERR_INVALID_ARG;
  int nxe, nye, nz;
  les::dd_widened_shape(d, &nxe, &nye, &nz);
  *out = les::dd_config(d);
  out->nx = nxe;
  out->ny = nye;
  return LES_OK;
}

int les_dd_halo_exchange(les_dd* d, les_handle* h, const les_dd_ops* ops, int32_t nfields, const int32_t* fields) {
  if (!d || !h || !ops || !ops->exchange || !fields) return LES_ERR_INVALID_ARG;
  if (!dd_matches(d, h)) return h->fail(LES_ERR_INVALID_ARG, "the handle is not the widened sub-domain");
  if (nfields < 1 || nfields > LES_DD_MAX_FIELDS) return h->fail(LES_ERR_INVALID_ARG, "bad field count");
  void* ptr[LES_DD_MAX_FIELDS];
  for (int q = 0; q < nfields; ++q) {
    ptr[q] = h->field_ptr(fields[q]);
    if (!ptr[q]) return h->fail(LES_ERR_INVALID_ARG, "bad field id");
    for (int r = 0; r < q; ++r)
      if (ptr[r] == ptr[q]) return h->fail(LES_ERR_INVALID_ARG, "repeated field");
  }
  std::string err;
  const int rc = les::dd_halo_exchange(d, ops, ptr, nfields, h->st, &err);
  if (rc != LES_OK) return h->fail(rc, err);
  return LES_OK;
}

int les_dd_stage_solve(les_dd* d, les_handle* h, const les_dd_ops* ops, les_step_stats* stats) {
  if (!d || !h || !ops || !ops->exchange || !ops->allreduce) return LES_ERR_INVALID_ARG;
  if (!dd_matches(d, h)) return h->fail(LES_ERR_INVALID_ARG, "the handle is not the widened sub-domain");
  if (h->cfg.warm_start == LES_WARM_LEARNED || h->cfg.precond != LES_PRECOND_NONE)
    return h->fail(LES_ERR_INVALID_ARG, "the decomposed solve has no learned warm start or preconditioner");
  if (h->next_stage != LES_STAGE_SOLVE)
    return h->fail(LES_ERR_STATE, "solve stage called, expected " + std::to_string(h->next_stage));
  const int rc = h->cfg.precision == 64 ? stage_solve_dd<double>(h, d, ops, stats)
                                        : stage_solve_dd<float>(h, d, ops, stats);
  if (rc == LES_OK || rc == LES_ERR_NOT_CONVERGED) h->next_stage = expected_after(h, LES_STAGE_SOLVE);
  if (stats) stats->dt = h->dt;
  return rc;
}

int les_ensemble_step(les_handle* const* hs, int32_t m, int32_t nsteps, les_step_stats* stats,
                      int32_t* failed) {
  if (failed) *failed = -1;
  if (!hs || m <= 0 || m > 1024 || nsteps < 0) return LES_ERR_INVALID_ARG;
  for (int i = 0; i < m; ++i) {
    if (!hs[i]) return LES_ERR_INVALID_ARG;
    for (int k = 0; k < i; ++k)
      if (hs[k] == hs[i]) return LES_ERR_INVALID_ARG;  // one thread per handle
  }
  std::vector<int> rc(m, LES_OK);
  std::vector<std::thread> workers;
  workers.reserve(m);
  for (int i = 0; i < m; ++i)
    workers.emplace_back([&, i] {
      if (cudaSetDevice(hs[i]->dev) != cudaSuccess) {
        rc[i] = LES_ERR_CUDA;
        return;
      }
      rc[i] = les_step(hs[i], nsteps, stats ? &stats[i] : nullptr);
    });
  for (auto& w : workers) w.join();
  int worst = LES_OK;
  for (int i = 0; i < m; ++i) {
    if (rc[i] == LES_OK) continue;
    if (rc[i] == LES_ERR_NOT_CONVERGED && worst == LES_OK) {
      worst = rc[i];
      if (failed) *failed = i;
    } else if (rc[i] != LES_ERR_NOT_CONVERGED) {
      if (failed) *failed = i;
      return rc[i];
    }
  }
  return worst;
}

int les_poisson_solve(les_handle* h, const void* d_rhs, void* d_x, double rtol, int32_t maxit, int32_t* iters,
                      double* rel_res) {
  if (!h || !d_rhs || !d_x || !(rtol > 0) || maxit < 0) return LES_ERR_INVALID_ARG;
  int it = 0;
  double rel = 0;
  std::string err;
  int rc;
  const bool fcg = h->cfg.precond == LES_PRECOND_LEARNED;
  if (fcg && !h->model) return h->fail(LES_ERR_NO_MODEL, "learned preconditioner requested but no model is attached");
  int fb = 0;
  if (h->cfg.precision == 64) {
    auto s = solver_args<double>(h);
    rc = fcg ? poisson_solve_fcg<double>(s, h->model, (const double*)d_rhs, (double*)d_x, rtol, maxit, &it, &rel, &fb,
                                         &err)
             : poisson_solve<double>(s, (const double*)d_rhs, (double*)d_x, rtol, maxit, &it, &rel, &err);
  } else {
    auto s = solver_args<float>(h);
    rc = fcg ? poisson_solve_fcg<float>(s, h->model, (const float*)d_rhs, (float*)d_x, rtol, maxit, &it, &rel, &fb,
                                        &err)
             : poisson_solve<float>(s, (const float*)d_rhs, (float*)d_x, rtol, maxit, &it, &rel, &err);
  }
  if (iters) *iters = it;
  if (rel_res) *rel_res = rel;
  if (rc != LES_OK) h->err = err.empty() ? "Poisson solve reached maxit" : err;
  return rc;
}

int les_apply_poisson(les_handle* h, int32_t op, const void* d_x, void* d_y) {
  if (!h || !d_x || !d_y) return LES_ERR_INVALID_ARG;
  if (op != LES_OP_COMPACT && op != LES_OP_WIDE) return h->fail(LES_ERR_INVALID_ARG, "bad operator");
  cudaError_t e;
  if (h->cfg.precision == 64) e = launch_apply<double>(solver_args<double>(h), op, (const double*)d_x, (double*)d_y);
  else e = launch_apply<float>(solver_args<float>(h), op, (const float*)d_x, (float*)d_y);
  return e == cudaSuccess ? LES_OK : h->cuda_fail(e, "apply_poisson");
}

int les_diagnostics(les_handle* h, double* out) {
  if (!h || !out) return LES_ERR_INVALID_ARG;
  cudaError_t e;
  void* const* F = h->fixed;
  const int th = h->cur ? B_THB : B_THA, qt = h->cur ? B_QTB : B_QTA;
  if (h->cfg.precision == 64) {
    auto a = stage_args<double>(h);
    e = launch_diag<double>(a, (double*)F[B_U], (double*)F[B_V], (double*)F[B_W], (double*)F[B_P], (double*)F[th],
                            (double*)F[qt], (double*)F[B_QL], h->partials, h->ctl, h->diag);
  } else {
    auto a = stage_args<float>(h);
    e = launch_diag<float>(a, (float*)F[B_U], (float*)F[B_V], (float*)F[B_W], (float*)F[B_P], (float*)F[th],
                           (float*)F[qt], (float*)F[B_QL], h->partials, h->ctl, h->diag);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, h->diag, LES_NDIAG * sizeof(double), cudaMemcpyDeviceToHost, h->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) return h->cuda_fail(e, "diagnostics");
  return out[8] > 0 ? LES_ERR_NONFINITE : LES_OK;
}

int les_get_tuning(les_handle* h, les_tuning* out) {
  if (!h || !out) return LES_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  out->struct_size = sizeof(les_tuning);
  out->cg_tile_rows = h->fused.ty;
  out->cg_tile_planes = h->fused.zc;
  out->cg_max_blocks = h->fused.max_blocks;
  out->barrier_timeout_ms = h->fused.timeout_ms;
  out->fault_missing_arrivals = h->fused.missing;
  out->stencil_path = h->fused.stencil_path;
  out->cg_variant = h->fused.variant;
  out->cg_resident = h->fused.resident;
  return LES_OK;
}

int les_set_tuning(les_handle* h, const les_tuning* in) {
  if (!h || !in) return LES_ERR_INVALID_ARG;
  if (in->struct_size != sizeof(les_tuning)) return h->fail(LES_ERR_INVALID_ARG, "les_tuning.struct_size mismatch");
  const int ty = in->cg_tile_rows;
  if (ty != 0 && ty != 1 && ty != 2 && ty != 4 && ty != 8)
    return h->fail(LES_ERR_INVALID_ARG, "cg_tile_rows must be 1, 2, 4 or 8");
  if (in->cg_tile_planes < 0 || in->cg_max_blocks < 0 || in->barrier_timeout_ms < 0 ||
      in->fault_missing_arrivals < 0)
    return h->fail(LES_ERR_INVALID_ARG, "negative tuning value");
  if (ty) h->fused.ty = ty;
  if (in->cg_tile_planes) h->fused.zc = in->cg_tile_planes;
  if (in->cg_max_blocks) h->fused.max_blocks = in->cg_max_blocks;
  if (in->barrier_timeout_ms > 0) {
    int dev = 0, khz = 2000000;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
    h->fused.timeout_ms = in->barrier_timeout_ms;
    h->fused.spin_cycles = (long long)(in->barrier_timeout_ms * (double)khz);
  }
  h->fused.missing = in->fault_missing_arrivals;
  if (in->stencil_path < 0 || in->stencil_path > 1)
    return h->fail(LES_ERR_INVALID_ARG, "stencil_path must be 0 (columns) or 1 (rolling)");
  h->fused.stencil_path = in->stencil_path;
  if (in->cg_variant < 0 || in->cg_variant > 4 || in->cg_variant == 1)
    return h->fail(LES_ERR_INVALID_ARG, "cg_variant must be 0, 2, 3 or 4");
  h->fused.variant = in->cg_variant;
  if (in->cg_resident < 0 || in->cg_resident > 2) return h->fail(LES_ERR_INVALID_ARG, "cg_resident must be 0, 1 or 2");
  h->fused.resident = in->cg_resident;
  return LES_OK;
}

int les_set_warm_model(les_handle* h, les_unet* u) {
  if (!h) return LES_ERR_INVALID_ARG;
  if (u) {
    const int n = unet_grid(u);
    if (h->cfg.nx != n || h->cfg.ny != n || h->cfg.nz != n)
      return h->fail(LES_ERR_INVALID_ARG, "the model's grid differs from the handle's");
  }
  h->model = u;
  return LES_OK;
}

int les_profile_enable(les_handle* h, int32_t enable) {
  if (!h) return LES_ERR_INVALID_ARG;
  h->prof.collect();
  h->prof.on = enable != 0;
  return LES_OK;
}

int les_profile_read(les_handle* h, les_kernel_stat* out, int32_t max_entries, int32_t* count) {
  if (!h || !out || max_entries < 0 || !count) return LES_ERR_INVALID_ARG;
  cudaError_t e = h->prof.collect();
  if (e != cudaSuccess) return h->cuda_fail(e, "profile collect");
  int c = 0;
  for (int id = 0; id < KI_COUNT && c < max_entries; ++id) {
    if (h->prof.launches[id] == 0) continue;
    les_kernel_stat& k = out[c++];
    std::memset(&k, 0, sizeof(k));
    std::strncpy(k.name, kKernelNames[id], sizeof(k.name) - 1);
    k.fields_per_cell = fields_per_cell(h->cfg, id);
    k.launches = h->prof.launches[id];
    k.timed = h->prof.timed[id];
    k.total_ms = h->prof.ms[id];
    k.bytes_per_launch = h->prof.bytes[id] > 0 ? h->prof.bytes[id] / (double)k.launches
                                               : (double)k.fields_per_cell * (double)h->n * (double)h->es;
  }
  *count = c;
  return LES_OK;
}

int les_profile_reset(les_handle* h) {
  if (!h) return LES_ERR_INVALID_ARG;
  h->prof.reset();
  return LES_OK;
}

int64_t les_launch_count(const les_handle* h) {
  if (!h) return 0;
  int64_t t = 0;
  for (int id = 0; id < KI_COUNT; ++id) t += h->prof.launches[id];
  return t;
}

double les_get_dt(const les_handle* h) { return h ? h->dt : 0.0; }

int les_set_dt(les_handle* h, double dt) {
  if (!h || !(dt > 0) || !std::isfinite(dt)) return LES_ERR_INVALID_ARG;
  h->dt = dt;
  return LES_OK;
}

const char* les_last_error(const les_handle* h) {
  if (!h) return "no handle";
  return h->err.c_str();
}

const char* les_status_string(int s) {
  if (s < 0 || s > LES_ERR_NO_MODEL) return "unknown status";
  return kStatus[s];
}

}  // extern "C"
