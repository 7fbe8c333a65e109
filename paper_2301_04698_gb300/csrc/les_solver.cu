// les_solver.cu -- pressure-correction Poisson solve on sm_103a (Sec. 2.4,
// Appendix A): A psi = b with A the compact Laplacian L_c (homogeneous
// Neumann / periodic) or D(rho0 G .); the mean of b is removed first and psi
// is returned with zero mean.
//
// Conjugate gradient: one stencil kernel (p = r + beta p fused into A p and
// p.Ap) and one streaming kernel (x, r update and r.r) per iteration.  All dot
// products are FP64, reduced deterministically inside the kernels; alpha,
// beta, the residual and the stop decision stay on the device, so iterations
// are launched back to back and the host only polls the control block between
// batches.  Weighted Jacobi (the paper's solver) uses one kernel per sweep.
#include <algorithm>
#include <memory>
#include <string>

#include <condition_variable>
#include <mutex>

#include "les_internal.h"

namespace les {

// (A X)(i,j,k) for a node accessor X(i,j,k) that already applies the mirror
// (even) ghost rule in z and the periodic wrap.
template <typename T, typename X>
__device__ __forceinline__ T apply_op(const Grid<T>& g, int op, const T* __restrict__ rho0, const X& x,
                                      int i, int j, int k) {
  if (op == LES_OP_COMPACT) {
    const T c = x(i, j, k);
    return (x(i + 1, j, k) - T(2) * c + x(i - 1, j, k)) * (g.idx * g.idx) +
           (x(i, j + 1, k) - T(2) * c + x(i, j - 1, k)) * (g.idy * g.idy) +
           (x(i, j, k + 1) - T(2) * c + x(i, j, k - 1)) * (g.idz * g.idz);
  }
  // D(rho0 G x): central gradient, then central divergence; the vertical
  // component rho0 G_z x is antisymmetric across the walls.
  const T r0 = g.prof(rho0, k);
  auto gx = [&](int ii) { return r0 * (x(ii + 1, j, k) - x(ii - 1, j, k)) * (T(0.5) * g.idx); };
  auto gy = [&](int jj) { return r0 * (x(i, jj + 1, k) - x(i, jj - 1, k)) * (T(0.5) * g.idy); };
  auto gz = [&](int kk) {
    T s = T(1);
    int km = kk;
    if (g.walls) {
      if (kk < 0) {
        km = -1 - kk;
        s = T(-1);
      } else if (kk >= g.nz) {
        km = 2 * g.nz - 1 - kk;
        s = T(-1);
      }
    }
    return s * g.prof(rho0, km) * (x(i, j, km + 1) - x(i, j, km - 1)) * (T(0.5) * g.idz);
  };
  return (gx(i + 1) - gx(i - 1)) * (T(0.5) * g.idx) + (gy(j + 1) - gy(j - 1)) * (T(0.5) * g.idy) +
         (gz(k + 1) - gz(k - 1)) * (T(0.5) * g.idz);
}

template <typename T>
struct FieldX {
  Grid<T> g;
  const T* f;
  __device__ __forceinline__ T operator()(int i, int j, int k) const { return g.at(f, i, j, k, G_EVEN); }
};

// p = r + beta p_old evaluated at any node (beta = 0 on the first iteration)
template <typename T>
struct DirX {
  Grid<T> g;
  const T* r;
  const T* p;
  T beta;
  bool first;
  __device__ __forceinline__ T operator()(int i, int j, int k) const {
    const T rv = g.at(r, i, j, k, G_EVEN);
    return first ? rv : rv + beta * g.at(p, i, j, k, G_EVEN);
  }
};

template <typename T>
__global__ void __launch_bounds__(NTHREADS) k_apply(Grid<T> g, int op, const T* __restrict__ rho0,
                                                    const T* __restrict__ x, T* __restrict__ y) {
  FieldX<T> X{g, x};
  for (long long t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
    int i, j, k0, k1;
    tile_origin(g, t, i, j, k0, k1);
    if (i >= g.nx || j >= g.ny) continue;
    for (int k = k0; k < k1; ++k) y[g.lin(i, j, k)] = apply_op(g, op, rho0, X, i, j, k);
  }
}

template <typename T>
__global__ void __launch_bounds__(NTHREADS) k_sum(Grid<T> g, const T* __restrict__ x, double* partials,
                                                  SolverCtl* ctl) {
  double acc[1] = {0.0};
  for (long long t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
    int i, j, k0, k1;
    tile_origin(g, t, i, j, k0, k1);
    if (i >= g.nx || j >= g.ny) continue;
    for (int k = k0; k < k1; ++k) acc[0] += (double)x[g.lin(i, j, k)];
  }
  double res[1];
  if (grid_reduce<1>(acc, 0u, partials, &ctl->tickets[TK_SUM], res)) ctl->sum = res[0];
}

__global__ void k_ctl_reset(SolverCtl* ctl, double tol, int maxit) {
  ctl->tol = tol;
  ctl->maxit = maxit;
  ctl->iter = 0;
  ctl->done = 0;
  ctl->first = 1;
  ctl->answer = 0;
  ctl->beta = 0.0;
  ctl->alpha = 0.0;
}

// r = (b - mean b) - A x; ||b - mean b||^2, r.r; stop at once if already converged
template <typename T>
__global__ void __launch_bounds__(NTHREADS) k_init(Grid<T> g, int op, const T* __restrict__ rho0,
                                                   const T* __restrict__ b, const T* __restrict__ x,
                                                   T* __restrict__ r, double* partials, SolverCtl* ctl) {
  const double n = (double)g.nx * g.ny * g.nz;
  const T mean = (T)(ctl->sum / n);
  FieldX<T> X{g, x};
  double acc[2] = {0.0, 0.0};
  for (long long t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
    int i, j, k0, k1;
    tile_origin(g, t, i, j, k0, k1);
    if (i >= g.nx || j >= g.ny) continue;
    for (int k = k0; k < k1; ++k) {
      const size_t m = g.lin(i, j, k);
      const T bc = b[m] - mean;
      const T rv = bc - apply_op(g, op, rho0, X, i, j, k);
      r[m] = rv;
      acc[0] += (double)rv * (double)rv;
      acc[1] += (double)bc * (double)bc;
    }
  }
  double res[2];
  if (grid_reduce<2>(acc, 0u, partials, &ctl->tickets[TK_INIT], res)) {
    ctl->rr = res[0];
    ctl->bn2 = res[1];
    ctl->scal = ctl->sum / n;  // mean of b, kept for Jacobi sweeps
    if (res[1] == 0.0) {
      ctl->done = 4;
      ctl->rel = 0.0;
    } else {
      ctl->rel = sqrt(res[0] / res[1]);
      if (ctl->rel <= ctl->tol) ctl->done = 1;
      else if (ctl->maxit <= 0) ctl->done = 2;
    }
  }
}

// a learned first guess that leaves a larger residual than zero is dropped:
// x = 0, r = b - mean b (decided on the device from the init reduction)
template <typename T>
__global__ void __launch_bounds__(NTHREADS) k_guard(Grid<T> g, const T* __restrict__ b, T* __restrict__ x,
                                                    T* __restrict__ r, SolverCtl* ctl) {
  if (ctl->done || !(ctl->rr > ctl->bn2)) return;
  const T mean = (T)ctl->scal;
  for (long long t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
    int i, j, k0, k1;
    tile_origin(g, t, i, j, k0, k1);
    if (i >= g.nx || j >= g.ny) continue;
    for (int k = k0; k < k1; ++k) {
      const size_t m = g.lin(i, j, k);
      x[m] = T(0);
      r[m] = b[m] - mean;
    }
  }
}
__global__ void k_guard_fix(SolverCtl* ctl) {
  if (ctl->done || !(ctl->rr > ctl->bn2)) return;
  ctl->rr = ctl->bn2;
  ctl->rel = 1.0;
}

// CG, part 1: p_new = r + beta p_old (at all stencil nodes), q = A p_new, p_new.q
template <typename T>
__global__ void __launch_bounds__(NTHREADS) k_cg_matvec(Grid<T> g, int op, const T* __restrict__ rho0,
                                                        const T* __restrict__ r, const T* __restrict__ pold,
                                                        T* __restrict__ pnew, T* __restrict__ q,
                                                        double* partials, SolverCtl* ctl) {
  if (ctl->done) return;
  const bool first = ctl->first != 0;
  DirX<T> P{g, r, pold, (T)ctl->beta, first};
  double acc[1] = {0.0};
  for (long long t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
    int i, j, k0, k1;
    tile_origin(g, t, i, j, k0, k1);
    if (i >= g.nx || j >= g.ny) continue;
    for (int k = k0; k < k1; ++k) {
      const size_t m = g.lin(i, j, k);
      const T pv = P(i, j, k);
      const T qv = apply_op(g, op, rho0, P, i, j, k);
      pnew[m] = pv;
      q[m] = qv;
      acc[0] += (double)pv * (double)qv;
    }
  }
  double res[1];
  if (grid_reduce<1>(acc, 0u, partials, &ctl->tickets[TK_MATVEC], res)) {
    ctl->pq = res[0];
    ctl->first = 0;
    if (res[0] == 0.0 || !isfinite(res[0])) ctl->done = 3;
    else ctl->alpha = ctl->rr / res[0];
  }
}

// CG, part 2: x += alpha p, r -= alpha q, r.r -> beta, residual, stop test
template <typename T>
__global__ void __launch_bounds__(NTHREADS) k_cg_update(Grid<T> g, T* __restrict__ x, const T* __restrict__ p,
                                                        T* __restrict__ r, const T* __restrict__ q,
                                                        double* partials, SolverCtl* ctl) {
  if (ctl->done) return;
  const T alpha = (T)ctl->alpha;
  double acc[1] = {0.0};
  for (long long t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
    int i, j, k0, k1;
    tile_origin(g, t, i, j, k0, k1);
    if (i >= g.nx || j >= g.ny) continue;
    for (int k = k0; k < k1; ++k) {
      const size_t m = g.lin(i, j, k);
      x[m] += alpha * p[m];
      const T rv = r[m] - alpha * q[m];
      r[m] = rv;
      acc[0] += (double)rv * (double)rv;
    }
  }
  double res[1];
  if (grid_reduce<1>(acc, 0u, partials, &ctl->tickets[TK_UPDATE], res)) {
    const double rr_new = res[0];
    ctl->iter += 1;
    ctl->rel = sqrt(rr_new / ctl->bn2);
    ctl->beta = rr_new / ctl->rr;
    ctl->rr = rr_new;
    if (ctl->rel <= ctl->tol) ctl->done = 1;
    else if (ctl->iter >= ctl->maxit) ctl->done = 2;
    else if (!isfinite(rr_new)) ctl->done = 3;
  }
}

// weighted Jacobi sweep s: residual of x_s, x_{s+1} = x_s + omega r / diag(L_c)
template <typename T>
__global__ void __launch_bounds__(NTHREADS) k_jacobi(Grid<T> g, const T* __restrict__ b,
                                                     const T* __restrict__ xin, T* __restrict__ xout,
                                                     double omega, int sweep, double* partials,
                                                     SolverCtl* ctl) {
  if (ctl->done) return;
  const T mean = (T)ctl->scal;
  FieldX<T> X{g, xin};
  const T dxy = -T(2) * g.idx * g.idx - T(2) * g.idy * g.idy;
  double acc[1] = {0.0};
  for (long long t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
    int i, j, k0, k1;
    tile_origin(g, t, i, j, k0, k1);
    if (i >= g.nx || j >= g.ny) continue;
    for (int k = k0; k < k1; ++k) {
      const size_t m = g.lin(i, j, k);
      T dzz = -T(2) * g.idz * g.idz;
      if (g.walls && (k == 0 || k == g.nz - 1)) dzz = g.nz == 1 ? T(0) : -g.idz * g.idz;
      const T rv = (b[m] - mean) - apply_op(g, (int)LES_OP_COMPACT, (const T*)nullptr, X, i, j, k);
      xout[m] = xin[m] + (T)omega * rv / (dxy + dzz);
      acc[0] += (double)rv * (double)rv;
    }
  }
  double res[1];
  if (grid_reduce<1>(acc, 0u, partials, &ctl->tickets[TK_JACOBI], res)) {
    ctl->rel = sqrt(res[0] / ctl->bn2);
    if (ctl->rel <= ctl->tol || !isfinite(res[0])) {
      ctl->done = isfinite(res[0]) ? 1 : 3;
      ctl->answer = sweep & 1;
    } else if (sweep >= ctl->maxit) {
      ctl->done = 2;
      ctl->answer = sweep & 1;
    } else {
      ctl->iter = sweep + 1;
    }
  }
}

// x = src - mean(src) (mean from the preceding k_sum), or 0 for a zero rhs
template <typename T>
__global__ void __launch_bounds__(NTHREADS) k_finish(Grid<T> g, const T* __restrict__ src, T* __restrict__ x,
                                                     SolverCtl* ctl) {
  const double n = (double)g.nx * g.ny * g.nz;
  const bool zero = ctl->done == 4;
  const T mean = (T)(ctl->sum / n);
  for (long long t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
    int i, j, k0, k1;
    tile_origin(g, t, i, j, k0, k1);
    if (i >= g.nx || j >= g.ny) continue;
    for (int k = k0; k < k1; ++k) {
      const size_t m = g.lin(i, j, k);
      x[m] = zero ? T(0) : src[m] - mean;
    }
  }
}

template <typename T>
cudaError_t launch_apply(const SolverArgs<T>& a, int op, const T* x, T* y) {
  ProfScope ps(a.prof, KI_APPLY, a.st);
  k_apply<T><<<a.lc.grid, a.lc.block, 0, a.st>>>(a.g, op, a.rho0, x, y);
  return cudaGetLastError();
}

// Persistent CG launches spin on their own grid barrier, so every block of
// a launch must be resident at once.  Solves of different handles (ensemble
// members stepped from several host threads) share the device's SMs through
// a budget: a launch capped at B <= nsm blocks (les_tuning.cg_max_blocks)
// holds B units, an uncapped one all nsm, until it returns.  Launches whose
// caps sum to at most the SM count are then resident together (each block
// fits on an SM, and the non-persistent kernels beside them finish), and
// uncapped solves run one at a time.
struct SmBudget {
  std::mutex m;
  std::condition_variable cv;
  int used = 0;
};
SmBudget& sm_budget(int dev) {
  static SmBudget b[64];
  return b[(dev >= 0 && dev < 64) ? dev : 0];
}
class SmHold {
 public:
  SmHold(int dev, int units, int total) : b_(sm_budget(dev)), units_(std::max(1, std::min(units, total))) {
    std::unique_lock<std::mutex> lk(b_.m);
    b_.cv.wait(lk, [&] { return b_.used + units_ <= total; });
    b_.used += units_;
  }
  ~SmHold() {
    {
      std::lock_guard<std::mutex> lk(b_.m);
      b_.used -= units_;
    }
    b_.cv.notify_all();
  }
  SmHold(const SmHold&) = delete;
  SmHold& operator=(const SmHold&) = delete;

 private:
  SmBudget& b_;
  int units_;
};

template <typename T>
int poisson_solve(const SolverArgs<T>& a, const T* b, T* x, double tol, int maxit, int* iters, double* rel,
                  std::string* err) {
  // persistent CG: on chip when the grid fits there (p, r and q in
  // registers on FP32 grids 128 nodes wide, else every vector in shared
  // memory); else the
  // one-pass kernel with 64 x 16 columns (variant 4, and variant 0 for FP32
  // grids of whole columns), the two-phase streaming kernel on tile-aligned
  // grids (variant 0 or 2) or the one-pass kernel (variant 0 on other grids,
  // or variant 3).  Persistent solves of
  // different handles (ensemble members stepped from several host threads)
  // share the SMs through the budget above: capped ones run together, an
  // uncapped one alone.
  const bool cg_c = a.op == LES_OP_COMPACT && a.solver == LES_SOLVER_CG;
  std::unique_ptr<SmHold> hold;
  if (a.bar && a.fused) {
    int dev = 0;
    cudaGetDevice(&dev);
    const int nsm = std::max(1, a.nsm);
    hold.reset(new SmHold(dev, a.fused->max_blocks < nsm ? a.fused->max_blocks : nsm, nsm));
  }
  const int var = a.fused ? a.fused->variant : -1;
  const bool tiled = a.fused && fused_cg_eligible(a.g, a.op, a.solver, a.fused->ty);
  if (a.bar && cg_c && var == 0 && a.fused->resident != 1) {
    bool used = false;
    const int rc = poisson_solve_resident<T>(a, *a.fused, b, x, tol, maxit, iters, rel, err, &used);
    if (used || rc != LES_OK) return rc;
  }
  // FP32 grids of whole 64 x 16 columns: the one-pass kernel with register
  // windows is the default (1.5x the two-phase kernel on 1536^2 x 256)
  if (a.bar && cg_c && (var == 4 || (var == 0 && sizeof(T) == 4)) && wave_cg_eligible(a.g.nx, a.g.ny, a.g.nz))
    return poisson_solve_wave<T>(a, *a.fused, b, x, tol, maxit, iters, rel, err);
  if (a.bar && cg_c && (var == 3 || var == 4 || (var == 0 && !tiled)))
    return poisson_solve_roll<T>(a, *a.fused, b, x, tol, maxit, iters, rel, err);
  if (a.bar && tiled && (var == 0 || var == 2))
    return poisson_solve_fused<T>(a, *a.fused, b, x, tol, maxit, iters, rel, err);
  auto fail = [&](cudaError_t e, const char* where) {
    if (err) *err = std::string(where) + ": " + cudaGetErrorString(e);
    return LES_ERR_CUDA;
  };
  cudaError_t e;
  const dim3 G = a.lc.grid, B = a.lc.block;
  {
    ProfScope ps(a.prof, KI_CTL, a.st);
    k_ctl_reset<<<1, 1, 0, a.st>>>(a.ctl, tol, maxit);
  }
  {
    ProfScope ps(a.prof, KI_SUM, a.st);
    k_sum<T><<<G, B, 0, a.st>>>(a.g, b, a.partials, a.ctl);
  }
  {
    ProfScope ps(a.prof, KI_CG_INIT, a.st);
    k_init<T><<<G, B, 0, a.st>>>(a.g, a.op, a.rho0, b, x, a.r, a.partials, a.ctl);
  }
  if (a.guard && a.solver == LES_SOLVER_CG) {
    k_guard<T><<<G, B, 0, a.st>>>(a.g, b, x, a.r, a.ctl);
    k_guard_fix<<<1, 1, 0, a.st>>>(a.ctl);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(e, "poisson init");
  T* pbuf[2] = {a.p0, a.p1};
  T* xbuf[2] = {x, a.p0};
  int s = 0;
  int batch = 8;
  for (;;) {
    for (int q = 0; q < batch; ++q, ++s) {
      if (a.solver == LES_SOLVER_CG) {
        {
          ProfScope ps(a.prof, KI_CG_MATVEC, a.st);
          k_cg_matvec<T><<<G, B, 0, a.st>>>(a.g, a.op, a.rho0, a.r, pbuf[s & 1], pbuf[(s + 1) & 1], a.q,
                                            a.partials, a.ctl);
        }
        {
          ProfScope ps(a.prof, KI_CG_UPDATE, a.st);
          k_cg_update<T><<<G, B, 0, a.st>>>(a.g, x, pbuf[(s + 1) & 1], a.r, a.q, a.partials, a.ctl);
        }
      } else {
        ProfScope ps(a.prof, KI_JACOBI, a.st);
        k_jacobi<T><<<G, B, 0, a.st>>>(a.g, b, xbuf[s & 1], xbuf[(s + 1) & 1], a.omega, s, a.partials,
                                       a.ctl);
      }
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(e, "poisson iterate");
    if ((e = cudaMemcpyAsync(a.ctl_host, a.ctl, sizeof(SolverCtl), cudaMemcpyDeviceToHost, a.st)) !=
        cudaSuccess)
      return fail(e, "poisson poll");
    if ((e = cudaStreamSynchronize(a.st)) != cudaSuccess) return fail(e, "poisson poll");
    if (a.ctl_host->done) break;
    if (s > maxit + 2 * batch + 8) {
      if (err) *err = "poisson: solver control block did not stop";
      return LES_ERR_CUDA;
    }
    batch = std::min(batch * 2, 64);
  }
  const SolverCtl& c = *a.ctl_host;
  const T* src = (a.solver == LES_SOLVER_JACOBI && c.answer == 1) ? a.p0 : x;
  {
    ProfScope ps(a.prof, KI_SUM, a.st);
    k_sum<T><<<G, B, 0, a.st>>>(a.g, src, a.partials, a.ctl);
  }
  {
    ProfScope ps(a.prof, KI_FINISH, a.st);
    k_finish<T><<<G, B, 0, a.st>>>(a.g, src, x, a.ctl);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(e, "poisson finish");
  if (iters) *iters = c.iter;
  if (rel) *rel = c.rel;
  if (c.done == 3) {
    if (err) *err = "poisson: breakdown (zero or non-finite p.Ap / residual)";
    return LES_ERR_NONFINITE;
  }
  return c.done == 2 ? LES_ERR_NOT_CONVERGED : LES_OK;
}

template cudaError_t launch_apply<float>(const SolverArgs<float>&, int, const float*, float*);
template cudaError_t launch_apply<double>(const SolverArgs<double>&, int, const double*, double*);
template int poisson_solve<float>(const SolverArgs<float>&, const float*, float*, double, int, int*, double*,
                                  std::string*);
template int poisson_solve<double>(const SolverArgs<double>&, const double*, double*, double, int, int*,
                                   double*, std::string*);

}  // namespace les
