// les_fcg.cu -- the pressure-correction Poisson solve (Sec. 2.4, compact
// operator of Appendix A) by flexible CG with the learned network as the
// preconditioner: the library's addition, an alternative to the learned
// first guess.
//
// The network maps a right side to an approximation of the solution, so it
// can stand for M^-1 r.  It is not linear (it normalises its input and uses
// leaky ReLUs), so the iteration is the flexible CG (Polak-Ribiere beta):
//   r_0 = b - A x_0,  z_0 = M(r_0),  p_0 = z_0
//   alpha_k = r_k.z_k / p_k.A p_k,  x += alpha_k p_k,  r_{k+1} = r_k - alpha_k A p_k
//   z_{k+1} = M(r_{k+1}),  beta_k = z_{k+1}.(r_{k+1} - r_k) / r_k.z_k,
//   p_{k+1} = z_{k+1} + beta_k p_k.
// L_c is negative semi-definite, so a preconditioner close to L_c^-1 gives
// r.M(r) < 0.  The plain iteration is the fallback and the arbiter: where
// r.M(r) is not negative (an untrained network answers 0) z = -r is used,
// which with every z so chosen gives the plain CG iterates; every solve stops
// at the same relative residual ||r|| <= tol ||b|| as the plain CG.
// One host-driven loop: each iteration reads three FP64 dot products back.
#include <algorithm>
#include <cmath>
#include <string>

#include "les_internal.h"

namespace les {
namespace {

// per-block partial sums of up to three dot products a_i . b_i (FP64)
template <typename T>
__global__ void __launch_bounds__(NTHREADS) k_fcg_dots(Grid<T> g, const T* a0, const T* b0, const T* a1, const T* b1,
                                                       const T* a2, const T* b2, int nv, double* partials) {
  __shared__ double sh[32];
  double acc[3] = {0.0, 0.0, 0.0};
  const long long n = (long long)g.nx * g.ny * g.nz;
  const int nthr = blockDim.x * blockDim.y;
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  for (long long m = (long long)blockIdx.x * nthr + tid; m < n; m += (long long)gridDim.x * nthr) {
    acc[0] += (double)a0[m] * (double)b0[m];
    if (nv > 1) acc[1] += (double)a1[m] * (double)b1[m];
    if (nv > 2) acc[2] += (double)a2[m] * (double)b2[m];
  }
  for (int v = 0; v < nv; ++v) {
    const double s = block_reduce<false>(acc[v], sh);
    if (tid == 0) partials[(size_t)v * gridDim.x + blockIdx.x] = s;
  }
}
__global__ void k_fcg_fold(const double* partials, int nblk, int nv, double* out) {
  __shared__ double sh[32];
  for (int v = 0; v < nv; ++v) {
    double a = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) a += partials[(size_t)v * nblk + b];
    const double s = block_reduce<false>(a, sh);
    if (threadIdx.x == 0) out[v] = s;
    __syncthreads();
  }
}
// y = a x + b y elementwise; with shift: y = x - shift
template <typename T>
__global__ void k_fcg_axpby(long long n, double a, const T* x, double b, T* y) {
  for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < n; m += (long long)gridDim.x * blockDim.x)
    y[m] = (T)(a * (double)x[m] + b * (double)y[m]);
}
template <typename T>
__global__ void k_fcg_shift(long long n, const T* x, double shift, T* y) {
  for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < n; m += (long long)gridDim.x * blockDim.x)
    y[m] = (T)((double)x[m] - shift);
}
template <typename T>
__global__ void k_fcg_sum(long long n, const T* x, double* partials) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < n; m += (long long)gridDim.x * blockDim.x)
    acc += (double)x[m];
  const double s = block_reduce<false>(acc, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

}  // namespace

template <typename T>
int poisson_solve_fcg(const SolverArgs<T>& a, les_unet* model, const T* b_in, T* x, double tol, int maxit,
                      int* iters, double* rel, int* fallbacks, std::string* err) {
  const long long n = (long long)a.g.nx * a.g.ny * a.g.nz;
  const unsigned nb = std::min<unsigned>(a.lc.grid.x, 1024u);
  const unsigned eb = (unsigned)std::min<long long>((n + 255) / 256, 4096);
  cudaStream_t st = a.st;
  // work vectors: b (mean-free) in q first, then q = A p; r, r_old, p, z
  T *bv = a.e1, *r = a.r, *ro = a.p0, *p = a.p1, *q = a.q, *z = a.e0;
  double host[3];
  double* sums = a.partials + 4096;  // past the block partials (at most 3 x 1024)
  cudaError_t e;
  auto fail = [&](cudaError_t ce, const char* where) {
    if (err) *err = std::string(where) + ": " + cudaGetErrorString(ce);
    return LES_ERR_CUDA;
  };
  auto dots = [&](int nv, const T* a0, const T* b0, const T* a1, const T* b1, const T* a2, const T* b2) -> cudaError_t {
    k_fcg_dots<T><<<nb, a.lc.block, 0, st>>>(a.g, a0, b0, a1, b1, a2, b2, nv, a.partials);
    k_fcg_fold<<<1, 256, 0, st>>>(a.partials, nb, nv, sums);
    cudaError_t ce = cudaMemcpyAsync(host, sums, nv * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    return ce;
  };
  // z = M(r), or -r where r.M(r) is not negative; returns r.z
  int fb = 0;
  auto precondition = [&](double rr, double* rz) -> int {
    std::string merr;
    const int mrc = unet_predict(model, sizeof(T) == 8 ? 64 : 32, r, z, st, &merr);
    double v = 0.0;
    if (mrc == LES_OK) {
      if ((e = dots(1, r, z, nullptr, nullptr, nullptr, nullptr)) != cudaSuccess) return fail(e, "fcg r.z");
      v = host[0];
    }
    if (mrc != LES_OK || !(v < 0.0) || !std::isfinite(v)) {
      fb += 1;
      if ((e = cudaMemsetAsync(z, 0, n * sizeof(T), st)) != cudaSuccess) return fail(e, "fcg fallback");
      k_fcg_axpby<T><<<eb, 256, 0, st>>>(n, -1.0, r, 0.0, z);
      v = -rr;
    }
    *rz = v;
    return LES_OK;
  };
  // mean-free b and its norm
  k_fcg_sum<T><<<nb, 256, 0, st>>>(n, b_in, a.partials);
  k_fcg_fold<<<1, 256, 0, st>>>(a.partials, nb, 1, sums);
  if ((e = cudaMemcpyAsync(host, sums, sizeof(double), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return fail(e, "fcg mean");
  k_fcg_shift<T><<<eb, 256, 0, st>>>(n, b_in, host[0] / (double)n, bv);
  if ((e = dots(1, bv, bv, nullptr, nullptr, nullptr, nullptr)) != cudaSuccess) return fail(e, "fcg |b|");
  const double bn = std::sqrt(host[0]);
  int it = 0, rc = LES_OK;
  double relres = 0.0;
  if (bn == 0.0) {
    if ((e = cudaMemsetAsync(x, 0, n * sizeof(T), st)) != cudaSuccess) return fail(e, "fcg zero");
  } else {
    // r = b - A x
    if ((e = launch_apply<T>(a, LES_OP_COMPACT, x, q)) != cudaSuccess) return fail(e, "fcg matvec");
    if ((e = cudaMemcpyAsync(r, bv, n * sizeof(T), cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
      return fail(e, "fcg copy");
    k_fcg_axpby<T><<<eb, 256, 0, st>>>(n, -1.0, q, 1.0, r);
    if ((e = dots(1, r, r, nullptr, nullptr, nullptr, nullptr)) != cudaSuccess) return fail(e, "fcg r.r");
    double rr = host[0], rz = 0.0;
    relres = std::sqrt(rr) / bn;
    if (relres > tol) {
      if (precondition(rr, &rz) != LES_OK) return LES_ERR_CUDA;
      if ((e = cudaMemcpyAsync(p, z, n * sizeof(T), cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
        return fail(e, "fcg p");
    }
    while (relres > tol && it < maxit) {
      if ((e = launch_apply<T>(a, LES_OP_COMPACT, p, q)) != cudaSuccess) return fail(e, "fcg matvec");
      if ((e = dots(1, p, q, nullptr, nullptr, nullptr, nullptr)) != cudaSuccess) return fail(e, "fcg p.q");
      const double pq = host[0];
      const double alpha = rz / pq;
      if (!(alpha > 0.0) || !std::isfinite(alpha)) {
        if (err) *err = "flexible CG breakdown: r.z / p.Ap is not positive";
        return LES_ERR_NONFINITE;
      }
      k_fcg_axpby<T><<<eb, 256, 0, st>>>(n, alpha, p, 1.0, x);
      if ((e = cudaMemcpyAsync(ro, r, n * sizeof(T), cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
        return fail(e, "fcg r_old");
      k_fcg_axpby<T><<<eb, 256, 0, st>>>(n, -alpha, q, 1.0, r);
      if ((e = dots(1, r, r, nullptr, nullptr, nullptr, nullptr)) != cudaSuccess) return fail(e, "fcg r.r");
      rr = host[0];
      ++it;
      relres = std::sqrt(rr) / bn;
      if (relres <= tol) break;
      double rz_new = 0.0;
      if (precondition(rr, &rz_new) != LES_OK) return LES_ERR_CUDA;
      // beta = z_{k+1}.(r_{k+1} - r_k) / r_k.z_k
      if ((e = dots(1, z, ro, nullptr, nullptr, nullptr, nullptr)) != cudaSuccess) return fail(e, "fcg z.r_old");
      const double beta = (rz_new - host[0]) / rz;
      k_fcg_axpby<T><<<eb, 256, 0, st>>>(n, 1.0, z, beta, p);
      rz = rz_new;
      if ((e = cudaGetLastError()) != cudaSuccess) return fail(e, "fcg update");
    }
    if (relres > tol) rc = LES_ERR_NOT_CONVERGED;
  }
  // gauge: zero mean
  k_fcg_sum<T><<<nb, 256, 0, st>>>(n, x, a.partials);
  k_fcg_fold<<<1, 256, 0, st>>>(a.partials, nb, 1, sums);
  if ((e = cudaMemcpyAsync(host, sums, sizeof(double), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return fail(e, "fcg gauge");
  k_fcg_shift<T><<<eb, 256, 0, st>>>(n, x, host[0] / (double)n, x);
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return fail(e, "fcg finish");
  if (iters) *iters = it;
  if (rel) *rel = relres;
  if (fallbacks) *fallbacks = fb;
  return rc;
}

template int poisson_solve_fcg<float>(const SolverArgs<float>&, les_unet*, const float*, float*, double, int, int*,
                                      double*, int*, std::string*);
template int poisson_solve_fcg<double>(const SolverArgs<double>&, les_unet*, const double*, double*, double, int,
                                       int*, double*, int*, std::string*);

}  // namespace les
