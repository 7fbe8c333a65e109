// les_cg_fused.cu -- the whole conjugate-gradient Poisson solve in one
// persistent cooperative launch (Sec. 2.4: L_c psi = b, compact 7-point
// Laplacian, periodic in x, y, mirror or periodic in z; mean of b removed,
// psi returned with zero mean).
//
// Why: on a mid-size grid every CG iteration is two short memory-bound passes
// separated by global reductions; as separate launches with host polling, the
// launch gaps and 4-byte-per-thread loads left the passes at a small fraction
// of memory bandwidth.  Here the grid stays resident for the whole solve:
//   phase A  p = r + beta p_old evaluated on the fly, q = L_c p, p.q
//            -- 2.5-D march: a 32 x TY thread block owns a (32 VW) x TY x zc
//            tile, keeps plane k in shared memory (with x / y halos) and
//            planes k-1, k+1 in registers, prefetching plane k+1 while
//            computing plane k; each thread handles VW = 16 B of cells;
//   phase B  x += alpha p, r -= alpha q, r.r -- 16-byte vector streaming;
// each followed by a grid-wide FP64 sum (les_gridsync.cuh): every block
// posts its partial, and once all have arrived every block folds all
// partials in block order (deterministic), so all blocks compute the same
// alpha, beta and stop decision.  Data written by other blocks is
// read with ld.global.cg (L2), never through the non-coherent L1 path.
// Every barrier wait is bounded in time; on expiry the kernel records a
// timeout in the control block and returns.
#include <algorithm>
#include <string>

#include "les_gridsync.cuh"
#include "les_internal.h"

namespace les {
namespace {

template <typename T>
struct VT {
  static constexpr int VW = 16 / sizeof(T);  // cells per 16-byte vector
  static constexpr int W = 32 * VW;          // tile width in x
};

__device__ __forceinline__ void ldv(float (&o)[4], const float* p) {
  const float4 v = __ldcg(reinterpret_cast<const float4*>(p));
  o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void ldv(double (&o)[2], const double* p) {
  const double2 v = __ldcg(reinterpret_cast<const double2*>(p));
  o[0] = v.x; o[1] = v.y;
}
__device__ __forceinline__ void stv(float* p, const float (&o)[4]) {
  __stcg(reinterpret_cast<float4*>(p), make_float4(o[0], o[1], o[2], o[3]));
}
__device__ __forceinline__ void stv(double* p, const double (&o)[2]) {
  __stcg(reinterpret_cast<double2*>(p), make_double2(o[0], o[1]));
}
// FP64 sum of VW products; float products are formed in FP32 and the 16-byte
// group is added to the FP64 accumulator (the global reduction is FP64).
__device__ __forceinline__ double vdot(const float (&a)[4], const float (&b)[4]) {
  return (double)(a[0] * b[0] + a[1] * b[1] + a[2] * b[2] + a[3] * b[3]);
}
__device__ __forceinline__ double vdot(const double (&a)[2], const double (&b)[2]) {
  return a[0] * b[0] + a[1] * b[1];
}

template <typename T>
struct FusedArgs {
  int nx, ny, nz, walls;
  T cx, cy, cz;  // 1/dx^2, 1/dy^2, 1/dz^2
  int zc, ntx, nty, ntz;
  long long ntiles;
  long long n, nv;
  const T* b;
  T* x;
  T* r;
  T* p0;
  T* p1;
  T* q;
  double* partials;  // two slots of kSumSlot words per block
  FusedBar* bar;
  SolverCtl* ctl;
  double tol;
  int maxit;
  long long spin_cycles;
  unsigned expected;
  int guard;  // arrivals per barrier: gridDim.x (+ the test hook's missing ones)
};

__device__ __forceinline__ int zmap(int k, int nz, int walls) {
  if (walls) return k < 0 ? -1 - k : (k >= nz ? 2 * nz - 1 - k : k);
  return k < 0 ? k + nz : (k >= nz ? k - nz : k);
}

// One sweep of the compact Laplacian over this block's tiles.  A tile is
// (32 VW) x TY x zc nodes; all zc + 2 planes of the operand (with the x / y
// halos of the zc interior planes) are requested at once and staged in
// shared memory, so a tile costs one round of memory latency.
// loadP(o, m): the VW operand values at linear index m; emit(m, P, q).
template <typename T, typename LoadP, typename LoadP1, typename Emit>
__device__ __forceinline__ void stencil_sweep(const FusedArgs<T>& f, T* sm, const LoadP& loadP,
                                              const LoadP1& loadP1, const Emit& emit) {
  constexpr int VW = VT<T>::VW, W = VT<T>::W;
  const int tx = threadIdx.x, ty = threadIdx.y, TY = blockDim.y;
  const int SW = W + 2, SP = (TY + 2) * SW;  // row and plane strides of the staging buffer
  for (long long t = blockIdx.x; t < f.ntiles; t += gridDim.x) {
    const int ti = (int)(t % f.ntx);
    const long long rr = t / f.ntx;
    const int tj = (int)(rr % f.nty);
    const int tk = (int)(rr / f.nty);
    const int x0 = ti * W, y0 = tj * TY, k0 = tk * f.zc, k1 = min(k0 + f.zc, f.nz);
    const int nzt = k1 - k0;
    const int xs = x0 + tx * VW, y = y0 + ty;
    const int yd = y0 == 0 ? f.ny - 1 : y0 - 1;
    const int yu = y0 + TY == f.ny ? 0 : y0 + TY;
    const int xl = x0 == 0 ? f.nx - 1 : x0 - 1;
    const int xr = x0 + W == f.nx ? 0 : x0 + W;
    auto lin = [&](int xx, int yy, int kk) -> size_t { return ((size_t)kk * f.ny + yy) * f.nx + xx; };
    __syncthreads();  // the previous tile's reads of the staging buffer are done
    // plane q of the buffer holds global plane k0 - 1 + q (ghost-mapped);
    // the loads of UNR planes are all issued before any of them is stored
    constexpr int UNR = 2;
    for (int q0 = 0; q0 < nzt + 2; q0 += UNR) {
      T c[UNR][VW], hd[UNR][VW], hu[UNR][VW], hl[UNR], hr[UNR];
#pragma unroll
      for (int u = 0; u < UNR; ++u) {
        const int q = q0 + u;
        if (q < nzt + 2) {
          const int kk = zmap(k0 - 1 + q, f.nz, f.walls);
          loadP(c[u], lin(xs, y, kk));
          if (q >= 1 && q <= nzt) {  // x / y halos only for the interior planes
            if (ty == 0) loadP(hd[u], lin(xs, yd, kk));
            if (ty == TY - 1) loadP(hu[u], lin(xs, yu, kk));
            if (tx == 0) hl[u] = loadP1(lin(xl, y, kk));
            if (tx == 31) hr[u] = loadP1(lin(xr, y, kk));
          }
        }
      }
#pragma unroll
      for (int u = 0; u < UNR; ++u) {
        const int q = q0 + u;
        if (q < nzt + 2) {
          T* row = sm + q * SP + (1 + ty) * SW + 1 + tx * VW;
#pragma unroll
          for (int e = 0; e < VW; ++e) row[e] = c[u][e];
          if (q >= 1 && q <= nzt) {
            if (ty == 0)
#pragma unroll
              for (int e = 0; e < VW; ++e) row[e - SW] = hd[u][e];
            if (ty == TY - 1)
#pragma unroll
              for (int e = 0; e < VW; ++e) row[e + SW] = hu[u][e];
            if (tx == 0) row[-1] = hl[u];
            if (tx == 31) row[VW] = hr[u];
          }
        }
      }
    }
    __syncthreads();
    for (int q = 1; q <= nzt; ++q) {
      const T* row = sm + q * SP + (1 + ty) * SW + 1 + tx * VW;
      T P[VW], qv[VW];
#pragma unroll
      for (int e = 0; e < VW; ++e) {
        const T c = row[e];
        P[e] = c;
        qv[e] = (row[e - 1] + row[e + 1] - T(2) * c) * f.cx + (row[e - SW] + row[e + SW] - T(2) * c) * f.cy +
                (row[e - SP] + row[e + SP] - T(2) * c) * f.cz;
      }
      emit(lin(xs, y, k0 + q - 1), P, qv);
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256, 2) k_cg_fused(FusedArgs<T> f) {
  constexpr int VW = VT<T>::VW;
  extern __shared__ unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const long long gstride = (long long)gridDim.x * blockDim.x * blockDim.y;
  const long long gtid = (long long)blockIdx.x * blockDim.x * blockDim.y + tid;
  GridSync gs{f.bar, f.partials, f.spin_cycles, f.expected, 0u};
  int status = 0;  // 0 running, 1 converged, 2 maxit, 3 breakdown, 4 zero rhs, 5 timeout

  // mean of b
  double s1[1] = {0.0};
  for (long long v = gtid; v < f.nv; v += gstride) {
    T bv[VW];
    ldv(bv, f.b + v * VW);
#pragma unroll
    for (int e = 0; e < VW; ++e) s1[0] += (double)bv[e];
  }
  if (!grid_sum<1>(s1, gs)) status = 5;
  const T mean = (T)(s1[0] / (double)f.n);

  // r = (b - mean) - L_c x0;  r.r and |b - mean|^2
  double s2[2] = {0.0, 0.0};
  if (!status) {
    auto loadX = [&](T (&o)[VW], size_t m) { ldv(o, f.x + m); };
    auto loadX1 = [&](size_t m) { return __ldcg(f.x + m); };
    auto emitR = [&](size_t m, const T (&P)[VW], const T (&qv)[VW]) {
      T bv[VW], rv[VW];
      ldv(bv, f.b + m);
#pragma unroll
      for (int e = 0; e < VW; ++e) {
        bv[e] -= mean;
        rv[e] = bv[e] - qv[e];
      }
      stv(f.r + m, rv);
      s2[0] += vdot(rv, rv);
      s2[1] += vdot(bv, bv);
    };
    stencil_sweep(f, sm, loadX, loadX1, emitR);
    if (!grid_sum<2>(s2, gs)) status = 5;
  }
  // the plain solver judges a learned first guess: if it leaves a larger
  // residual than x0 = 0, restart from zero (r = b - mean b, r.r = |b|^2)
  if (!status && f.guard && s2[0] > s2[1]) {
    for (long long v = gtid; v < f.nv; v += gstride) {
      T bv[VW], zv[VW];
      ldv(bv, f.b + v * VW);
#pragma unroll
      for (int e = 0; e < VW; ++e) {
        bv[e] -= mean;
        zv[e] = T(0);
      }
      stv(f.x + v * VW, zv);
      stv(f.r + v * VW, bv);
    }
    double sz[1] = {0.0};
    if (!grid_sum<1>(sz, gs)) status = 5;
    s2[0] = s2[1];
  }
  double rr = s2[0];
  const double bb = s2[1];
  double rel = 0.0;
  if (!status) {
    if (bb == 0.0) status = 4;
    else {
      rel = sqrt(rr / bb);
      if (rel <= f.tol) status = 1;
      else if (f.maxit <= 0) status = 2;
    }
  }

  int iter = 0;
  double beta = 0.0;
  bool first = true;
  T* pold = f.p0;
  T* pnew = f.p1;
  while (!status) {
    // phase A: p = r + beta p_old, q = L_c p, p.q
    double sa[1] = {0.0};
    const T tb = (T)beta;
    const T* r = f.r;
    const T* po = pold;
    T* pn = pnew;
    auto loadP = [&](T (&o)[VW], size_t m) {
      ldv(o, r + m);
      if (!first) {
        T pv[VW];
        ldv(pv, po + m);
#pragma unroll
        for (int e = 0; e < VW; ++e) o[e] += tb * pv[e];
      }
    };
    auto loadP1 = [&](size_t m) { return first ? __ldcg(r + m) : __ldcg(r + m) + tb * __ldcg(po + m); };
    auto emitQ = [&](size_t m, const T (&P)[VW], const T (&qv)[VW]) {
      stv(pn + m, P);
      stv(f.q + m, qv);
      sa[0] += vdot(P, qv);
    };
    stencil_sweep(f, sm, loadP, loadP1, emitQ);
    if (!grid_sum<1>(sa, gs)) {
      status = 5;
      break;
    }
    const double pq = sa[0];
    if (pq == 0.0 || !isfinite(pq)) {
      status = 3;
      break;
    }
    const double alpha = rr / pq;
    const T ta = (T)alpha;
    // phase B: x += alpha p, r -= alpha q, r.r
    double sb[1] = {0.0};
    constexpr int U = 2;  // vectors in flight per thread
    for (long long v0 = gtid; v0 < f.nv; v0 += U * gstride) {
      T xv[U][VW], pv[U][VW], rv[U][VW], qv[U][VW];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const long long v = v0 + u * gstride;
        if (v < f.nv) {
          const size_t m = (size_t)v * VW;
          ldv(xv[u], f.x + m);
          ldv(pv[u], pn + m);
          ldv(rv[u], f.r + m);
          ldv(qv[u], f.q + m);
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const long long v = v0 + u * gstride;
        if (v < f.nv) {
          const size_t m = (size_t)v * VW;
#pragma unroll
          for (int e = 0; e < VW; ++e) {
            xv[u][e] += ta * pv[u][e];
            rv[u][e] -= ta * qv[u][e];
          }
          stv(f.x + m, xv[u]);
          stv(f.r + m, rv[u]);
          sb[0] += vdot(rv[u], rv[u]);
        }
      }
    }
    if (!grid_sum<1>(sb, gs)) {
      status = 5;
      break;
    }
    const double rr_new = sb[0];
    iter += 1;
    rel = sqrt(rr_new / bb);
    beta = rr_new / rr;
    rr = rr_new;
    first = false;
    T* tmp = pold;
    pold = pnew;
    pnew = tmp;
    if (rel <= f.tol) status = 1;
    else if (iter >= f.maxit) status = 2;
    else if (!isfinite(rr_new)) status = 3;
  }

  // zero-mean gauge (or zero for a zero right side)
  if (status != 5) {
    double sx[1] = {0.0};
    for (long long v = gtid; v < f.nv; v += gstride) {
      T xv[VW];
      ldv(xv, f.x + v * VW);
#pragma unroll
      for (int e = 0; e < VW; ++e) sx[0] += (double)xv[e];
    }
    if (!grid_sum<1>(sx, gs)) {
      status = 5;
    } else {
      const T mx = (T)(sx[0] / (double)f.n);
      for (long long v = gtid; v < f.nv; v += gstride) {
        T xv[VW];
        ldv(xv, f.x + v * VW);
#pragma unroll
        for (int e = 0; e < VW; ++e) xv[e] = status == 4 ? T(0) : xv[e] - mx;
        stv(f.x + v * VW, xv);
      }
    }
  }
  if (blockIdx.x == 0 && tid == 0) {
    f.ctl->iter = iter;
    f.ctl->rel = rel;
    f.ctl->done = status;
  }
}


}  // namespace

template <typename T>
bool fused_cg_eligible(const Grid<T>& g, int op, int solver, int ty) {
  constexpr int W = VT<T>::W;
  return op == LES_OP_COMPACT && solver == LES_SOLVER_CG && g.nx % W == 0 && ty > 0 && g.ny % ty == 0 &&
         g.nz >= 2;
}

template <typename T>
int poisson_solve_fused(const SolverArgs<T>& a, const FusedCfg& fc, const T* b, T* x, double tol, int maxit,
                        int* iters, double* rel, std::string* err) {
  constexpr int W = VT<T>::W;
  FusedArgs<T> f;
  f.nx = a.g.nx;
  f.ny = a.g.ny;
  f.nz = a.g.nz;
  f.walls = a.g.walls;
  f.cx = a.g.idx * a.g.idx;
  f.cy = a.g.idy * a.g.idy;
  f.cz = a.g.idz * a.g.idz;
  f.zc = std::max(1, std::min(std::min(fc.zc, 32), f.nz));
  f.ntx = f.nx / W;
  f.nty = f.ny / fc.ty;
  f.ntz = (f.nz + f.zc - 1) / f.zc;
  f.ntiles = (long long)f.ntx * f.nty * f.ntz;
  f.n = (long long)f.nx * f.ny * f.nz;
  f.nv = f.n / VT<T>::VW;
  f.b = b;
  f.x = x;
  f.r = a.r;
  f.p0 = a.p0;
  f.p1 = a.p1;
  f.q = a.q;
  f.partials = a.partials;
  f.bar = a.bar;
  f.ctl = a.ctl;
  f.tol = tol;
  f.maxit = maxit;
  f.spin_cycles = fc.spin_cycles;
  const dim3 block(32, fc.ty);
  const size_t smem = (size_t)(f.zc + 2) * (fc.ty + 2) * (W + 2) * sizeof(T);
  const void* kern = (const void*)k_cg_fused<T>;
  int per_sm = 0, dev = 0, nsm = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess ||
      (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * fc.ty, smem)) != cudaSuccess) {
    if (err) *err = std::string("fused CG occupancy: ") + cudaGetErrorString(e);
    return LES_ERR_CUDA;
  }
  long long G = (long long)per_sm * nsm;
  G = std::min<long long>(G, fc.max_blocks);
  G = std::max<long long>(1, std::min<long long>(G, std::max<long long>(f.ntiles, nsm)));
  G = std::min<long long>(G, 8LL * nsm);  // the partials hold 2 x kSumSlot words of 8 blocks per SM
  f.expected = (unsigned)G + (unsigned)std::max(0, fc.missing);
  f.guard = a.guard;
  if ((e = cudaMemsetAsync(a.bar, 0, sizeof(FusedBar), a.st)) != cudaSuccess) {
    if (err) *err = std::string("fused CG barrier reset: ") + cudaGetErrorString(e);
    return LES_ERR_CUDA;
  }
  void* args[] = {&f};
  {
    ProfScope ps(a.prof, KI_CG_FUSED, a.st);
    e = cudaLaunchCooperativeKernel(kern, dim3((unsigned)G), block, args, smem, a.st);
  }
  if (e != cudaSuccess) {
    if (err) *err = std::string("fused CG launch: ") + cudaGetErrorString(e);
    return LES_ERR_CUDA;
  }
  if ((e = cudaMemcpyAsync(a.ctl_host, a.ctl, sizeof(SolverCtl), cudaMemcpyDeviceToHost, a.st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(a.st)) != cudaSuccess) {
    if (err) *err = std::string("fused CG: ") + cudaGetErrorString(e);
    return LES_ERR_CUDA;
  }
  const SolverCtl& c = *a.ctl_host;
  if (iters) *iters = c.iter;
  if (rel) *rel = c.rel;
  // algorithmic traffic of the solve (kCgIterFields per iteration; this
  // kernel streams 10: phase A r, p_old in, p, q out; phase B x, p, r, q in,
  // x, r out)
  if (a.prof) a.prof->bytes[KI_CG_FUSED] += (kCgSetupFields + kCgIterFields * c.iter) * (double)f.n * sizeof(T);
  switch (c.done) {
    case 1:
    case 4: return LES_OK;
    case 2: return LES_ERR_NOT_CONVERGED;
    case 3:
      if (err) *err = "poisson: breakdown (zero or non-finite p.Ap / residual)";
      return LES_ERR_NONFINITE;
    case 5:
      if (err) *err = "poisson: a grid barrier wait timed out";
      return LES_ERR_TIMEOUT;
    default:
      if (err) *err = "poisson: fused solver returned no status";
      return LES_ERR_CUDA;
  }
}

template bool fused_cg_eligible<float>(const Grid<float>&, int, int, int);
template bool fused_cg_eligible<double>(const Grid<double>&, int, int, int);
template int poisson_solve_fused<float>(const SolverArgs<float>&, const FusedCfg&, const float*, float*, double,
                                        int, int*, double*, std::string*);
template int poisson_solve_fused<double>(const SolverArgs<double>&, const FusedCfg&, const double*, double*,
                                         double, int, int*, double*, std::string*);

}  // namespace les
