// les_common.cuh -- device-side building blocks shared by the LES kernels:
// grid description, the periodic / wall ghost rules, the 2.5-D tile walk and
// deterministic FP64 block reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "les.h"

namespace les {

// ---- tiling ---------------------------------------------------------------
// Stencil and solver kernels run thread blocks of TX x TY threads over (x, y)
// and march each thread through ZC consecutive z-planes of a tile, so that
// the plane below and above a node are still in L1 when the next node is
// processed.  Grids are capped at a multiple of the SM count and walk the
// tiles grid-stride.
constexpr int TX = 32;
constexpr int TY = 8;
constexpr int NTHREADS = TX * TY;

// z-ghost rules at the surface (k < 0) and the lid (k >= nz)
enum Ghost : int {
  G_EVEN = 0,  // mirror: scalars, pressure, psi, rho0, nu_t, b
  G_ODD = 1,   // antisymmetric: w and vertical mass fluxes
  G_UV = 2,    // horizontal velocity: free slip at the surface, no slip at the lid
};

template <typename T>
struct Grid {
  int nx, ny, nz, walls;
  T dx, dy, dz;
  T idx, idy, idz;
  int zc;          // z-planes per tile
  int ntx, nty, ntz;
  long long ntiles;

  __device__ __forceinline__ T h(int d) const { return d == 0 ? dx : (d == 1 ? dy : dz); }
  __device__ __forceinline__ T ih(int d) const { return d == 0 ? idx : (d == 1 ? idy : idz); }

  __device__ __forceinline__ int wrap(int i, int n) const {
    while (i < 0) i += n;
    while (i >= n) i -= n;
    return i;
  }
  __device__ __forceinline__ size_t lin(int i, int j, int k) const {
    return ((size_t)k * ny + j) * nx + i;
  }
  // value of f at node (i,j,k) under the periodic wrap and z-ghost rule g
  __device__ __forceinline__ T at(const T* __restrict__ f, int i, int j, int k, int g) const {
    i = wrap(i, nx);
    j = wrap(j, ny);
    T s = T(1);
    if (walls) {
      if (k < 0) {
        k = -1 - k;
        if (g == G_ODD) s = T(-1);
      } else if (k >= nz) {
        k = 2 * nz - 1 - k;
        if (g != G_EVEN) s = T(-1);
      }
    } else {
      k = wrap(k, nz);
    }
    return s * __ldg(f + lin(i, j, k));
  }
  // 1-D profile at level k (mirror with walls, wrap when periodic)
  __device__ __forceinline__ T prof(const T* __restrict__ a, int k) const {
    if (walls) {
      if (k < 0) k = -1 - k;
      if (k >= nz) k = 2 * nz - 1 - k;
    } else {
      k = wrap(k, nz);
    }
    return __ldg(a + k);
  }
  __device__ __forceinline__ bool surface_face(int d, int klower) const {
    return walls && d == 2 && klower == -1;
  }
  __device__ __forceinline__ bool wall_face(int d, int klower) const {
    return walls && d == 2 && (klower == -1 || klower == nz - 1);
  }
};

// decode tile t -> first node of the tile
template <typename T>
__device__ __forceinline__ void tile_origin(const Grid<T>& g, long long t, int& i, int& j, int& k0,
                                            int& k1) {
  int tx = (int)(t % g.ntx);
  long long r = t / g.ntx;
  int ty = (int)(r % g.nty);
  int tz = (int)(r / g.nty);
  i = tx * TX + threadIdx.x;
  j = ty * TY + threadIdx.y;
  k0 = tz * g.zc;
  k1 = min(k0 + g.zc, g.nz);
}

// ---- advection face values (Sec. 2.4) ----------------------------------------
// Value of phi on the face between nodes n and n+1 carried by the face mass
// flux F, from phi_{n-1}, phi_n, phi_{n+1}, phi_{n+2}.
//   QUICK: quadratic upstream interpolation, (-phi_{n-1} + 6 phi_n +
//          3 phi_{n+1}) / 8 for F >= 0, mirrored for F < 0.
//   WENO3 with the local Lax-Friedrichs flux: the upwind-side third-order
//          WENO reconstruction -- the candidates (3 phi_up - phi_upup) / 2 and
//          (phi_up + phi_across) / 2 blended with ideal weights 1/3, 2/3
//          scaled by 1 / (eps + beta)^2, beta the squared one-sided
//          differences, eps = 1e-6 max|phi|^2 + 1e-18 (the weights are formed
//          as d0 (eps+b1)^2 : d1 (eps+b0)^2, which stays finite in FP32).
template <typename T>
__device__ __forceinline__ T weno3_side(T fa, T fb, T fc) {
  const T q0 = T(0.5) * (T(3) * fb - fa);
  const T q1 = T(0.5) * (fb + fc);
  const T b0 = (fb - fa) * (fb - fa);
  const T b1 = (fc - fb) * (fc - fb);
  const T m = fmax(fabs(fa), fmax(fabs(fb), fabs(fc)));
  const T eps = T(1e-6) * m * m + T(1e-18);
  const T e0 = (eps + b0) * (eps + b0), e1 = (eps + b1) * (eps + b1);
  const T w0 = e1, w1 = T(2) * e0;  // (1/3)/e0 : (2/3)/e1, times 3 e0 e1
  return (w0 * q0 + w1 * q1) / (w0 + w1);
}
template <typename T>
__device__ __forceinline__ T face_value(int scheme, T F, T fm1, T f0, T f1, T f2) {
  if (scheme == LES_ADV_WENO3) return F >= T(0) ? weno3_side(fm1, f0, f1) : weno3_side(f2, f1, f0);
  return F >= T(0) ? (-fm1 + T(6) * f0 + T(3) * f1) * T(0.125) : (T(3) * f0 + T(6) * f1 - f2) * T(0.125);
}

// ---- reductions -----------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide sum (or max) in a fixed order; result valid in thread 0.
template <bool MAX>
__device__ __forceinline__ double block_reduce(double v, double* sh /* >= 32 */) {
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nthr = blockDim.x * blockDim.y * blockDim.z;
  v = MAX ? warp_max(v) : warp_sum(v);
  __syncthreads();
  if ((tid & 31) == 0) sh[tid >> 5] = v;
  __syncthreads();
  double r = 0.0;
  if (tid < 32) {
    int nw = (nthr + 31) >> 5;
    r = tid < nw ? sh[tid] : (MAX ? -1.0e300 : 0.0);
    r = MAX ? warp_max(r) : warp_sum(r);
  }
  return r;
}

// Cross-block reduction of NV values per block.  Each block stores its
// partials; the last block to arrive (atomic ticket) folds all partials in
// block order -- deterministic for a fixed grid -- and returns true in
// thread 0 with the results in out[].  The ticket is reset for the next
// launch.  maxmask bit v selects max instead of sum for value v.
template <int NV>
__device__ bool grid_reduce(const double (&v)[NV], unsigned maxmask, double* partials,
                            unsigned* ticket, double (&out)[NV]) {
  __shared__ double sh[32];
  __shared__ bool last;
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nthr = blockDim.x * blockDim.y * blockDim.z;
  const unsigned nb = gridDim.x * gridDim.y * gridDim.z;
  const unsigned bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    double r = (maxmask >> q) & 1u ? block_reduce<true>(v[q], sh) : block_reduce<false>(v[q], sh);
    if (tid == 0) partials[(size_t)q * nb + bid] = r;
  }
  if (tid == 0) {
    __threadfence();
    unsigned t = atomicAdd(ticket, 1u);
    last = (t == nb - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    const bool mx = (maxmask >> q) & 1u;
    double acc = mx ? -1.0e300 : 0.0;
    for (unsigned b = tid; b < nb; b += nthr) {
      double x = __ldcg(partials + (size_t)q * nb + b);
      acc = mx ? fmax(acc, x) : acc + x;
    }
    double r = mx ? block_reduce<true>(acc, sh) : block_reduce<false>(acc, sh);
    if (tid == 0) out[q] = r;
  }
  if (tid == 0) *ticket = 0u;
  return tid == 0;
}

// element-wise asynchronous global -> shared copies (cp.async, L1-allocating)
__device__ __forceinline__ void cp_async(float* dst, const float* src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async(double* dst, const double* src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(src) : "memory");
}
// asynchronous copies of N = 8 or 16 bytes (both addresses N-byte aligned);
// 16-byte copies bypass L1
template <int N>
__device__ __forceinline__ void cp_async_bytes(void* dst, const void* src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  if constexpr (N == 16) asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(src) : "memory");
  else asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

}  // namespace les
