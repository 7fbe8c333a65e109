// les_gridsync.cuh -- grid-wide FP64 sums for persistent cooperative kernels
// (the global reductions of the conjugate-gradient solve, Sec. 2.4).
//
// Every block posts its partials; the last block to arrive folds them in
// block order (deterministic for a fixed grid), publishes the totals and
// bumps the generation that the other blocks poll.  Every wait is bounded in
// time: on expiry the fail flag is raised and the call returns false in
// every thread, leaving the device usable.
#pragma once

#include "les_common.cuh"
#include "les_internal.h"

namespace les {

__device__ __forceinline__ unsigned ld_volatile(const unsigned* p) {
  return *reinterpret_cast<const volatile unsigned*>(p);
}
// GPU-scope acquire load / release store / acq_rel fetch-add: the ordering the
// barrier needs without full membar.gl fences
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

// Grid-wide FP64 sum of NV values.  Every block posts its partials; the last
// block to arrive folds them in block order (deterministic), publishes the
// totals and bumps the generation that the others poll.  Returns false (in
// every thread) if a wait ran past its limit.
template <int NV>
__device__ bool grid_sum(double (&v)[NV], FusedBar* bar, double* partials, long long spin_cycles,
                         unsigned expected) {
  __shared__ double sh[32];
  __shared__ unsigned s_last, s_gen;
  __shared__ int s_fail;
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int nthr = blockDim.x * blockDim.y;
  const unsigned G = gridDim.x;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    const double bv = block_reduce<false>(v[q], sh);
    if (tid == 0) partials[(size_t)q * G + blockIdx.x] = bv;
  }
  if (tid == 0) {
    s_gen = ld_acquire(&bar->gen.v);
    // the arrival releases this block's partials and, for the last block,
    // acquires everybody else's
    s_last = atom_add_acq_rel(&bar->count.v, 1u) == expected - 1;
    s_fail = 0;
  }
  __syncthreads();
  if (s_last) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      // up to 8 independent loads in flight per thread, then a fixed-order sum
      double acc = 0.0;
      for (unsigned b0 = tid; b0 < G; b0 += 8 * nthr) {
        double x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const unsigned b = b0 + u * nthr;
          x[u] = b < G ? __ldcg(partials + (size_t)q * G + b) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) acc += x[u];
      }
      const double tot = block_reduce<false>(acc, sh);
      if (tid == 0) bar->value[q] = tot;
    }
    if (tid == 0) {
      bar->count.v = 0u;
      // publish the totals and the reset counter with the new generation
      st_release(&bar->gen.v, s_gen + 1u);
    }
  } else if (tid == 0) {
    const long long t0 = clock64();
    unsigned spins = 0;
    while (ld_acquire(&bar->gen.v) == s_gen) {
      if ((++spins & 63u) == 0u &&
          (ld_volatile(&bar->fail.v) != 0u || clock64() - t0 > spin_cycles)) {
        atomicExch(&bar->fail.v, 1u);
        s_fail = 1;
        break;
      }
    }
  }
  __syncthreads();
  if (s_fail) return false;
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = __ldcg(&bar->value[q]);
  return true;
}

}  // namespace les
