// les_gridsync.cuh -- grid-wide sums for persistent cooperative kernels (the
// global reductions of the conjugate-gradient solve, Sec. 2.4).
//
// Protocol: the arrival counter only grows.  At its e-th grid sum a block
// writes its block partials into slot e mod 2 of the partials array, adds
// one to the counter with release semantics and waits until the counter
// reaches (e + 1) x (arrivals per sum); then every block reads all partials
// and folds them in block order, so every block obtains the same totals
// (deterministic for a fixed grid) and no block has to publish them.  Two
// slots suffice: a block writes slot e mod 2 again only at sum e + 2, which
// it can reach only after every block has arrived at sum e + 1, i.e. after
// every block has finished reading the slot of sum e.  The slots have a
// fixed size (kSumSlot values of every block) whatever the number of values
// of a sum, so that consecutive sums of different sizes never share memory.
//
// Every wait is bounded in time: on expiry the fail flag is raised and the
// call returns false in every thread of the block, leaving the device usable.
//
// Block and grid combinations of FP32 dot products use compensated FP32
// pairs (hi + lo, Knuth's TwoSum for the exact error of each addition) and
// yield FP64 totals: on this GPU an FP64 instruction costs tens of FP32
// ones, and the compensated pair keeps about 48 significant bits.
#pragma once

#include <type_traits>

#include "les_common.cuh"
#include "les_internal.h"

namespace les {

__device__ __forceinline__ unsigned ld_volatile(const unsigned* p) {
  return *reinterpret_cast<const volatile unsigned*>(p);
}
// GPU-scope acquire load / release store and reduction: the ordering the
// grid sum needs without full membar.gl fences
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// ---- compensated FP32 pair ---------------------------------------------------
struct F2 {
  float hi, lo;
};
// a + b: TwoSum of the high parts (exact error e), low parts added to e, then
// renormalised with Fast2Sum so that |lo| <= ulp(hi) / 2
__device__ __forceinline__ F2 f2_add(F2 a, F2 b) {
  const float s = a.hi + b.hi;
  const float bp = s - a.hi;
  const float e = (a.hi - (s - bp)) + (b.hi - bp);
  const float t = e + (a.lo + b.lo);
  const float h = s + t;
  return F2{h, t - (h - s)};
}
// a += v for one FP32 term (no renormalisation: the low part only collects
// the exact rounding errors of the high part)
__device__ __forceinline__ void f2_acc(F2& a, float v) {
  const float s = a.hi + v;
  const float bp = s - a.hi;
  a.lo += (a.hi - (s - bp)) + (v - bp);
  a.hi = s;
}
__device__ __forceinline__ double f2_value(F2 a) { return (double)a.hi + (double)a.lo; }

// Per-thread accumulator of a sum of T terms.  A thread sums its own few
// dozen FP32 terms in FP32 (relative error below 1e-6 for sums of positive
// terms; CG in FP32 reaches the same iterates as with exact dots); the block
// and grid combination of the thread sums is compensated.  FP64 terms are
// summed in FP64.
template <typename T>
struct Dot;
template <>
struct Dot<float> {
  float s = 0.f;
  __device__ __forceinline__ void add(float v) { s += v; }
  __device__ __forceinline__ F2 acc() const { return F2{s, 0.f}; }
};
template <>
struct Dot<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double v) { s += v; }
  __device__ __forceinline__ double acc() const { return s; }
};

// ---- block reductions with the total broadcast to every thread ---------------
template <int NV>
__device__ __forceinline__ void block_sum_bcast(F2 (&v)[NV]) {
  __shared__ F2 sh[NV][32];
  __shared__ F2 out[NV];
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int nw = (blockDim.x * blockDim.y + 31) >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const F2 b{__shfl_xor_sync(0xffffffffu, v[q].hi, o), __shfl_xor_sync(0xffffffffu, v[q].lo, o)};
      v[q] = f2_add(v[q], b);
    }
  }
  __syncthreads();  // earlier readers of sh / out are done
  if ((tid & 31) == 0)
#pragma unroll
    for (int q = 0; q < NV; ++q) sh[q][tid >> 5] = v[q];
  __syncthreads();
  if (tid < 32) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      F2 a = tid < nw ? sh[q][tid] : F2{0.f, 0.f};
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const F2 b{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
        a = f2_add(a, b);
      }
      if (tid == 0) out[q] = a;
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = out[q];
}

template <int NV>
__device__ __forceinline__ void block_sum_bcast(double (&v)[NV]) {
  __shared__ double sh[NV][32];
  __shared__ double out[NV];
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int nw = (blockDim.x * blockDim.y + 31) >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = warp_sum(v[q]);
  __syncthreads();
  if ((tid & 31) == 0)
#pragma unroll
    for (int q = 0; q < NV; ++q) sh[q][tid >> 5] = v[q];
  __syncthreads();
  if (tid < 32) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double a = tid < nw ? sh[q][tid] : 0.0;
      a = warp_sum(a);
      if (tid == 0) out[q] = a;
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = out[q];
}

// ---- the grid sum ---------------------------------------------------------------
// Values per block in one slot of the partials array: the partials array
// holds at least 2 x kSumSlot x gridDim.x 8-byte words.
constexpr int kSumSlot = 8;
template <typename A>
__device__ __forceinline__ A* sum_slot(void* partials, unsigned epoch) {
  return reinterpret_cast<A*>(partials) + (size_t)(epoch & 1u) * kSumSlot * gridDim.x;
}

// Per-block state of the grid sums of one launch (held in registers).
struct GridSync {
  FusedBar* bar;
  void* partials;     // >= 2 x kSumSlot x gridDim.x 8-byte words
  long long spin;     // wait limit in clock cycles
  unsigned expected;  // arrivals per sum: gridDim.x (+ the test hook's missing ones)
  unsigned epoch;     // sums completed by this block
};

// arrive after this block's partials are written, wait for all arrivals
__device__ __forceinline__ bool grid_arrive_wait(GridSync& gs) {
  __shared__ int s_fail;
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  if (tid == 0) {
    s_fail = 0;
    // the release orders this block's partials (and, through the barrier
    // before it, every thread's earlier writes) before the arrival
    red_release_add(&gs.bar->count.v, 1u);
    const unsigned target = (gs.epoch + 1u) * gs.expected;
    const long long t0 = clock64();
    unsigned spins = 0;
    while ((int)(ld_acquire(&gs.bar->count.v) - target) < 0) {
      if ((++spins & 63u) == 0u && (ld_volatile(&gs.bar->fail.v) != 0u || clock64() - t0 > gs.spin)) {
        atomicExch(&gs.bar->fail.v, 1u);
        s_fail = 1;
        break;
      }
    }
  }
  __syncthreads();
  return s_fail == 0;
}

// Grid-wide sum of NV per-thread FP32-pair partials; totals in FP64.
template <int NV>
__device__ bool grid_sum(F2 (&v)[NV], GridSync& gs, double (&tot)[NV]) {
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int nthr = blockDim.x * blockDim.y;
  const unsigned G = gridDim.x;
  static_assert(NV <= kSumSlot, "too many values for one slot");
  float2* slot = sum_slot<float2>(gs.partials, gs.epoch);
  block_sum_bcast<NV>(v);
  if (tid == 0)
#pragma unroll
    for (int q = 0; q < NV; ++q) slot[(size_t)q * G + blockIdx.x] = make_float2(v[q].hi, v[q].lo);
  __syncthreads();
  if (!grid_arrive_wait(gs)) return false;
  F2 a[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    a[q] = F2{0.f, 0.f};
    for (unsigned b = tid; b < G; b += nthr) {
      const float2 p = __ldcg(slot + (size_t)q * G + b);
      a[q] = f2_add(a[q], F2{p.x, p.y});
    }
  }
  block_sum_bcast<NV>(a);
#pragma unroll
  for (int q = 0; q < NV; ++q) tot[q] = f2_value(a[q]);
  gs.epoch += 1u;
  return true;
}

// Grid-wide sum of NV per-thread FP64 partials (totals replace v).
template <int NV>
__device__ bool grid_sum(double (&v)[NV], GridSync& gs) {
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int nthr = blockDim.x * blockDim.y;
  const unsigned G = gridDim.x;
  static_assert(NV <= kSumSlot, "too many values for one slot");
  double* slot = sum_slot<double>(gs.partials, gs.epoch);
  block_sum_bcast<NV>(v);
  if (tid == 0)
#pragma unroll
    for (int q = 0; q < NV; ++q) slot[(size_t)q * G + blockIdx.x] = v[q];
  __syncthreads();
  if (!grid_arrive_wait(gs)) return false;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    double acc = 0.0;
    for (unsigned b = tid; b < G; b += nthr) acc += __ldcg(slot + (size_t)q * G + b);
    v[q] = acc;
  }
  block_sum_bcast<NV>(v);
  gs.epoch += 1u;
  return true;
}

// ---- grid sum with the totals in thread 0 only ---------------------------------
// For kernels whose scalar recurrences run in one thread: after the block
// partials are combined in shared memory, warp 0 alone posts, waits and
// folds, so the block pays two barriers per sum and no thread but thread 0
// does FP64 work.  tot[] and the return value are valid in thread 0 only;
// the caller broadcasts what it derives and must __syncthreads() before the
// next grid sum.
__device__ __forceinline__ F2 warp_sum_f2(F2 a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const F2 b{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
    a = f2_add(a, b);
  }
  return a;
}
__device__ __forceinline__ F2 acc_add(F2 a, F2 b) { return f2_add(a, b); }
__device__ __forceinline__ double acc_add(double a, double b) { return a + b; }
__device__ __forceinline__ F2 acc_warp(F2 a) { return warp_sum_f2(a); }
__device__ __forceinline__ double acc_warp(double a) { return warp_sum(a); }
__device__ __forceinline__ F2 acc_zero(F2) { return F2{0.f, 0.f}; }
__device__ __forceinline__ double acc_zero(double) { return 0.0; }
__device__ __forceinline__ double acc_value(F2 a) { return f2_value(a); }
__device__ __forceinline__ double acc_value(double a) { return a; }
// a <= b without leaving the accumulator's precision (normalised pairs:
// |lo| <= ulp(hi) / 2, so the high parts decide unless they are equal)
__device__ __forceinline__ bool acc_le(F2 a, F2 b) { return a.hi < b.hi || (a.hi == b.hi && a.lo <= b.lo); }
__device__ __forceinline__ bool acc_le(double a, double b) { return a <= b; }
// an FP64 value as an accumulator: a normalised FP32 pair, or itself
__device__ __forceinline__ void acc_from(double x, F2& a) {
  a.hi = (float)x;
  a.lo = (float)(x - (double)a.hi);
}
__device__ __forceinline__ void acc_from(double x, double& a) { a = x; }
__device__ __forceinline__ void acc_store(F2* slot, F2 a) {
  *reinterpret_cast<float2*>(slot) = make_float2(a.hi, a.lo);
}
__device__ __forceinline__ void acc_store(double* slot, double a) { *slot = a; }
__device__ __forceinline__ F2 acc_load(const F2* slot) {
  const float2 p = __ldcg(reinterpret_cast<const float2*>(slot));
  return F2{p.x, p.y};
}
__device__ __forceinline__ double acc_load(const double* slot) { return __ldcg(slot); }

struct NoWork {
  __device__ void operator()(int, int) const {}
};
// work(w, nw) runs in warps 1 .. nw-1 (w = warp - 1 of nw - 1 warps) once
// warp 0 has issued this block's release, i.e. while the grid sum is in
// flight; it must not depend on the sum.  Memory operations it starts cannot
// delay the release, which is why it waits for warp 0 (named barrier 1).
// U: partials per lane and sum loaded together when folding.  The totals
// come back as accumulators (an FP32 pair or an FP64 value) in thread 0.
template <int NV, int U = 5, typename A, typename W>
__device__ bool grid_sum_t0_acc(A (&v)[NV], GridSync& gs, A (&tot)[NV], W&& work) {
  constexpr bool kWork = !std::is_same<std::decay_t<W>, NoWork>::value;
  __shared__ A sh[NV][32];
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int lane = tid & 31, warp = tid >> 5;
  const int nw = (blockDim.x * blockDim.y + 31) >> 5;
  const unsigned G = gridDim.x;
  static_assert(NV <= kSumSlot, "too many values for one slot");
  A* slot = sum_slot<A>(gs.partials, gs.epoch);
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = acc_warp(v[q]);
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < NV; ++q) sh[q][warp] = v[q];
  // also orders every thread's earlier global writes before the release below
  __syncthreads();
  bool ok = true;
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      A a = lane < nw ? sh[q][lane] : acc_zero(v[q]);
      a = acc_warp(a);
      if (lane == 0) acc_store(slot + (size_t)q * G + blockIdx.x, a);
    }
    if (lane == 0) red_release_add(&gs.bar->count.v, 1u);
    __syncwarp();
    if (kWork && nw > 1) asm volatile("bar.arrive 1, %0;" ::"r"(nw * 32) : "memory");
    if (lane == 0) {
      const unsigned target = (gs.epoch + 1u) * gs.expected;
      const long long t0 = clock64();
      unsigned spins = 0;
      while ((int)(ld_acquire(&gs.bar->count.v) - target) < 0) {
        if ((++spins & 63u) == 0u && (ld_volatile(&gs.bar->fail.v) != 0u || clock64() - t0 > gs.spin)) {
          atomicExch(&gs.bar->fail.v, 1u);
          ok = false;
          break;
        }
      }
    }
    ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
    if (ok) {
      // the partials of all NV sums, U per lane and sum in flight at once
      // (a fold that waited for each load would pay one memory round trip
      // per 32 blocks and sum)
      A a[NV];
#pragma unroll
      for (int q = 0; q < NV; ++q) a[q] = acc_zero(v[q]);
      for (unsigned b0 = lane; b0 < G; b0 += 32 * U) {
        A w[NV][U];
#pragma unroll
        for (int q = 0; q < NV; ++q)
#pragma unroll
          for (int u = 0; u < U; ++u)
            w[q][u] = b0 + 32 * u < G ? acc_load(slot + (size_t)q * G + b0 + 32 * u) : acc_zero(v[q]);
#pragma unroll
        for (int q = 0; q < NV; ++q)
#pragma unroll
          for (int u = 0; u < U; ++u) a[q] = acc_add(a[q], w[q][u]);
      }
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        const A t = acc_warp(a[q]);
        if (lane == 0) tot[q] = t;
      }
    }
  } else if (kWork) {
    asm volatile("bar.sync 1, %0;" ::"r"(nw * 32) : "memory");
    work(warp - 1, nw - 1);
  }
  gs.epoch += 1u;
  return ok;
}
template <int NV, int U = 5, typename A, typename W>
__device__ __forceinline__ bool grid_sum_t0(A (&v)[NV], GridSync& gs, double (&tot)[NV], W&& work) {
  A t[NV];
  const bool ok = grid_sum_t0_acc<NV, U>(v, gs, t, work);
  if (threadIdx.x + blockDim.x * threadIdx.y == 0)
#pragma unroll
    for (int q = 0; q < NV; ++q) tot[q] = acc_value(t[q]);
  return ok;
}
template <int NV, int U = 5, typename A>
__device__ __forceinline__ bool grid_sum_t0(A (&v)[NV], GridSync& gs, double (&tot)[NV]) {
  return grid_sum_t0<NV, U>(v, gs, tot, NoWork{});
}

// one grid sum of a Dot<T> accumulator per value
template <int NV>
__device__ __forceinline__ bool grid_dot(Dot<float> (&d)[NV], GridSync& gs, double (&tot)[NV]) {
  F2 v[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = d[q].acc();
  return grid_sum<NV>(v, gs, tot);
}
template <int NV>
__device__ __forceinline__ bool grid_dot(Dot<double> (&d)[NV], GridSync& gs, double (&tot)[NV]) {
#pragma unroll
  for (int q = 0; q < NV; ++q) tot[q] = d[q].s;
  return grid_sum<NV>(tot, gs);
}

template <int NV, typename T, typename W>
__device__ __forceinline__ bool grid_dot_t0(Dot<T> (&d)[NV], GridSync& gs, double (&tot)[NV], W&& work) {
  decltype(d[0].acc()) v[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = d[q].acc();
  return grid_sum_t0<NV>(v, gs, tot, work);
}
template <int NV, typename T>
__device__ __forceinline__ bool grid_dot_t0(Dot<T> (&d)[NV], GridSync& gs, double (&tot)[NV]) {
  return grid_dot_t0<NV>(d, gs, tot, NoWork{});
}

}  // namespace les
