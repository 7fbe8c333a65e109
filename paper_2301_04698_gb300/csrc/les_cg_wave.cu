// les_cg_wave.cu -- conjugate-gradient Poisson solve in one persistent
// cooperative launch with one pass over memory and one grid-wide sum per
// iteration, for grids whose horizontal extents are multiples of 64 x 16 or
// 32 x 32 (Sec. 2.4: L_c psi = b, compact 7-point Laplacian, periodic in x, y,
// mirror or periodic in z; mean of b removed, psi returned with zero mean).
//
// The iterates are those of standard CG, formed as in the one-pass kernel of
// les_cg_roll.cu: with alpha_i and beta_i known, iteration i forms
//   p_i = r_i + beta_i p_{i-1},  q_i = L_c p_i,  x += alpha_i p_i,
//   r_{i+1} = r_i - alpha_i q_i,  w = L_c r_{i+1},
// and r'.r', r'.w, r'.q, p.q (r' = r_{i+1}) in one grid-wide sum; then
// alpha_{i+1} = r'.r' / (r'.w + 2 beta r'.q + beta^2 p.q) and
// beta_{i+1} = r'.r' / r_i.r_i (p_{i+1}.L_c p_{i+1} expanded with L_c
// symmetric), every vector formed from its definition.
//
// A block of 256 threads owns a 64 x 16 (or 32 x 32) column and marches a
// run of planes.  Each thread holds fixed positions of the column's plane
// with its halo of two (four owned nodes and two of the halo ring per
// thread) for the whole run, so the z neighbours of both stencils are
// registers: per position p on the planes f-2 .. f, r' on f-3 .. f-1 and r_i
// on f-1 .. f, where f is the plane that enters the march.  Only in-plane
// neighbours pass through shared memory (one plane of p and one of r', each
// double-buffered by plane parity).  The planes of r_i and p_{i-1} (halo
// two) and of x (owned nodes) arrive through rings filled three planes
// ahead: for an interior column as TMA boxes completing on one mbarrier per
// ring slot, for a column at a periodic edge (whose wrap is not a box) as
// per-thread cp.async copies of 16-byte chunks and node pairs.  Per plane
// step, after one block barrier:
//   A  p(f) = r(f) + beta p_old(f) at every position
//   B  q(f-1) = L_c p, r'(f-1) = r(f-1) - alpha q(f-1) within the halo of one
//   C  w(f-2) = L_c r' at the owned positions
//   D  x += alpha p, and p, r' of plane f-2 stored
// r and p are double-buffered by iteration parity (the pass reads the
// neighbours' r_i while writing r_{i+1}); the grid sum is the barrier
// between passes.  Per iteration each node is read three times (r_i,
// p_{i-1}, x) and written three times (p_i, r_{i+1}, x); the halo re-reads a
// third of r_i and p_{i-1}, mostly from L2.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdint>
#include <mutex>
#include <string>

#include <type_traits>

#include "les_gridsync.cuh"
#include "les_internal.h"

namespace les {
namespace {

constexpr int WH = 2;   // halo of the staged planes
constexpr int NT = 256;  // threads per block
constexpr int D = 4;     // r_i / p_{i-1} ring: planes f .. f+3
constexpr int DX = 6;    // x ring: planes f-2 .. f+3

// A column shape: WX x WY owned nodes (64 x 16 or 32 x 32).  Staged planes
// keep rows of SP elements with the owned columns from element 4 on (16-byte
// aligned rows, so whole 16-byte chunks are copied).  Positions per thread:
// four owned nodes (x = lane + 32 (m mod NWX), y = warp + 8 (m / NWX)) and
// two of the halo ring (two rows below and above, two columns left and
// right).
template <int WX_, int WY_>
struct Col {
  static constexpr int WX = WX_, WY = WY_;
  static constexpr int SX = WX + 2 * WH, SY = WY + 2 * WH;
  static constexpr int SP = WX + 8, SN = SP * SY;
  static constexpr int NWX = WX / 32, NWARP = NT / 32;
  static constexpr int NO = WX * WY / NT, NR = 2 * SX * WH + 2 * WH * WY, NS = NO + (NR + NT - 1) / NT;
  static_assert(NO == 4 && NS == 6 && NWARP * (NO / NWX) == WY, "column shape and thread count");
};
using Col64 = Col<64, 16>;
using Col32 = Col<32, 32>;

// the staging copies of a plane: owned rows in 16-byte chunks; each halo row
// in chunks with a pair of nodes at either end; a pair at either end of each
// owned row
template <typename T, typename C>
struct Copies {
  static constexpr int V = 16 / (int)sizeof(T);        // nodes per 16-byte chunk
  static constexpr int OC = C::WX * C::WY / V / NT;     // owned chunks per thread
  static constexpr int RC = C::WX / V + 2;              // copies per halo row
  static constexpr int NH = 2 * WH * RC + 2 * C::WY;    // halo copies per plane
  static_assert(OC * V * NT == C::WX * C::WY && NH <= NT, "copy plan");
};

template <typename T, typename C>
size_t wave_smem() {
  return ((size_t)(2 * D + 4) * C::SN + (size_t)DX * C::WX * C::WY) * sizeof(T);
}

template <typename T>
struct WaveArgs {
  // TMA descriptors of r[0], r[1], p[0], p[1] (boxes of a staged plane, SP x
  // SY x 1) and x (boxes of the owned nodes, WX x WY x 1); use_tma = 0 when
  // they could not be encoded
  CUtensorMap tm_r[2], tm_p[2], tm_x;
  int use_tma;
  int nx, ny, nz, walls;
  T cx, cy, cz;  // 1/dx^2, 1/dy^2, 1/dz^2
  int ntx, nty, zrun, nchunk;
  // runs of a block: units (column, z-run of zrun planes) u = blockIdx.x,
  // + gridDim.x, ... below nunits; then, with more columns than blocks, an
  // equal share (tail_per planes) of the tail_planes of the columns left
  int nunits, tail_planes, tail_per;
  long long n;
  const T* b;
  T* x;
  T* r[2];  // r_i in r[i & 1]
  T* p[2];  // p_i in p[i & 1]
  double* partials;
  FusedBar* bar;
  SolverCtl* ctl;
  double tol;
  int maxit;
  long long spin_cycles;
  unsigned expected;
  int guard;
};

__device__ __forceinline__ int wrapw(int i, int n) {
  while (i < 0) i += n;
  while (i >= n) i -= n;
  return i;
}
// the stored plane that stands for plane k: mirror images across the walls
// (planes beyond one image: any valid plane, unused), or periodic
__device__ __forceinline__ int zmapw(int k, int nz, int walls) {
  if (walls) {
    k = k < 0 ? -1 - k : (k >= nz ? 2 * nz - 1 - k : k);
    return k < 0 ? 0 : (k >= nz ? nz - 1 : k);
  }
  return wrapw(k, nz);
}

// Long per-thread sums: FP32 within a run of 16 planes, compensated across
template <typename T>
struct WaveSum;
template <>
struct WaveSum<float> {
  F2 s{0.f, 0.f};
  float run = 0.f;
  __device__ __forceinline__ void add(float v) { run += v; }
  __device__ __forceinline__ void flush() {
    f2_acc(s, run);
    run = 0.f;
  }
  __device__ __forceinline__ F2 acc() const { return s; }
};
template <>
struct WaveSum<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double v) { s += v; }
  __device__ __forceinline__ void flush() {}
  __device__ __forceinline__ double acc() const { return s; }
};

template <int NV, typename T>
__device__ __forceinline__ bool wave_sum_t0(WaveSum<T> (&d)[NV], GridSync& gs, double (&tot)[NV]) {
  decltype(d[0].acc()) v[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    d[q].flush();
    v[q] = d[q].acc();
  }
  return grid_sum_t0<NV, 2>(v, gs, tot);
}

// mbarrier and TMA (cp.async.bulk.tensor) helpers
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
          "r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

template <typename T, typename C>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 2 : 1) k_cg_wave(const __grid_constant__ WaveArgs<T> f) {
  constexpr int WX = C::WX, WY = C::WY, SX = C::SX, SP = C::SP, SN = C::SN;
  constexpr int NO = C::NO, NR = C::NR, NS = C::NS, NWX = C::NWX, NWARP = C::NWARP;
  extern __shared__ __align__(128) unsigned char smraw[];
  T* RINGR = reinterpret_cast<T*>(smraw);  // [D][SN] r_i as copied
  T* RINGP = RINGR + D * SN;               // [D][SN] p_{i-1} as copied
  T* PP = RINGP + D * SN;                  // [2][SN] p of a plane, by plane parity
  T* RP = PP + 2 * SN;                     // [2][SN] r' of a plane, by plane parity
  T* RINGX = RP + 2 * SN;                  // [DX][WY][WX] x of the owned nodes
  // one barrier per ring slot: the TMA copies of a plane (r_i, p_{i-1}, x)
  // complete on it; bit s of phase is the parity this thread waits for next
  __shared__ __align__(8) uint64_t bars[D];
  unsigned phase = 0;
  if (threadIdx.x == 0) {
    for (int q = 0; q < D; ++q) mbar_init(&bars[q], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  __shared__ struct {
    T ta, tb, mean;
    int status, restart;
  } sc;
  const int tid = threadIdx.x;
  const long long ncol = (long long)f.ntx * f.nty;
  const size_t plane = (size_t)f.nx * f.ny;
  const T cx = f.cx, cy = f.cy, cz = f.cz;
  GridSync gs{f.bar, f.partials, f.spin_cycles, f.expected, 0u};
  const long long gstride = (long long)gridDim.x * NT;
  const long long gtid = (long long)blockIdx.x * NT + tid;

  // the set-up and gauge sweeps in 16-byte chunks of VC nodes along x (nx is
  // a multiple of 32 and every vector 16-byte aligned here), chunks dealt to
  // the grid's threads in order
  constexpr int VC = 16 / (int)sizeof(T);
  using VQ = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  struct Ch {
    T e[VC];
  };
  auto ldch = [](const T* ptr) -> Ch {
    const VQ q = __ldcg(reinterpret_cast<const VQ*>(ptr));
    Ch c;
    if constexpr (sizeof(T) == 4) {
      c.e[0] = q.x, c.e[1] = q.y, c.e[2] = q.z, c.e[3] = q.w;
    } else {
      c.e[0] = q.x, c.e[1] = q.y;
    }
    return c;
  };
  auto stch = [](T* ptr, const Ch& c) {
    VQ q;
    if constexpr (sizeof(T) == 4) {
      q.x = c.e[0], q.y = c.e[1], q.z = c.e[2], q.w = c.e[3];
    } else {
      q.x = c.e[0], q.y = c.e[1];
    }
    __stcg(reinterpret_cast<VQ*>(ptr), q);
  };
  const int cpr = f.nx / VC;  // chunks per row
  const long long nch = f.n / VC;
  auto each_chunk = [&](auto&& body) {
    for (long long c = gtid; c < nch; c += gstride) {
      const long long rw = c / cpr;
      const int i0 = (int)(c - rw * cpr) * VC;
      body((size_t)c * VC, i0, (int)(rw % f.ny), (int)(rw / f.ny));
    }
  };
  // the 7-point operator at a chunk's nodes straight from global memory
  // (set-up sweeps only), and the chunk's own values
  auto lap_chunk = [&](const T* v, size_t m, int i0, int j, int k, Ch& lap, Ch& own) {
    const size_t row = (size_t)k * plane + (size_t)j * f.nx;
    own = ldch(v + m);
    const T xl = __ldcg(v + row + wrapw(i0 - 1, f.nx)), xr = __ldcg(v + row + wrapw(i0 + VC, f.nx));
    const Ch ym = ldch(v + (size_t)k * plane + (size_t)wrapw(j - 1, f.ny) * f.nx + i0);
    const Ch yp = ldch(v + (size_t)k * plane + (size_t)wrapw(j + 1, f.ny) * f.nx + i0);
    const Ch zm = ldch(v + (size_t)zmapw(k - 1, f.nz, f.walls) * plane + (size_t)j * f.nx + i0);
    const Ch zp = ldch(v + (size_t)zmapw(k + 1, f.nz, f.walls) * plane + (size_t)j * f.nx + i0);
#pragma unroll
    for (int q = 0; q < VC; ++q) {
      const T c2 = T(2) * own.e[q];
      const T xm = q == 0 ? xl : own.e[q - 1], xp = q == VC - 1 ? xr : own.e[q + 1];
      lap.e[q] = (xm + xp - c2) * cx + (ym.e[q] + yp.e[q] - c2) * cy + (zm.e[q] + zp.e[q] - c2) * cz;
    }
  };

  double rr = 0.0, bb = 0.0, rel = 0.0, pq = 0.0;  // meaningful in thread 0
  int status = 0;  // 0 running, 1 converged, 2 maxit, 3 breakdown, 4 zero rhs, 5 timeout

  // ---- set-up: mean of b ---------------------------------------------------------
  {
    WaveSum<T> s[1];
    int cnt = 0;
    for (long long c = gtid; c < nch; c += gstride) {
      const Ch bq = ldch(f.b + (size_t)c * VC);
#pragma unroll
      for (int q = 0; q < VC; ++q) s[0].add(bq.e[q]);
      if ((++cnt & 3) == 0) s[0].flush();
    }
    double t[1];
    const bool ok = wave_sum_t0<1>(s, gs, t);
    if (tid == 0) {
      sc.status = ok ? 0 : 5;
      sc.mean = (T)(t[0] / (double)f.n);
    }
    __syncthreads();
    status = sc.status;
  }
  const T mean = sc.mean;
  // ---- r_0 = (b - mean) - L_c x0 into r[0]; r.r and |b - mean|^2 ----------------
  if (!status) {
    WaveSum<T> s[2];
    int cnt = 0;
    each_chunk([&](size_t m, int i0, int j, int k) {
      Ch lap, xo;
      lap_chunk(f.x, m, i0, j, k, lap, xo);
      const Ch bq = ldch(f.b + m);
      Ch rq;
#pragma unroll
      for (int q = 0; q < VC; ++q) {
        const T bm = bq.e[q] - mean;
        const T rv = bm - lap.e[q];
        rq.e[q] = rv;
        s[0].add(rv * rv);
        s[1].add(bm * bm);
      }
      stch(f.r[0] + m, rq);
      if ((++cnt & 3) == 0) {
        s[0].flush();
        s[1].flush();
      }
    });
    double t[2];
    const bool ok = wave_sum_t0<2>(s, gs, t);
    if (tid == 0) {
      // the plain solver judges a learned first guess: if it leaves a larger
      // residual than x0 = 0, restart from zero (r = b - mean b, r.r = |b|^2)
      sc.status = ok ? 0 : 5;
      sc.restart = ok && f.guard && t[0] > t[1];
      rr = sc.restart ? t[1] : t[0];
      bb = t[1];
    }
    __syncthreads();
    status = sc.status;
    if (!status && sc.restart) {
      for (long long m = gtid; m < f.n; m += gstride) {
        __stcg(f.x + m, T(0));
        __stcg(f.r[0] + m, __ldcg(f.b + m) - mean);
      }
      WaveSum<T> none[1];
      double t1[1];
      const bool ok2 = wave_sum_t0<1>(none, gs, t1);  // a grid barrier: r_0 complete everywhere
      if (tid == 0) sc.status = ok2 ? 0 : 5;
      __syncthreads();
      status = sc.status;
    }
  }
  if (tid == 0) {
    if (!status) {
      if (bb == 0.0) status = 4;
      else {
        rel = sqrt(rr / bb);
        if (rel <= f.tol) status = 1;
        else if (f.maxit <= 0) status = 2;
      }
    }
    sc.status = status;
  }
  __syncthreads();
  status = sc.status;
  // ---- p_0 = r_0: r_0 . L_c r_0 gives alpha_0 --------------------------------------
  if (!status) {
    WaveSum<T> s[1];
    int cnt = 0;
    each_chunk([&](size_t m, int i0, int j, int k) {
      Ch lap, ro;
      lap_chunk(f.r[0], m, i0, j, k, lap, ro);
#pragma unroll
      for (int q = 0; q < VC; ++q) s[0].add(ro.e[q] * lap.e[q]);
      if ((++cnt & 3) == 0) s[0].flush();
    });
    double t[1];
    const bool ok = wave_sum_t0<1>(s, gs, t);
    if (tid == 0) {
      pq = t[0];
      if (!ok) status = 5;
      else if (pq == 0.0 || !isfinite(pq)) status = 3;
      else {
        sc.ta = (T)(rr / pq);
        sc.tb = T(0);
      }
      sc.status = status;
    }
    __syncthreads();
    status = sc.status;
  }

  // ---- iterations ----------------------------------------------------------------
  int iter = 0;
  while (!status) {
    const T ta = sc.ta, tb = sc.tb;
    const bool first = iter == 0;
    const T* ri = f.r[iter & 1];
    T* ro = f.r[(iter + 1) & 1];
    const T* pold = f.p[(iter + 1) & 1];  // p_{i-1}
    T* pw = f.p[iter & 1];
    WaveSum<T> s[4];  // r'.r', r'.w, r'.q, p.q
    int u = blockIdx.x;
    int ts = (int)blockIdx.x * f.tail_per, te = min(ts + f.tail_per, f.tail_planes);
    for (;;) {
      int col, k0, k1;
      if (u < f.nunits) {
        col = u % (int)ncol;
        k0 = (u / (int)ncol) * f.zrun;
        k1 = min(k0 + f.zrun, f.nz);
        u += gridDim.x;
      } else if (ts < te) {  // the units are whole columns here
        col = f.nunits + ts / f.nz;
        k0 = ts % f.nz;
        k1 = min(f.nz, k0 + (te - ts));
        ts += k1 - k0;
      } else {
        break;
      }
      const int x0 = (col % f.ntx) * WX, y0 = (col / f.ntx) * WY;
      // this thread's positions: index in a staged plane, in-plane global
      // offset; the halo slots' classes (valid, within the halo of one)
      // (owned slots: a base plus constants, x = lane + 32 (m mod NWX),
      // y = warp + 8 (m / NWX))
      int esr[NS - NO] = {};  // halo slots
      unsigned valid = (1u << NO) - 1u, in1 = (1u << NO) - 1u;
      const int go0 = (y0 + (tid >> 5)) * f.nx + x0 + (tid & 31);  // global offset of owned slot 0
      const int eo0 = ((tid >> 5) + WH) * SP + (tid & 31) + 4;      // staged index of owned slot 0
      auto es = [&](int m) { return m < NO ? eo0 + NWARP * (m / NWX) * SP + 32 * (m % NWX) : esr[m - NO]; };
#pragma unroll
      for (int m = NO; m < NS; ++m) {
        int ex, ey;
        {
          const int j = tid + (m - NO) * NT;
          if (j < 2 * SX * WH) {  // the two rows below and the two above
            const int top = j >= SX * WH;
            const int jj = j - top * SX * WH;
            ey = (top ? WY : -WH) + jj / SX;
            ex = jj % SX - WH;
          } else {  // two columns left and right of the owned rows
            const int jj = min(j - 2 * SX * WH, 4 * WY - 1);
            const int c = jj & 3;
            ey = jj >> 2;
            ex = c < 2 ? c - WH : WX - 2 + c;
          }
          if (j < NR) {
            valid |= 1u << m;
            if (ex >= -1 && ex <= WX && ey >= -1 && ey <= WY) in1 |= 1u << m;
          }
        }
        esr[m - NO] = (ey + WH) * SP + (ex + 4);
      }
      // interior columns take TMA boxes (the periodic wrap of an edge column
      // is not a box); the others take per-thread copies
      const bool tma = f.use_tma && x0 >= 4 && x0 + WX + 4 <= f.nx && y0 >= WH && y0 + WY + WH <= f.ny;
      // this thread's staging copies (shared and in-plane global offsets)
      using CP = Copies<T, C>;
      int od[CP::OC], os[CP::OC];
#pragma unroll
      for (int j = 0; j < CP::OC; ++j) {
        const int c = tid + j * NT, ey = c / (WX / CP::V), ex = (c % (WX / CP::V)) * CP::V;
        od[j] = (ey + WH) * SP + ex + 4;  // in a staged plane; x rows are dense: ey WX + ex
        os[j] = (y0 + ey) * f.nx + x0 + ex;
      }
      int hd = 0, hs = 0, hk = 0;  // halo copy: kind 0 none, 1 a pair of nodes, 2 a chunk
      if (tid < CP::NH) {
        int ey, ex;
        if (tid < 2 * WH * CP::RC) {
          const int r = tid / CP::RC, j = tid % CP::RC;
          ey = r < WH ? r - WH : WY + r - WH;
          ex = j == 0 ? -WH : (j == CP::RC - 1 ? WX : (j - 1) * CP::V);
          hk = (j == 0 || j == CP::RC - 1) ? 1 : 2;
        } else {
          const int c = tid - 2 * WH * CP::RC;
          ey = c >> 1;
          ex = (c & 1) ? WX : -WH;
          hk = 1;
        }
        hd = (ey + WH) * SP + ex + 4;
        hs = wrapw(y0 + ey, f.ny) * f.nx + wrapw(x0 + ex, f.nx);
      }
      // plane kk of r_i, p_{i-1} (every position) and of x (owned positions,
      // planes of the run) into their ring slots; one commit group per plane
      auto fetch = [&](int kk) {
        const int zs = zmapw(kk, f.nz, f.walls);
        const size_t base = (size_t)zs * plane;
        const int slot = (kk + 2 * D) % D;
        T* rr_ = RINGR + slot * SN;
        T* pp_ = RINGP + slot * SN;
        T* xx_ = RINGX + ((kk + 2 * DX) % DX) * (WX * WY);
        const bool xrun = kk >= k0 && kk < k1;
        if (tma) {
          if (tid == 0) {
            const unsigned bytes = (unsigned)((first ? 1 : 2) * SN * sizeof(T) + (xrun ? WX * WY * sizeof(T) : 0));
            mbar_expect_tx(&bars[slot], bytes);
            tma_load_3d(rr_, &f.tm_r[iter & 1], x0 - 4, y0 - WH, zs, &bars[slot]);
            if (!first) tma_load_3d(pp_, &f.tm_p[(iter + 1) & 1], x0 - 4, y0 - WH, zs, &bars[slot]);
            if (xrun) tma_load_3d(xx_, &f.tm_x, x0, y0, kk, &bars[slot]);
          }
          return;
        }
        const T* rs = ri + base;
        const T* ps = pold + base;
        const T* xs = f.x + base;
#pragma unroll
        for (int j = 0; j < CP::OC; ++j) {
          const int c = tid + j * NT;
          cp_async_bytes<16>(rr_ + od[j], rs + os[j]);
          if (!first) cp_async_bytes<16>(pp_ + od[j], ps + os[j]);
          if (xrun) cp_async_bytes<16>(xx_ + (c / (WX / CP::V)) * WX + (c % (WX / CP::V)) * CP::V, xs + os[j]);
        }
        if (hk == 2) {
          cp_async_bytes<16>(rr_ + hd, rs + hs);
          if (!first) cp_async_bytes<16>(pp_ + hd, ps + hs);
        } else if (hk == 1) {
          cp_async_bytes<2 * sizeof(T)>(rr_ + hd, rs + hs);
          if (!first) cp_async_bytes<2 * sizeof(T)>(pp_ + hd, ps + hs);
        }
        cp_commit();
      };
      // register windows per position: p on f-2 .. f, r' on f-3 .. f-1, r_i
      // on f-1 .. f
      T pw0[NS], pw1[NS], pw2[NS], rw0[NS], rw1[NS], rw2[NS], ra0[NS], ra1[NS];
#pragma unroll
      for (int m = 0; m < NS; ++m) pw0[m] = pw1[m] = pw2[m] = rw0[m] = rw1[m] = rw2[m] = ra0[m] = ra1[m] = T(0);
      __syncthreads();  // the previous column's readers are done with every buffer
      for (int kk = k0 - 2; kk < k0 - 2 + D - 1; ++kk) fetch(kk);
      int cnt = 0;
      // wait (bounded) for the TMA copies of plane kk; a wait that runs out
      // raises the grid's fail flag, so every grid sum of the launch fails
      auto wait_plane = [&](int kk) {
        const int slot = (kk + 2 * D) % D;
        const long long t0 = clock64();
        unsigned spins = 0;
        while (!mbar_try_wait(&bars[slot], (phase >> slot) & 1u)) {
          if ((++spins & 63u) == 0u && (ld_volatile(&f.bar->fail.v) != 0u || clock64() - t0 > f.spin_cycles)) {
            atomicExch(&f.bar->fail.v, 1u);
            break;
          }
        }
        phase ^= 1u << slot;
      };
      for (int fp = k0 - 2; fp <= k1 + 1; ++fp) {
        // plane fp has landed: the later copies may still fly
        if (tma) wait_plane(fp);
        else cp_wait<D - 2>();
        __syncthreads();
        // the slot of plane fp - 1 is free (its r_i is held in registers)
        fetch(fp + D - 1);
        const T* rr_ = RINGR + ((fp + 2 * D) % D) * SN;
        const T* pp_ = RINGP + ((fp + 2 * D) % D) * SN;
        T* pnew = PP + (fp & 1) * SN;
        // A: p(fp) = r(fp) + beta p_old(fp)
#pragma unroll
        for (int m = 0; m < NS; ++m) {
          if (m >= NO && !(valid >> m & 1u)) continue;
          const int e = es(m);
          const T rv = rr_[e];
          const T pv = first ? rv : rv + tb * pp_[e];
          pw2[m] = pv;
          ra1[m] = rv;
          pnew[e] = pv;
        }
        // B: q(fp-1), r'(fp-1) within the halo of one (needs p(fp-2))
        if (fp >= k0) {
          const T* pc = PP + ((fp - 1) & 1) * SN;
          T* rnew = RP + ((fp - 1) & 1) * SN;
          const bool count = fp - 1 >= k0 && fp - 1 < k1;
#pragma unroll
          for (int m = 0; m < NS; ++m) {
            if (m >= NO && !(in1 >> m & 1u)) continue;
            const int e = es(m);
            const T c2 = T(2) * pw1[m];
            const T qv = (pc[e - 1] + pc[e + 1] - c2) * cx + (pc[e - SP] + pc[e + SP] - c2) * cy +
                         (pw0[m] + pw2[m] - c2) * cz;
            const T r1 = ra0[m] - ta * qv;
            rw2[m] = r1;
            rnew[e] = r1;
            if (m < NO && count) {
              s[2].add(r1 * qv);
              s[3].add(pw1[m] * qv);
            }
          }
        }
        // C, D: w(fp-2) and the outputs of plane fp-2 (needs r'(fp-3))
        if (fp >= k0 + 2) {
          const int k = fp - 2;
          const T* rc = RP + (k & 1) * SN;
          const T* xx_ = RINGX + ((k + 2 * DX) % DX) * (WX * WY);
          const size_t base = (size_t)k * plane;
#pragma unroll
          for (int m = 0; m < NO; ++m) {
            const int e = es(m);
            const T c2 = T(2) * rw1[m];
            const T w = (rc[e - 1] + rc[e + 1] - c2) * cx + (rc[e - SP] + rc[e + SP] - c2) * cy +
                        (rw0[m] + rw2[m] - c2) * cz;
            s[0].add(rw1[m] * rw1[m]);
            s[1].add(rw1[m] * w);
            const size_t g = base + go0 + (NWARP * (m / NWX)) * f.nx + 32 * (m % NWX);
            __stcg(f.x + g, xx_[((tid >> 5) + NWARP * (m / NWX)) * WX + (tid & 31) + 32 * (m % NWX)] + ta * pw0[m]);
            __stcg(pw + g, pw0[m]);
            __stcg(ro + g, rw1[m]);
          }
          if ((++cnt & 15) == 0)
#pragma unroll
            for (int q = 0; q < 4; ++q) s[q].flush();
        }
        // roll the windows
#pragma unroll
        for (int m = 0; m < NS; ++m) {
          pw0[m] = pw1[m];
          pw1[m] = pw2[m];
          rw0[m] = rw1[m];
          rw1[m] = rw2[m];
          ra0[m] = ra1[m];
        }
      }
      // the copies issued beyond the run (planes k1 + 2 .. k1 + D) land
      // before the buffers are used again
      if (tma)
        for (int kk = k1 + 2; kk <= k1 + D; ++kk) wait_plane(kk);
      cp_wait<0>();
    }
    double t[4];
    const bool ok = wave_sum_t0<4>(s, gs, t);
    iter += 1;
    if (tid == 0) {
      if (!ok) {
        status = 5;
      } else {
        const double rr_new = t[0];
        rel = sqrt(rr_new / bb);
        if (rel <= f.tol) status = 1;
        else if (iter >= f.maxit) status = 2;
        else if (!isfinite(rr_new)) status = 3;
        else {
          const double beta = rr_new / rr;
          const double pq_new = t[1] + 2.0 * beta * t[2] + beta * beta * t[3];
          if (pq_new == 0.0 || !isfinite(pq_new)) status = 3;
          else {
            sc.ta = (T)(rr_new / pq_new);
            sc.tb = (T)beta;
          }
        }
        rr = rr_new;
      }
      sc.status = status;
    }
    __syncthreads();
    status = sc.status;
  }

  // ---- zero-mean gauge (or zero for a zero right side) ------------------------
  if (status != 5) {
    WaveSum<T> s[1];
    int cnt = 0;
    for (long long c = gtid; c < nch; c += gstride) {
      const Ch xq = ldch(f.x + (size_t)c * VC);
#pragma unroll
      for (int q = 0; q < VC; ++q) s[0].add(xq.e[q]);
      if ((++cnt & 3) == 0) s[0].flush();
    }
    double t[1];
    const bool ok = wave_sum_t0<1>(s, gs, t);
    if (tid == 0) {
      if (!ok) status = 5;
      sc.mean = (T)(t[0] / (double)f.n);
      sc.status = status;
    }
    __syncthreads();
    status = sc.status;
    if (status != 5) {
      const T mx = sc.mean;
      for (long long c = gtid; c < nch; c += gstride) {
        Ch xq = ldch(f.x + (size_t)c * VC);
#pragma unroll
        for (int q = 0; q < VC; ++q) xq.e[q] = status == 4 ? T(0) : xq.e[q] - mx;
        stch(f.x + (size_t)c * VC, xq);
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

namespace {

bool col_fits(int nx, int ny, int wx, int wy) { return nx % wx == 0 && ny % wy == 0; }

// cuTensorMapEncodeTiled from the driver, looked up once
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static std::mutex mu;
  static bool tried = false;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// a 3-D map of an nx x ny x nz vector with bx x by x 1 boxes (no swizzle,
// no interleave; out-of-range elements are never requested)
template <typename T>
bool encode_map(CUtensorMap* m, const void* base, int nx, int ny, int nz, int bx, int by) {
  const auto enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
  const cuuint64_t strides[2] = {(cuuint64_t)nx * sizeof(T), (cuuint64_t)nx * ny * sizeof(T)};
  const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1u};
  const cuuint32_t estr[3] = {1u, 1u, 1u};
  return enc(m, sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3,
             const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename T, typename C>
int solve_wave(const SolverArgs<T>& a, const FusedCfg& fc, const T* b, T* x, double tol, int maxit, int* iters,
               double* rel, std::string* err) {
  WaveArgs<T> f;
  f.nx = a.g.nx;
  f.ny = a.g.ny;
  f.nz = a.g.nz;
  f.walls = a.g.walls;
  f.cx = a.g.idx * a.g.idx;
  f.cy = a.g.idy * a.g.idy;
  f.cz = a.g.idz * a.g.idz;
  f.ntx = f.nx / C::WX;
  f.nty = f.ny / C::WY;
  f.n = (long long)f.nx * f.ny * f.nz;
  f.b = b;
  f.x = x;
  f.r[0] = a.r;
  f.r[1] = a.q;
  f.p[0] = a.p0;
  f.p[1] = a.p1;
  f.partials = a.partials;
  f.bar = a.bar;
  f.ctl = a.ctl;
  f.tol = tol;
  f.maxit = maxit;
  f.spin_cycles = fc.spin_cycles;
  f.guard = a.guard;
  // TMA boxes for the interior columns: a staged plane of r and p_{i-1}
  // (SP x SY, from x0 - 4), the owned nodes of x (WX x WY)
  f.use_tma = encode_map<T>(&f.tm_r[0], a.r, f.nx, f.ny, f.nz, C::SP, C::SY) &&
              encode_map<T>(&f.tm_r[1], a.q, f.nx, f.ny, f.nz, C::SP, C::SY) &&
              encode_map<T>(&f.tm_p[0], a.p0, f.nx, f.ny, f.nz, C::SP, C::SY) &&
              encode_map<T>(&f.tm_p[1], a.p1, f.nx, f.ny, f.nz, C::SP, C::SY) &&
              encode_map<T>(&f.tm_x, x, f.nx, f.ny, f.nz, C::WX, C::WY);
  int per_sm = 0, dev = 0, nsm = 0;
  cudaError_t e;
  const void* kern = (const void*)k_cg_wave<T, C>;
  const size_t smem = wave_smem<T, C>();
  if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess ||
      (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem)) != cudaSuccess) {
    if (err) *err = std::string("wave CG occupancy: ") + cudaGetErrorString(e);
    return LES_ERR_CUDA;
  }
  if (per_sm < 1) {
    if (err) *err = "wave CG: no block fits on an SM";
    return LES_ERR_CUDA;
  }
  long long G = (long long)per_sm * nsm;
  G = std::min<long long>(G, fc.max_blocks);
  G = std::min<long long>(G, 8LL * nsm);  // the partials hold 2 x kSumSlot words of 8 blocks per SM
  // z-runs as long as possible (each run re-forms two planes of p and r'
  // below it)
  const long long ncol = (long long)f.ntx * f.nty;
  // the (column, run) units are dealt to the G persistent blocks in turns.
  // Fewer columns than blocks: at most G units, one turn (a G-th + 1 unit
  // would double the iteration for the rest).  More: whole columns in full
  // turns, then the planes of the columns left in equal shares, so that no
  // block takes a whole extra column (on 1536 x 1536 x 256: 2304 columns,
  // 7 turns of 304 and 148 planes each of the last 176 columns)
  if (ncol >= G) {
    f.zrun = f.nz;
    f.nchunk = 1;
    f.nunits = (int)((ncol / G) * G);
    f.tail_planes = (int)((ncol - f.nunits) * f.nz);
    f.tail_per = (int)((f.tail_planes + G - 1) / G);
  } else {
    const long long want = std::max<long long>(1, std::min<long long>((long long)f.nz, G / ncol));
    f.zrun = (int)((f.nz + want - 1) / want);
    f.nchunk = (f.nz + f.zrun - 1) / f.zrun;
    f.nunits = (int)(ncol * f.nchunk);
    f.tail_planes = 0;
    f.tail_per = 0;
    G = std::max<long long>(1, std::min<long long>(G, f.nunits));
  }
  f.expected = (unsigned)G + (unsigned)std::max(0, fc.missing);
  if ((e = cudaMemsetAsync(a.bar, 0, sizeof(FusedBar), a.st)) != cudaSuccess) {
    if (err) *err = std::string("wave CG barrier reset: ") + cudaGetErrorString(e);
    return LES_ERR_CUDA;
  }
  void* args[] = {&f};
  {
    ProfScope ps(a.prof, KI_CG_WAVE, a.st);
    e = cudaLaunchCooperativeKernel(kern, dim3((unsigned)G), dim3(NT), args, smem, a.st);
  }
  if (e != cudaSuccess) {
    if (err) *err = std::string("wave CG launch: ") + cudaGetErrorString(e);
    return LES_ERR_CUDA;
  }
  if ((e = cudaMemcpyAsync(a.ctl_host, a.ctl, sizeof(SolverCtl), cudaMemcpyDeviceToHost, a.st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(a.st)) != cudaSuccess) {
    if (err) *err = std::string("wave CG: ") + cudaGetErrorString(e);
    return LES_ERR_CUDA;
  }
  const SolverCtl& c = *a.ctl_host;
  if (iters) *iters = c.iter;
  if (rel) *rel = c.rel;
  // algorithmic traffic of the solve (kCgIterFields per iteration; this
  // kernel streams 6 per iteration plus a third of r_i and p_{i-1} again for
  // the halo, and one set-up sweep for alpha_0)
  if (a.prof) a.prof->bytes[KI_CG_WAVE] += (kCgSetupFields + 1.0 + kCgIterFields * c.iter) * (double)f.n * sizeof(T);
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
      if (err) *err = "poisson: wave solver returned no status";
      return LES_ERR_CUDA;
  }
}

}  // namespace

bool wave_cg_eligible(int nx, int ny, int nz) {
  return (col_fits(nx, ny, Col64::WX, Col64::WY) || col_fits(nx, ny, Col32::WX, Col32::WY)) && nz >= 2 &&
         (long long)nx * ny < (1LL << 31);
}

template <typename T>
int poisson_solve_wave(const SolverArgs<T>& a, const FusedCfg& fc, const T* b, T* x, double tol, int maxit,
                       int* iters, double* rel, std::string* err) {
  // the staging copies move 16-byte chunks: every vector must start on a
  // 16-byte boundary (a caller's view at an odd offset takes the one-pass
  // kernel for any grid instead)
  auto aligned = [](const void* p) { return ((uintptr_t)p & 15u) == 0; };
  if (!wave_cg_eligible(a.g.nx, a.g.ny, a.g.nz) ||
      !(aligned(b) && aligned(x) && aligned(a.r) && aligned(a.q) && aligned(a.p0) && aligned(a.p1)))
    return poisson_solve_roll<T>(a, fc, b, x, tol, maxit, iters, rel, err);
  if (col_fits(a.g.nx, a.g.ny, Col64::WX, Col64::WY))
    return solve_wave<T, Col64>(a, fc, b, x, tol, maxit, iters, rel, err);
  return solve_wave<T, Col32>(a, fc, b, x, tol, maxit, iters, rel, err);
}

template int poisson_solve_wave<float>(const SolverArgs<float>&, const FusedCfg&, const float*, float*, double, int,
                                       int*, double*, std::string*);
template int poisson_solve_wave<double>(const SolverArgs<double>&, const FusedCfg&, const double*, double*, double,
                                        int, int*, double*, std::string*);

}  // namespace les
