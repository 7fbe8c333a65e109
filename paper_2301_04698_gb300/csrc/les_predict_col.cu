// les_predict_col.cu -- the scalar predictor (Eq. scalar_prediction_step,
// Sec. 2.3-2.4: QUICK or WENO3 advection by the u^k mass flux, Smagorinsky-
// Lilly diffusion with f_B, subsidence, radiation and surface fluxes) as a
// column march over two-node lanes.
//
// Tile: 32 lanes x 8 rows; a lane owns V = 2 consecutive x nodes of its row
// (an 8-byte chunk in FP32, 16 bytes in FP64), so a tile is 64 nodes wide.  A block has ten
// warps: warps 0-7 own the tile's rows, warps 8 and 9 the rows just below
// and above it, whose nu_t the y faces need.  The block marches its tile up
// a run of z-planes.  Every input plane is staged into shared memory as 12
// rows (the tile's 8 rows and two on each side) of 32 V + 2 V nodes (one
// lane chunk beyond each end): u^k, v^k, w^k (and b for f_B) by one chunk-
// sized cp.async per lane and row into a four-plane ring, issued a plane
// ahead; theta_l and q_t as phibar = (phi^k + phi^{n+1/2}) / 2 in a
// four-plane ring, averaged from a raw staging plane.  Planes beyond a wall
// take the mirror rule; the few whose rule flips a sign are staged through
// registers.
// Per plane, every warp computes nu_t on the plane above the output plane
// for its row (lanes 0 and 31 also the node just beyond the tile), into a
// two-plane ring; after one barrier the row warps form the face fluxes of
// their nodes -- V + 1 x faces per lane, two y faces per node, and one z
// face per node, the lower z face being the upper one of the plane below,
// carried up the march -- and write phi^{k+1}.
#include <algorithm>

#include "les_internal.h"

namespace les {
namespace {

constexpr int PW = 32;            // lanes per row
constexpr int PR = 8;             // rows per tile
constexpr int PWARP = PR + 2;     // row warps + two halo-row warps
constexpr int NROW = PR + 4;      // staged rows: j0-2 .. j0+9
constexpr int NUROW = PR + 2;     // nu rows: j0-1 .. j0+8

// a lane owns two consecutive x nodes (8 bytes in FP32, 16 in FP64): FP32
// blocks then fit twice per SM (about 97 KB of shared memory each)
template <typename T>
constexpr int kV = 2;
template <typename T>
constexpr int kLB = kV<T> * (int)sizeof(T);     // bytes of a lane's chunk
template <typename T>
constexpr int kMinBlocks = sizeof(T) == 4 ? 2 : 1;  // resident blocks per SM
template <typename T>
constexpr int kTW = PW * kV<T>;                 // tile width
template <typename T>
constexpr int kRL = kTW<T> + 2 * kV<T>;         // staged row length (a lane chunk each side)
template <typename T>
constexpr int kPL = NROW * kRL<T>;              // elements of one staged field-plane
template <typename T>
constexpr int kNPL = NUROW * kRL<T>;            // elements of one nu plane

template <typename T>
struct Vec {
  T v[kV<T>];
};
template <typename T>
__device__ __forceinline__ Vec<T> lds(const T* p) {
  Vec<T> r;
  if constexpr (sizeof(T) == 4) {
    const float2 q = *reinterpret_cast<const float2*>(p);
    r.v[0] = q.x, r.v[1] = q.y;
  } else {
    const double2 q = *reinterpret_cast<const double2*>(p);
    r.v[0] = q.x, r.v[1] = q.y;
  }
  return r;
}
template <typename T>
__device__ __forceinline__ void sts(T* p, const Vec<T>& r) {
  if constexpr (sizeof(T) == 4) *reinterpret_cast<float2*>(p) = make_float2(r.v[0], r.v[1]);
  else *reinterpret_cast<double2*>(p) = make_double2(r.v[0], r.v[1]);
}
template <typename T>
__device__ __forceinline__ Vec<T> ldgv(const T* p) {
  Vec<T> r;
  if constexpr (sizeof(T) == 4) {
    const float2 q = __ldg(reinterpret_cast<const float2*>(p));
    r.v[0] = q.x, r.v[1] = q.y;
  } else {
    const double2 q = __ldg(reinterpret_cast<const double2*>(p));
    r.v[0] = q.x, r.v[1] = q.y;
  }
  return r;
}
template <typename T>
__device__ __forceinline__ void stgv(T* p, const Vec<T>& r) {
  if constexpr (sizeof(T) == 4) __stcs(reinterpret_cast<float2*>(p), make_float2(r.v[0], r.v[1]));
  else __stcs(reinterpret_cast<double2*>(p), make_double2(r.v[0], r.v[1]));
}

__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// The lane's V nodes of a staged row and H nodes beyond each end: e[H + c]
// is node c; neighbours come from the adjacent lanes by shuffles, and lanes
// 0 and 31 read the staged chunk beyond the tile (p points at the lane's
// first node in shared memory).
template <typename T, int H>
struct Ext {
  T e[kV<T> + 2 * H];
};
template <typename T, int H>
__device__ __forceinline__ Ext<T, H> lext(const T* p, int lane) {
  constexpr int V = kV<T>;
  const Vec<T> o = lds(p);
  Ext<T, H> x;
#pragma unroll
  for (int c = 0; c < V; ++c) x.e[H + c] = o.v[c];
#pragma unroll
  for (int q = 0; q < H; ++q) {
    T l = __shfl_up_sync(0xffffffffu, o.v[V - 1 - q], 1);
    T r = __shfl_down_sync(0xffffffffu, o.v[q], 1);
    if (lane == 0) l = p[-1 - q];
    if (lane == 31) r = p[V + q];
    x.e[H - 1 - q] = l;
    x.e[H + V + q] = r;
  }
  return x;
}
__device__ __forceinline__ float c_sqrt(float a) { return sqrtf(a); }
__device__ __forceinline__ double c_sqrt(double a) { return sqrt(a); }
__device__ __forceinline__ float c_sin(float a) { return sinf(a); }
__device__ __forceinline__ double c_sin(double a) { return sin(a); }

// plane holding level kk under ghost rule gh, and the rule's sign: mirror
// across the walls (planes beyond one mirror are clamped: they are staged
// but never used), wrap when periodic
template <typename T>
__device__ __forceinline__ int zsrc(const Grid<T>& g, int kk, int gh, T& sgn) {
  sgn = T(1);
  if (!g.walls) {  // kk is within two periods of the range (nz >= 2)
    kk += kk < 0 ? g.nz : 0;
    kk += kk < 0 ? g.nz : 0;
    kk -= kk >= g.nz ? g.nz : 0;
    kk -= kk >= g.nz ? g.nz : 0;
    return kk;
  }
  if (kk < 0) {
    if (gh == G_ODD) sgn = T(-1);
    kk = -1 - kk;
  } else if (kk >= g.nz) {
    if (gh != G_EVEN) sgn = T(-1);
    kk = 2 * g.nz - 1 - kk;
  }
  return kk < 0 ? 0 : (kk >= g.nz ? g.nz - 1 : kk);
}


// nu_t = (c_s Delta)^2 f_B S (Sec. 2.3) of the lane's V nodes on staged row r
// of level kk, from the velocity rings (planes kk-1 .. kk+1) and the b ring;
// x neighbours by shuffles (lext), y and z neighbours by chunk loads.
template <typename T>
__device__ __forceinline__ void nu_lane(const T* sm, int ringU, int ringB, int kk, int r, int xl, int lane,
                                        const Grid<T>& g, const Phys<T>& ph, unsigned flags, bool fb,
                                        T (&out)[kV<T>]) {
  constexpr int V = kV<T>, RL = kRL<T>, PL = kPL<T>;
  if (flags & LES_PHYS_CONST_NU) {
#pragma unroll
    for (int n = 0; n < V; ++n) out[n] = ph.nu_const;
    return;
  }
  if (!(flags & LES_PHYS_SGS)) {
#pragma unroll
    for (int n = 0; n < V; ++n) out[n] = T(0);
    return;
  }
  const T hx = T(0.5) * g.idx, hy = T(0.5) * g.idy, hz = T(0.5) * g.idz;
  const size_t o = (size_t)r * RL + V + xl;
  T gr[3][3][V];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const T* P = sm + (size_t)(ringU + 4 * c + (kk & 3)) * PL + o;
    const T* Pm = sm + (size_t)(ringU + 4 * c + ((kk - 1) & 3)) * PL + o;
    const T* Pp = sm + (size_t)(ringU + 4 * c + ((kk + 1) & 3)) * PL + o;
    const Ext<T, 1> ex = lext<T, 1>(P, lane);
    const Vec<T> ym = lds(P - RL), yp = lds(P + RL), zm = lds(Pm), zp = lds(Pp);
#pragma unroll
    for (int n = 0; n < V; ++n) {
      gr[c][0][n] = (ex.e[n + 2] - ex.e[n]) * hx;
      gr[c][1][n] = (yp.v[n] - ym.v[n]) * hy;
      gr[c][2][n] = (zp.v[n] - zm.v[n]) * hz;
    }
  }
  Vec<T> bm, bp;
  if (fb) {
    bm = lds(sm + (size_t)(ringB + ((kk - 1) & 3)) * PL + o);
    bp = lds(sm + (size_t)(ringB + ((kk + 1) & 3)) * PL + o);
  }
#pragma unroll
  for (int n = 0; n < V; ++n) {
    T S2 = T(0);
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const T sv = T(0.5) * (gr[c][d][n] + gr[d][c][n]);
        S2 += T(2) * sv * sv;
      }
    T fB = T(1);
    if (fb && S2 > T(0)) {
      const T N2 = (bp.v[n] - bm.v[n]) * hz;
      T q = T(1) - N2 / (T(1) / ph.inv_pr * S2);
      q = q < T(0) ? T(0) : (q > T(1) ? T(1) : q);
      fB = c_sqrt(q);
    }
    out[n] = ph.cs2d2 * fB * c_sqrt(S2);
  }
}

template <typename T>
struct ScaCol {
  Grid<T> g;
  Phys<T> ph;
  int zrun, nchunk, ntx, nty;
  const T *u, *v, *w, *b, *thk, *qtk, *thh, *qth, *srad;
  T *tho, *qto;
};

// Shared memory (elements of T): velocity ring U, V, W [4 planes each], b ring
// [4] (f_B only), phibar rings PT, PQ [4], raw staging of theta_l^k,
// theta_l^{n+1/2}, q_t^k, q_t^{n+1/2} [1 each], nu ring [2].
template <typename T>
struct ScaSmem {
  static constexpr int U = 0, V = 4, W = 8, B = 12, PT = 16, PQ = 20, RAW = 24, NPLANES = 28;
  // after the planes: the nu ring [2 nu planes], then the fluxes of both
  // scalars through the tile's PR + 1 y faces of one level
  static constexpr size_t yf_offset() { return (size_t)NPLANES * kPL<T> + 2 * (size_t)kNPL<T>; }
  static constexpr size_t bytes() { return (yf_offset() + (size_t)(PR + 1) * 2 * kTW<T>) * sizeof(T); }
};

template <typename T, int ADV, unsigned FIX>
__global__ void __launch_bounds__(PW* PWARP, kMinBlocks<T>) k_scalar_col(ScaCol<T> a) {
  constexpr int VV = kV<T>, TW = kTW<T>, RL = kRL<T>, PL = kPL<T>;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  T* NU = sm + (size_t)ScaSmem<T>::NPLANES * PL;
  T* YF = sm + ScaSmem<T>::yf_offset();  // [PR + 1 faces][2 scalars][TW]
  const Grid<T>& g = a.g;
  const Phys<T>& ph = a.ph;
  // the physics switches, fixed at compile time for the common set
  const unsigned flags = FIX ? FIX : ph.flags;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const size_t plane = (size_t)g.nx * g.ny;
  const long long ncol = (long long)a.ntx * a.nty;
  const long long nblk = ncol * a.nchunk;
  const bool fb = flags & LES_PHYS_FB;
  const bool adv_on = flags & LES_PHYS_ADV;
  const bool sgs = flags & LES_PHYS_SGS, cst = flags & LES_PHYS_CONST_NU;
  const T hx = T(0.5) * g.idx, hy = T(0.5) * g.idy, hz = T(0.5) * g.idz;
  constexpr int RINGU = ScaSmem<T>::U, RINGB = ScaSmem<T>::B;
  const T inv_s[2] = {ph.inv_pr, ph.inv_sc};
  const T sflux[2] = {ph.sflux_th, ph.sflux_qt};
  // the field-plane of ring `ring` holding level kk, and element (row, xl)
  auto fp = [&](int ring, int kk) { return sm + (size_t)(ring + (kk & 3)) * PL; };
  auto at = [&](T* base, int row, int xl) { return base + row * RL + VV + xl; };
  auto nup = [&](int kk) { return NU + (size_t)(kk & 1) * kNPL<T>; };
  // staged rows of this warp: row warps their own row, the halo warps two
  const int nst = wid < PR ? 1 : 2;
  const int st0 = wid < PR ? wid + 2 : (wid == PR ? 0 : NROW - 2);
  const int st1 = wid == PR ? 1 : NROW - 1;

  for (long long blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    const int col = (int)(blk % ncol), chunk = (int)(blk / ncol);
    const int x0 = (col % a.ntx) * TW, j0 = (col / a.ntx) * PR;
    const int k0 = chunk * a.zrun, k1 = min(k0 + a.zrun, g.nz);
    const int xl = lane * VV;
    // global offsets (in a plane) of this lane's chunks on its staged rows;
    // lanes 0 and 31 also copy the chunk beyond the tile's end
    size_t src_own[2], src_ext[2];
    int dst_ext = lane == 0 ? -VV : TW;
    const int xext = lane == 0 ? wrapi(x0 - VV, g.nx) : wrapi(x0 + TW, g.nx);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int r = q == 0 ? st0 : st1;
      const size_t gy = (size_t)wrapi(j0 - 2 + r, g.ny) * g.nx;
      src_own[q] = gy + x0 + xl;
      src_ext[q] = gy + xext;
    }
    const bool edge = lane == 0 || lane == PW - 1;

    // stage level kk of a cp.async field (ring r, ghost rule gh)
    auto stage_async = [&](const T* src, int ring, int kk, int gh) {
      T sg;
      const int gz = zsrc(g, kk, gh, sg);
      T* dstp = fp(ring, kk);
      const T* s0 = src + (size_t)gz * plane;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        if (q >= nst) break;
        const int r = q == 0 ? st0 : st1;
        if (sg == T(1)) {
          cp_async_bytes<kLB<T>>(at(dstp, r, xl), s0 + src_own[q]);
          if (edge) cp_async_bytes<kLB<T>>(at(dstp, r, dst_ext), s0 + src_ext[q]);
        } else {
          Vec<T> x = ldgv(s0 + src_own[q]);
#pragma unroll
          for (int c = 0; c < VV; ++c) x.v[c] = -x.v[c];
          sts(at(dstp, r, xl), x);
          if (edge) {
            Vec<T> y = ldgv(s0 + src_ext[q]);
#pragma unroll
            for (int c = 0; c < VV; ++c) y.v[c] = -y.v[c];
            sts(at(dstp, r, dst_ext), y);
          }
        }
      }
    };
    auto stage_vel = [&](int kk) {
      stage_async(a.u, ScaSmem<T>::U, kk, G_UV);
      stage_async(a.v, ScaSmem<T>::V, kk, G_UV);
      stage_async(a.w, ScaSmem<T>::W, kk, G_ODD);
      if (fb) stage_async(a.b, ScaSmem<T>::B, kk, G_EVEN);
    };
    // raw theta_l / q_t of level kk (mirror rule: no sign)
    auto stage_raw = [&](int kk) {
      T sg;
      const int gz = zsrc(g, kk, G_EVEN, sg);
      const T* src[4] = {a.thk, a.thh, a.qtk, a.qth};
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        T* dstp = sm + (size_t)(ScaSmem<T>::RAW + f) * PL;
        const T* s0 = src[f] + (size_t)gz * plane;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          if (q >= nst) break;
          const int r = q == 0 ? st0 : st1;
          cp_async_bytes<kLB<T>>(at(dstp, r, xl), s0 + src_own[q]);
          if (edge) cp_async_bytes<kLB<T>>(at(dstp, r, dst_ext), s0 + src_ext[q]);
        }
      }
    };
    // phibar of level kk from the raw plane, all threads over the 12 rows
    auto average_raw = [&](int kk) {
      constexpr int NV = PL / VV;
      constexpr int NIT = (2 * NV + PW * PWARP - 1) / (PW * PWARP);
#pragma unroll
      for (int it = 0; it < NIT; ++it) {
        const int e = threadIdx.x + it * PW * PWARP;
        if (e >= 2 * NV) break;
        const int s = e / NV, o = (e - s * NV) * VV;
        const T* rk = sm + (size_t)(ScaSmem<T>::RAW + 2 * s) * PL + o;
        const T* rh = rk + PL;
        const Vec<T> x = lds(rk), y = lds(rh);
        Vec<T> z;
#pragma unroll
        for (int c = 0; c < VV; ++c) z.v[c] = T(0.5) * (x.v[c] + y.v[c]);
        sts(fp(s == 0 ? ScaSmem<T>::PT : ScaSmem<T>::PQ, kk) + o, z);
      }
    };
    // phibar of level kk straight from global memory (prologue)
    auto stage_bar_direct = [&](int kk) {
      T sg;
      const int gz = zsrc(g, kk, G_EVEN, sg);
      const T* src[4] = {a.thk, a.thh, a.qtk, a.qth};
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        T* dstp = fp(s == 0 ? ScaSmem<T>::PT : ScaSmem<T>::PQ, kk);
        const T* sk = src[2 * s] + (size_t)gz * plane;
        const T* sh = src[2 * s + 1] + (size_t)gz * plane;
        for (int q = 0; q < nst; ++q) {
          const int r = q == 0 ? st0 : st1;
          const Vec<T> x = ldgv(sk + src_own[q]), y = ldgv(sh + src_own[q]);
          Vec<T> z;
#pragma unroll
          for (int c = 0; c < VV; ++c) z.v[c] = T(0.5) * (x.v[c] + y.v[c]);
          sts(at(dstp, r, xl), z);
          if (edge) {
            const Vec<T> xe = ldgv(sk + src_ext[q]), ye = ldgv(sh + src_ext[q]);
#pragma unroll
            for (int c = 0; c < VV; ++c) z.v[c] = T(0.5) * (xe.v[c] + ye.v[c]);
            sts(at(dstp, r, dst_ext), z);
          }
        }
      }
    };
    // nu_t at one node (x offset xo in the tile, staged row r) of level kk
    // from the velocity planes kk-1, kk, kk+1 (Sec. 2.3)
    auto nu_node = [&](int kk, int r, int xo) -> T {
      if (cst) return ph.nu_const;
      if (!sgs) return T(0);
      T* vel[3] = {fp(ScaSmem<T>::U, kk), fp(ScaSmem<T>::V, kk), fp(ScaSmem<T>::W, kk)};
      T* vm[3] = {fp(ScaSmem<T>::U, kk - 1), fp(ScaSmem<T>::V, kk - 1), fp(ScaSmem<T>::W, kk - 1)};
      T* vp[3] = {fp(ScaSmem<T>::U, kk + 1), fp(ScaSmem<T>::V, kk + 1), fp(ScaSmem<T>::W, kk + 1)};
      T gr[3][3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        gr[c][0] = (*at(vel[c], r, xo + 1) - *at(vel[c], r, xo - 1)) * hx;
        gr[c][1] = (*at(vel[c], r + 1, xo) - *at(vel[c], r - 1, xo)) * hy;
        gr[c][2] = (*at(vp[c], r, xo) - *at(vm[c], r, xo)) * hz;
      }
      T S2 = T(0);
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const T sv = T(0.5) * (gr[c][d] + gr[d][c]);
          S2 += T(2) * sv * sv;
        }
      T fB = T(1);
      if (fb && S2 > T(0)) {
        const T N2 = (*at(fp(ScaSmem<T>::B, kk + 1), r, xo) - *at(fp(ScaSmem<T>::B, kk - 1), r, xo)) * hz;
        T q = T(1) - N2 / (T(1) / ph.inv_pr * S2);
        q = q < T(0) ? T(0) : (q > T(1) ? T(1) : q);
        fB = c_sqrt(q);
      }
      return ph.cs2d2 * fB * c_sqrt(S2);
    };
    // nu_t of level kk on this warp's nu row (row warps: their row; halo
    // warps: the row beyond the tile), lanes 0 / 31 also one node beyond
    const int nurow = wid < PR ? wid + 1 : (wid == PR ? 0 : NUROW - 1);
    auto nu_row = [&](int kk) {
      T* nr = nup(kk) + nurow * RL + VV;
      Vec<T> o;
      nu_lane<T>(sm, RINGU, RINGB, kk, nurow + 1, xl, lane, g, ph, flags, fb, o.v);
      sts(nr + xl, o);
    };
    // nu_t of level kk at the nodes just beyond the tile's ends on the row
    // warps' rows (the x faces at the ends read them): halo warp PR, one node
    // per lane of lanes 0 .. 2 PR - 1
    auto nu_edges = [&](int kk) {
      if (wid != PR || lane >= 2 * PR) return;
      const int r = 1 + (lane >> 1), xo = (lane & 1) ? TW : -1;
      nup(kk)[r * RL + VV + xo] = nu_node(kk, r + 1, xo);
    };

    // ---- the lower z face of the run's first plane (prologue) -------------
    const int j = j0 + wid;
    const int srow = wid + 2;  // staged row of this row warp
    T flz[2][VV];              // flux through the lower z face of each node
    __syncthreads();           // the previous run's readers are done
    for (int kk = k0 - 2; kk <= k0 + 1; ++kk) {
      stage_vel(kk);
      stage_bar_direct(kk);
    }
    cp_commit();
    cp_wait<0>();
    __syncthreads();
    // nu_t of level k0 on every row; of level k0-1 on the row warps' nodes
    nu_row(k0);
    nu_edges(k0);
    T nu_lo[VV];
    if (wid < PR) nu_lane<T>(sm, RINGU, RINGB, k0 - 1, srow, xl, lane, g, ph, flags, fb, nu_lo);
    __syncthreads();
    // the ring slot of level k0-2 is free: stage level k0+2
    stage_vel(k0 + 2);
    stage_raw(k0 + 2);
    cp_commit();
    // z face between levels k0-1 and k0
    auto zface = [&](int kl, const T* nul, const T* nuu, T (&out)[2][VV]) {
      const bool wall = g.walls && (kl == -1 || kl == g.nz - 1);
      if (wall) {
        const bool sfc = g.walls && kl == -1 && (flags & LES_PHYS_SFC);
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
          for (int c = 0; c < VV; ++c) out[q][c] = sfc ? -sflux[q] : T(0);
        return;
      }
      const T rl = g.prof(ph.rho0, kl), ru = g.prof(ph.rho0, kl + 1);
      const T rhof = T(0.5) * (rl + ru);
      const Vec<T> wl = lds(at(fp(ScaSmem<T>::W, kl), srow, xl)), wu = lds(at(fp(ScaSmem<T>::W, kl + 1), srow, xl));
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int ring = q == 0 ? ScaSmem<T>::PT : ScaSmem<T>::PQ;
        const Vec<T> fm = lds(at(fp(ring, kl - 1), srow, xl)), f0 = lds(at(fp(ring, kl), srow, xl));
        const Vec<T> f1 = lds(at(fp(ring, kl + 1), srow, xl)), f2 = lds(at(fp(ring, kl + 2), srow, xl));
#pragma unroll
        for (int c = 0; c < VV; ++c) {
          T F = T(0);
          if (adv_on) F = T(0.5) * (rl * wl.v[c] + ru * wu.v[c]);
          const T K = rhof * (T(0.5) * (nul[c] + nuu[c]));
          T adv = T(0);
          if (adv_on) adv = F * face_value(ADV, F, fm.v[c], f0.v[c], f1.v[c], f2.v[c]);
          out[q][c] = -adv + K * inv_s[q] * (f1.v[c] - f0.v[c]) * g.idz;
        }
      }
    };
    if (wid < PR) {
      const Vec<T> nu0 = lds(nup(k0) + (wid + 1) * RL + VV + xl);
      zface(k0 - 1, nu_lo, nu0.v, flz);
    }

    // fluxes of both scalars through the y face between staged rows sr and
    // sr + 1 of level kk, for this lane's nodes
    auto yface = [&](int kk, int sr, T (&out)[2][VV]) {
      const T r0 = g.prof(ph.rho0, kk);
      const T* nk = nup(kk) + VV + xl;
      const Vec<T> nlo = lds(nk + (sr - 1) * RL), nhi = lds(nk + sr * RL);
      const T* vr = at(fp(ScaSmem<T>::V, kk), sr, xl);
      const Vec<T> vlo = lds(vr), vhi = lds(vr + RL);
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const T* pr = at(fp(q == 0 ? ScaSmem<T>::PT : ScaSmem<T>::PQ, kk), sr, xl);
        const Vec<T> pm = lds(pr - RL), p0 = lds(pr), p1 = lds(pr + RL), p2 = lds(pr + 2 * RL);
#pragma unroll
        for (int c = 0; c < VV; ++c) {
          T F = T(0);
          if (adv_on) F = T(0.5) * (r0 * vlo.v[c] + r0 * vhi.v[c]);
          const T K = r0 * (T(0.5) * (nlo.v[c] + nhi.v[c]));
          T adv = T(0);
          if (adv_on) adv = F * face_value(ADV, F, pm.v[c], p0.v[c], p1.v[c], p2.v[c]);
          out[q][c] = -adv + K * inv_s[q] * (p1.v[c] - p0.v[c]) * g.idy;
        }
      }
    };

    // ---- the march ----------------------------------------------------------
    for (int k = k0; k < k1; ++k) {
      cp_wait<0>();
      __syncthreads();  // level k+2 staged; every reader of levels k-1 / k-2 is done
      average_raw(k + 2);
      stage_vel(k + 3);
      cp_commit();
      nu_row(k + 1);
      nu_edges(k + 1);
      // each row warp's upper y face of level k, and (halo warp PR + 1) the
      // face below the tile's first row: computed once, the lower faces read
      // back below
      T yup[2][VV];
      if (wid != PR) {
        const int sr = wid < PR ? srow : 1;
        yface(k, sr, yup);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          Vec<T> o;
#pragma unroll
          for (int c = 0; c < VV; ++c) o.v[c] = yup[q][c];
          sts(YF + ((size_t)(sr - 1) * 2 + q) * TW + xl, o);
        }
      }
      __syncthreads();  // nu_t of level k+1, phibar of level k+2, the y fluxes visible; raw plane free
      stage_raw(k + 3);
      cp_commit();
      if (wid >= PR) continue;
      // ---- fluxes of this row's nodes on level k ----
      const size_t m = (size_t)k * plane + (size_t)j * g.nx + x0 + xl;
      const T r0 = g.prof(ph.rho0, k);
      T tend[2][VV];
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int c = 0; c < VV; ++c) tend[q][c] = T(0);
      const T* nk = nup(k) + VV + xl;
      // x faces: V + 1 faces between nodes c-1 and c, c = 0 .. V
      {
        const Ext<T, 1> nxe = lext<T, 1>(nk + (wid + 1) * RL, lane);
        const Ext<T, 1> uxe = lext<T, 1>(at(fp(ScaSmem<T>::U, k), srow, xl), lane);
        const T* nx_ = nxe.e;
        const T* ux = uxe.e;
        const T rhof = r0;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const Ext<T, 2> pxe = lext<T, 2>(at(fp(q == 0 ? ScaSmem<T>::PT : ScaSmem<T>::PQ, k), srow, xl), lane);
          const T* px = pxe.e;
          T fl[VV + 1];
#pragma unroll
          for (int f = 0; f <= VV; ++f) {
            // face between node f-1 (px[f+1]) and node f (px[f+2])
            T F = T(0);
            if (adv_on) F = T(0.5) * (r0 * ux[f] + r0 * ux[f + 1]);
            const T K = rhof * (T(0.5) * (nx_[f] + nx_[f + 1]));
            T adv = T(0);
            if (adv_on) adv = F * face_value(ADV, F, px[f], px[f + 1], px[f + 2], px[f + 3]);
            fl[f] = -adv + K * inv_s[q] * (px[f + 2] - px[f + 1]) * g.idx;
          }
#pragma unroll
          for (int c = 0; c < VV; ++c) tend[q][c] += (fl[c + 1] - fl[c]) * g.idx;
        }
      }
      // y faces: the upper one of this row from yup, the lower one (the upper
      // face of the row below) from the shared buffer
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const Vec<T> lo = lds(YF + ((size_t)wid * 2 + q) * TW + xl);
#pragma unroll
        for (int c = 0; c < VV; ++c) tend[q][c] += (yup[q][c] - lo.v[c]) * g.idy;
      }
      // z faces: the upper face of this level; the lower one was carried up
      {
        T flu[2][VV];
        const Vec<T> nlo = lds(nk + (wid + 1) * RL), nhi = lds(nup(k + 1) + VV + xl + (wid + 1) * RL);
        zface(k, nlo.v, nhi.v, flu);
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
          for (int c = 0; c < VV; ++c) {
            tend[q][c] += (flu[q][c] - flz[q][c]) * g.idz;
            flz[q][c] = flu[q][c];
          }
      }
      if (flags & LES_PHYS_SUBS) {
        const T wsub = ph.subs_div * (T(k) + T(0.5)) * g.dz;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int ring = q == 0 ? ScaSmem<T>::PT : ScaSmem<T>::PQ;
          const Vec<T> p0 = lds(at(fp(ring, k), srow, xl)), p1 = lds(at(fp(ring, k + 1), srow, xl));
#pragma unroll
          for (int c = 0; c < VV; ++c) tend[q][c] += r0 * wsub * (p1.v[c] - p0.v[c]) * g.idz;
        }
      }
      if (flags & LES_PHYS_RAD) {
        const Vec<T> sr = ldgv(a.srad + m);
#pragma unroll
        for (int c = 0; c < VV; ++c) tend[0][c] += sr.v[c];
      }
      const Vec<T> hth = ldgv(a.thh + m), hqt = ldgv(a.qth + m);
      Vec<T> oth, oqt;
#pragma unroll
      const T dtr = ph.dt / r0;  // (rho0 phi^{n+1/2} + dt tend) / rho0
      for (int c = 0; c < VV; ++c) {
        oth.v[c] = hth.v[c] + dtr * tend[0][c];
        oqt.v[c] = hqt.v[c] + dtr * tend[1][c];
      }
      stgv(a.tho + m, oth);
      stgv(a.qto + m, oqt);
    }
    cp_wait<0>();  // copies of the run's last (unused) planes land before the next run reuses the rings
  }
}


// ---- a2 + a4: momentum predictor (Eq. momentum_prediction_step) -------------
// u^ = (rho0 u^n + dt [-rho0 G(alpha0 p') + R(u^{n+1/2})]) / rho0 with
// R = -QUICK advection by the u^{n+1/2} mass flux + div(rho0 nu_t (grad u +
// grad u^T)) + rho0 b k + Coriolis - sponge, all at u^{n+1/2} = (u^k + u^n) / 2.
// Same tile, warps and march as the scalar predictor.  Rings of four planes:
// u^{n+1/2} (three components), alpha0 p' and b; u^{n+1/2} and alpha0 p' of a
// level are formed, with the ghost rule's sign, from raw planes of u^k, u^n
// and p' staged by cp.async; b is staged by cp.async straight into its ring.
template <typename T>
struct MomCol {
  Grid<T> g;
  Phys<T> ph;
  int zrun, nchunk, ntx, nty;
  const T *uk, *vk, *wk, *un, *vn, *wn, *p, *b;
  T *ou, *ov, *ow;
};

template <typename T>
struct MomSmem {
  static constexpr int U = 0, V = 4, W = 8, AP = 12, B = 16, RAW = 20, NPLANES = 27;
  static constexpr size_t bytes() { return ((size_t)NPLANES * kPL<T> + 2 * (size_t)kNPL<T>) * sizeof(T); }
};

template <typename T, int ADV, unsigned FIX>
__global__ void __launch_bounds__(PW* PWARP, kMinBlocks<T>) k_momentum_col(MomCol<T> a) {
  constexpr int VV = kV<T>, TW = kTW<T>, RL = kRL<T>, PL = kPL<T>;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  T* NU = sm + (size_t)MomSmem<T>::NPLANES * PL;
  const Grid<T>& g = a.g;
  const Phys<T>& ph = a.ph;
  // the physics switches, fixed at compile time for the common set
  const unsigned flags = FIX ? FIX : ph.flags;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const size_t plane = (size_t)g.nx * g.ny;
  const long long ncol = (long long)a.ntx * a.nty;
  const long long nblk = ncol * a.nchunk;
  const bool fb = flags & LES_PHYS_FB;
  const bool adv_on = flags & LES_PHYS_ADV;
  const bool sgs = flags & LES_PHYS_SGS, cst = flags & LES_PHYS_CONST_NU;
  const T hx = T(0.5) * g.idx, hy = T(0.5) * g.idy, hz = T(0.5) * g.idz;
  constexpr int RINGU = MomSmem<T>::U, RINGB = MomSmem<T>::B;
  const T ih[3] = {g.idx, g.idy, g.idz};
  auto fp = [&](int ring, int kk) { return sm + (size_t)(ring + (kk & 3)) * PL; };
  auto at = [&](T* base, int row, int xl) { return base + row * RL + VV + xl; };
  auto nup = [&](int kk) { return NU + (size_t)(kk & 1) * kNPL<T>; };
  const int nst = wid < PR ? 1 : 2;
  const int st0 = wid < PR ? wid + 2 : (wid == PR ? 0 : NROW - 2);
  const int st1 = wid == PR ? 1 : NROW - 1;

  for (long long blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    const int col = (int)(blk % ncol), chunk = (int)(blk / ncol);
    const int x0 = (col % a.ntx) * TW, j0 = (col / a.ntx) * PR;
    const int k0 = chunk * a.zrun, k1 = min(k0 + a.zrun, g.nz);
    const int xl = lane * VV;
    size_t src_own[2], src_ext[2];
    const int dst_ext = lane == 0 ? -VV : TW;
    const int xext = lane == 0 ? wrapi(x0 - VV, g.nx) : wrapi(x0 + TW, g.nx);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int r = q == 0 ? st0 : st1;
      const size_t gy = (size_t)wrapi(j0 - 2 + r, g.ny) * g.nx;
      src_own[q] = gy + x0 + xl;
      src_ext[q] = gy + xext;
    }
    const bool edge = lane == 0 || lane == PW - 1;

    // raw u^k, v^k, w^k, u^n, v^n, w^n, p' of level kk (mirror plane)
    auto stage_raw = [&](int kk) {
      T sg;
      const int gz = zsrc(g, kk, G_EVEN, sg);
      const T* src[7] = {a.uk, a.vk, a.wk, a.un, a.vn, a.wn, a.p};
#pragma unroll
      for (int f = 0; f < 7; ++f) {
        T* dstp = sm + (size_t)(MomSmem<T>::RAW + f) * PL;
        const T* s0 = src[f] + (size_t)gz * plane;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          if (q >= nst) break;
          const int r = q == 0 ? st0 : st1;
          cp_async_bytes<kLB<T>>(at(dstp, r, xl), s0 + src_own[q]);
          if (edge) cp_async_bytes<kLB<T>>(at(dstp, r, dst_ext), s0 + src_ext[q]);
        }
      }
    };
    auto stage_b = [&](int kk) {
      if (!(fb || (flags & LES_PHYS_BUOY))) return;
      T sg;
      const int gz = zsrc(g, kk, G_EVEN, sg);
      T* dstp = fp(MomSmem<T>::B, kk);
      const T* s0 = a.b + (size_t)gz * plane;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        if (q >= nst) break;
        const int r = q == 0 ? st0 : st1;
        cp_async_bytes<kLB<T>>(at(dstp, r, xl), s0 + src_own[q]);
        if (edge) cp_async_bytes<kLB<T>>(at(dstp, r, dst_ext), s0 + src_ext[q]);
      }
    };
    // u^{n+1/2} (with the ghost rule's sign) and alpha0 p' of level kk from
    // the raw planes, all threads over the 12 rows
    auto form_raw = [&](int kk) {
      T su, sw, sp;
      const int gu = zsrc(g, kk, G_UV, su);
      zsrc(g, kk, G_ODD, sw);
      zsrc(g, kk, G_EVEN, sp);
      const T a0 = __ldg(ph.alpha0 + gu);
      constexpr int NV = PL / VV;
      for (int e = threadIdx.x; e < 4 * NV; e += PW * PWARP) {
        const int f = e / NV, o = (e - f * NV) * VV;
        Vec<T> z;
        if (f < 3) {
          const Vec<T> x = lds(sm + (size_t)(MomSmem<T>::RAW + f) * PL + o);
          const Vec<T> y = lds(sm + (size_t)(MomSmem<T>::RAW + 3 + f) * PL + o);
          const T sg = f == 2 ? sw : su;
#pragma unroll
          for (int c = 0; c < VV; ++c) z.v[c] = sg * (T(0.5) * (x.v[c] + y.v[c]));
          sts(fp(f == 0 ? MomSmem<T>::U : (f == 1 ? MomSmem<T>::V : MomSmem<T>::W), kk) + o, z);
        } else {
          const Vec<T> x = lds(sm + (size_t)(MomSmem<T>::RAW + 6) * PL + o);
#pragma unroll
          for (int c = 0; c < VV; ++c) z.v[c] = a0 * x.v[c];
          sts(fp(MomSmem<T>::AP, kk) + o, z);
        }
      }
    };
    // the same straight from global memory (prologue), b included
    auto stage_direct = [&](int kk) {
      T su, sw, sp;
      const int gz = zsrc(g, kk, G_UV, su);
      zsrc(g, kk, G_ODD, sw);
      zsrc(g, kk, G_EVEN, sp);
      const T a0 = __ldg(ph.alpha0 + gz);
      const size_t po = (size_t)gz * plane;
      for (int q = 0; q < nst; ++q) {
        const int r = q == 0 ? st0 : st1;
        for (int part = 0; part < (edge ? 2 : 1); ++part) {
          const size_t so = po + (part ? src_ext[q] : src_own[q]);
          const int dx = part ? dst_ext : xl;
          const T* uks[3] = {a.uk, a.vk, a.wk};
          const T* uns[3] = {a.un, a.vn, a.wn};
#pragma unroll
          for (int f = 0; f < 3; ++f) {
            const Vec<T> x = ldgv(uks[f] + so), y = ldgv(uns[f] + so);
            const T sg = f == 2 ? sw : su;
            Vec<T> z;
#pragma unroll
            for (int c = 0; c < VV; ++c) z.v[c] = sg * (T(0.5) * (x.v[c] + y.v[c]));
            sts(at(fp(f == 0 ? MomSmem<T>::U : (f == 1 ? MomSmem<T>::V : MomSmem<T>::W), kk), r, dx), z);
          }
          const Vec<T> pp = ldgv(a.p + so);
          Vec<T> z;
#pragma unroll
          for (int c = 0; c < VV; ++c) z.v[c] = a0 * pp.v[c];
          sts(at(fp(MomSmem<T>::AP, kk), r, dx), z);
          if (fb || (flags & LES_PHYS_BUOY)) sts(at(fp(MomSmem<T>::B, kk), r, dx), ldgv(a.b + so));
        }
      }
    };
    auto nu_node = [&](int kk, int r, int xo) -> T {
      if (cst) return ph.nu_const;
      if (!sgs) return T(0);
      T* vel[3] = {fp(MomSmem<T>::U, kk), fp(MomSmem<T>::V, kk), fp(MomSmem<T>::W, kk)};
      T* vm[3] = {fp(MomSmem<T>::U, kk - 1), fp(MomSmem<T>::V, kk - 1), fp(MomSmem<T>::W, kk - 1)};
      T* vp[3] = {fp(MomSmem<T>::U, kk + 1), fp(MomSmem<T>::V, kk + 1), fp(MomSmem<T>::W, kk + 1)};
      T gr[3][3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        gr[c][0] = (*at(vel[c], r, xo + 1) - *at(vel[c], r, xo - 1)) * hx;
        gr[c][1] = (*at(vel[c], r + 1, xo) - *at(vel[c], r - 1, xo)) * hy;
        gr[c][2] = (*at(vp[c], r, xo) - *at(vm[c], r, xo)) * hz;
      }
      T S2 = T(0);
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const T sv = T(0.5) * (gr[c][d] + gr[d][c]);
          S2 += T(2) * sv * sv;
        }
      T fB = T(1);
      if (fb && S2 > T(0)) {
        const T N2 = (*at(fp(MomSmem<T>::B, kk + 1), r, xo) - *at(fp(MomSmem<T>::B, kk - 1), r, xo)) * hz;
        T q = T(1) - N2 / (T(1) / ph.inv_pr * S2);
        q = q < T(0) ? T(0) : (q > T(1) ? T(1) : q);
        fB = c_sqrt(q);
      }
      return ph.cs2d2 * fB * c_sqrt(S2);
    };
    const int nurow = wid < PR ? wid + 1 : (wid == PR ? 0 : NUROW - 1);
    auto nu_row = [&](int kk) {
      T* nr = nup(kk) + nurow * RL + VV;
      Vec<T> o;
      nu_lane<T>(sm, RINGU, RINGB, kk, nurow + 1, xl, lane, g, ph, flags, fb, o.v);
      sts(nr + xl, o);
    };
    // nu_t just beyond the tile's ends on the row warps' rows: halo warp PR
    auto nu_edges = [&](int kk) {
      if (wid != PR || lane >= 2 * PR) return;
      const int r = 1 + (lane >> 1), xo = (lane & 1) ? TW : -1;
      nup(kk)[r * RL + VV + xo] = nu_node(kk, r + 1, xo);
    };
    const int j = j0 + wid;
    const int srow = wid + 2;
    // momentum flux of the three components through the z face between
    // levels kl and kl+1 of this lane's nodes (Sec. 2.4 with the wall rules:
    // no flux through the free-slip surface, no advection through the lid)
    auto zface = [&](int kl, const T* nul, const T* nuu, T (&out)[3][VV]) {
      if (g.walls && kl == -1) {
#pragma unroll
        for (int c3 = 0; c3 < 3; ++c3)
#pragma unroll
          for (int c = 0; c < VV; ++c) out[c3][c] = T(0);
        return;
      }
      const bool lid = g.walls && kl == g.nz - 1;
      const bool advz = adv_on && !lid;
      // nu_t beyond the lid mirrors the top level
      if (lid) nuu = nul;
      const T rl = g.prof(ph.rho0, kl), ru = g.prof(ph.rho0, kl + 1);
      const T rhof = T(0.5) * (rl + ru);
      T* W0 = fp(MomSmem<T>::W, kl);
      T* W1 = fp(MomSmem<T>::W, kl + 1);
      const Vec<T> wl = lds(at(W0, srow, xl)), wu = lds(at(W1, srow, xl));
      // tangential derivatives of w at both levels: along x (c = 0), along y (c = 1)
      T gx0[VV], gx1[VV], gy0[VV], gy1[VV];
      {
        const Vec<T> a0 = lds(at(W0, srow - 1, xl)), b0 = lds(at(W0, srow + 1, xl));
        const Vec<T> a1 = lds(at(W1, srow - 1, xl)), b1 = lds(at(W1, srow + 1, xl));
        const Ext<T, 1> x0e = lext<T, 1>(at(W0, srow, xl), lane), x1e = lext<T, 1>(at(W1, srow, xl), lane);
#pragma unroll
        for (int c = 0; c < VV; ++c) {
          gx0[c] = x0e.e[c + 2] - x0e.e[c];
          gx1[c] = x1e.e[c + 2] - x1e.e[c];
          gy0[c] = b0.v[c] - a0.v[c];
          gy1[c] = b1.v[c] - a1.v[c];
        }
      }
#pragma unroll
      for (int c3 = 0; c3 < 3; ++c3) {
        const int ring = c3 == 0 ? MomSmem<T>::U : (c3 == 1 ? MomSmem<T>::V : MomSmem<T>::W);
        const Vec<T> fm = lds(at(fp(ring, kl - 1), srow, xl)), f0 = lds(at(fp(ring, kl), srow, xl));
        const Vec<T> f1 = lds(at(fp(ring, kl + 1), srow, xl)), f2 = lds(at(fp(ring, kl + 2), srow, xl));
#pragma unroll
        for (int c = 0; c < VV; ++c) {
          T adv = T(0);
          if (advz) {
            const T F = T(0.5) * (rl * wl.v[c] + ru * wu.v[c]);
            adv = F * face_value(ADV, F, fm.v[c], f0.v[c], f1.v[c], f2.v[c]);
          }
          const T dn = (f1.v[c] - f0.v[c]) * g.idz;
          const T dtg = c3 == 2 ? dn : T(0.25) * (c3 == 0 ? gx0[c] + gx1[c] : gy0[c] + gy1[c]) * ih[c3];
          const T K = rhof * (T(0.5) * (nul[c] + nuu[c]));
          out[c3][c] = -adv + K * (dn + dtg);
        }
      }
    };

    // ---- prologue: levels k0-2 .. k0+1, nu_t of k0 (and k0-1 own), the lower z face
    T flz[3][VV];
    __syncthreads();
    for (int kk = k0 - 2; kk <= k0 + 1; ++kk) stage_direct(kk);
    __syncthreads();
    nu_row(k0);
    nu_edges(k0);
    T nu_lo[VV];
    if (wid < PR) nu_lane<T>(sm, RINGU, RINGB, k0 - 1, srow, xl, lane, g, ph, flags, fb, nu_lo);
    __syncthreads();
    if (wid < PR) {
      const Vec<T> nu0 = lds(nup(k0) + (wid + 1) * RL + VV + xl);
      zface(k0 - 1, nu_lo, nu0.v, flz);
    }
    stage_raw(k0 + 2);
    stage_b(k0 + 2);
    cp_commit();

    for (int k = k0; k < k1; ++k) {
      cp_wait<0>();
      __syncthreads();  // raw level k+2 and b of k+2 staged; readers of level k-2 done
      form_raw(k + 2);
      __syncthreads();  // u^{n+1/2}, alpha0 p' of level k+2 formed; the raw planes are free
      stage_raw(k + 3);
      stage_b(k + 3);
      cp_commit();
      nu_row(k + 1);
      nu_edges(k + 1);
      __syncthreads();  // nu_t of level k+1 visible
      if (wid >= PR) continue;
      const size_t m = (size_t)k * plane + (size_t)j * g.nx + x0 + xl;
      const T r0 = g.prof(ph.rho0, k);
      T R[3][VV];
#pragma unroll
      for (int c3 = 0; c3 < 3; ++c3)
#pragma unroll
        for (int c = 0; c < VV; ++c) R[c3][c] = T(0);
      const T* nk = nup(k) + VV + xl;
      T* Uk = fp(MomSmem<T>::U, k);
      T* Vk = fp(MomSmem<T>::V, k);
      T* Wk = fp(MomSmem<T>::W, k);
      // ---- x faces (V + 1 per lane)
      {
        const Ext<T, 1> nxe = lext<T, 1>(nk + (wid + 1) * RL, lane);
        const Ext<T, 1> uxe = lext<T, 1>(at(Uk, srow, xl), lane);
        const T* nx_ = nxe.e;
        const T* ux = uxe.e;
        // tangential derivatives of u at nodes -1 .. V: along y (for v), along z (for w)
        T gty[VV + 2], gtz[VV + 2];
        {
          const Ext<T, 1> ym = lext<T, 1>(at(Uk, srow - 1, xl), lane), yp = lext<T, 1>(at(Uk, srow + 1, xl), lane);
          const Ext<T, 1> zm = lext<T, 1>(at(fp(MomSmem<T>::U, k - 1), srow, xl), lane);
          const Ext<T, 1> zp = lext<T, 1>(at(fp(MomSmem<T>::U, k + 1), srow, xl), lane);
#pragma unroll
          for (int c = 0; c < VV + 2; ++c) gty[c] = yp.e[c] - ym.e[c], gtz[c] = zp.e[c] - zm.e[c];
        }
#pragma unroll
        for (int c3 = 0; c3 < 3; ++c3) {
          T* ringk = c3 == 0 ? Uk : (c3 == 1 ? Vk : Wk);
          const Ext<T, 2> pxe = lext<T, 2>(at(ringk, srow, xl), lane);
          const T* px = pxe.e;
          T fl[VV + 1];
#pragma unroll
          for (int f = 0; f <= VV; ++f) {
            T adv = T(0);
            if (adv_on) {
              const T F = T(0.5) * (r0 * ux[f] + r0 * ux[f + 1]);
              adv = F * face_value(ADV, F, px[f], px[f + 1], px[f + 2], px[f + 3]);
            }
            const T dn = (px[f + 2] - px[f + 1]) * g.idx;
            const T dtg = c3 == 0 ? dn : T(0.25) * (c3 == 1 ? gty[f] + gty[f + 1] : gtz[f] + gtz[f + 1]) * ih[c3];
            const T K = r0 * (T(0.5) * (nx_[f] + nx_[f + 1]));
            fl[f] = -adv + K * (dn + dtg);
          }
#pragma unroll
          for (int c = 0; c < VV; ++c) R[c3][c] += (fl[c + 1] - fl[c]) * g.idx;
        }
      }
      // ---- y faces (j-1/2 and j+1/2 of every node)
      {
        const Vec<T> nm = lds(nk + wid * RL), no = lds(nk + (wid + 1) * RL), np = lds(nk + (wid + 2) * RL);
        const T* vr = at(Vk, srow, xl);
        const Vec<T> vm = lds(vr - RL), vo = lds(vr), vp = lds(vr + RL);
        // tangential derivatives of v on rows j-1, j, j+1: along x (for u), along z (for w)
        T gtx[3][VV], gtz[3][VV];
        {
          const T* zm = at(fp(MomSmem<T>::V, k - 1), srow, xl);
          const T* zp = at(fp(MomSmem<T>::V, k + 1), srow, xl);
#pragma unroll
          for (int rr = 0; rr < 3; ++rr) {
            const Ext<T, 1> ex = lext<T, 1>(vr + (rr - 1) * RL, lane);
#pragma unroll
            for (int c = 0; c < VV; ++c) gtx[rr][c] = ex.e[c + 2] - ex.e[c];
            const Vec<T> a2 = lds(zm + (rr - 1) * RL), b2 = lds(zp + (rr - 1) * RL);
#pragma unroll
            for (int c = 0; c < VV; ++c) gtz[rr][c] = b2.v[c] - a2.v[c];
          }
        }
#pragma unroll
        for (int c3 = 0; c3 < 3; ++c3) {
          T* ringk = c3 == 0 ? Uk : (c3 == 1 ? Vk : Wk);
          const T* pr = at(ringk, srow, xl);
          const Vec<T> p2m = lds(pr - 2 * RL), p1m = lds(pr - RL), p0 = lds(pr), p1p = lds(pr + RL),
                       p2p = lds(pr + 2 * RL);
#pragma unroll
          for (int c = 0; c < VV; ++c) {
            T am = T(0), ap = T(0);
            if (adv_on) {
              const T Fm = T(0.5) * (r0 * vm.v[c] + r0 * vo.v[c]);
              const T Fp = T(0.5) * (r0 * vo.v[c] + r0 * vp.v[c]);
              am = Fm * face_value(ADV, Fm, p2m.v[c], p1m.v[c], p0.v[c], p1p.v[c]);
              ap = Fp * face_value(ADV, Fp, p1m.v[c], p0.v[c], p1p.v[c], p2p.v[c]);
            }
            const T dnm = (p0.v[c] - p1m.v[c]) * g.idy, dnp = (p1p.v[c] - p0.v[c]) * g.idy;
            T dtm, dtp;
            if (c3 == 1) {
              dtm = dnm, dtp = dnp;
            } else {
              const T(&gt)[3][VV] = c3 == 0 ? gtx : gtz;
              dtm = T(0.25) * (gt[0][c] + gt[1][c]) * ih[c3];
              dtp = T(0.25) * (gt[1][c] + gt[2][c]) * ih[c3];
            }
            const T Km = r0 * (T(0.5) * (nm.v[c] + no.v[c])), Kp = r0 * (T(0.5) * (no.v[c] + np.v[c]));
            const T flm = -am + Km * (dnm + dtm), flp = -ap + Kp * (dnp + dtp);
            R[c3][c] += (flp - flm) * g.idy;
          }
        }
      }
      // ---- z faces: the upper face of this level; the lower one carried up
      {
        T flu[3][VV];
        const Vec<T> nlo = lds(nk + (wid + 1) * RL), nhi = lds(nup(k + 1) + VV + xl + (wid + 1) * RL);
        zface(k, nlo.v, nhi.v, flu);
#pragma unroll
        for (int c3 = 0; c3 < 3; ++c3)
#pragma unroll
          for (int c = 0; c < VV; ++c) {
            R[c3][c] += (flu[c3][c] - flz[c3][c]) * g.idz;
            flz[c3][c] = flu[c3][c];
          }
      }
      // ---- sources, pressure gradient, update
      const Vec<T> uo = lds(at(Uk, srow, xl)), vo = lds(at(Vk, srow, xl)), wo = lds(at(Wk, srow, xl));
      if (flags & LES_PHYS_BUOY) {
        const Vec<T> bo = lds(at(fp(MomSmem<T>::B, k), srow, xl));
#pragma unroll
        for (int c = 0; c < VV; ++c) R[2][c] += r0 * bo.v[c];
      }
      if (flags & LES_PHYS_CORIOLIS) {
#pragma unroll
        for (int c = 0; c < VV; ++c) {
          R[0][c] += ph.f_cor * r0 * (vo.v[c] - ph.vg);
          R[1][c] -= ph.f_cor * r0 * (uo.v[c] - ph.ug);
        }
      }
      const T zc = (T(k) + T(0.5)) * g.dz;
      if ((flags & LES_PHYS_SPONGE) && zc > ph.sponge_zs) {
        const T sn = c_sin(T(1.5707963267948966) * (zc - ph.sponge_zs) / (ph.sponge_h - ph.sponge_zs));
        const T beta = ph.sponge_rate * sn * sn * r0;
#pragma unroll
        for (int c = 0; c < VV; ++c) {
          R[0][c] -= beta * (uo.v[c] - ph.ug);
          R[1][c] -= beta * (vo.v[c] - ph.vg);
          R[2][c] -= beta * (wo.v[c] - T(0));
        }
      }
      T gp[3][VV];
      {
        T* A0 = fp(MomSmem<T>::AP, k);
        const T* ar = at(A0, srow, xl);
        const Vec<T> ym = lds(ar - RL), yp = lds(ar + RL);
        const Vec<T> zm = lds(at(fp(MomSmem<T>::AP, k - 1), srow, xl)), zp = lds(at(fp(MomSmem<T>::AP, k + 1), srow, xl));
        const Ext<T, 1> ae = lext<T, 1>(ar, lane);
        const T* e = ae.e;
#pragma unroll
        for (int c = 0; c < VV; ++c) {
          gp[0][c] = (e[c + 2] - e[c]) * hx;
          gp[1][c] = (yp.v[c] - ym.v[c]) * hy;
          gp[2][c] = (zp.v[c] - zm.v[c]) * hz;
        }
      }
      const T* uns[3] = {a.un, a.vn, a.wn};
      T* outs[3] = {a.ou, a.ov, a.ow};
      const T ir0 = T(1) / r0;  // (rho0 u^n + dt (-rho0 G + R)) / rho0
#pragma unroll
      for (int c3 = 0; c3 < 3; ++c3) {
        const Vec<T> un = ldgv(uns[c3] + m);
        Vec<T> res;
#pragma unroll
        for (int c = 0; c < VV; ++c) res.v[c] = un.v[c] + ph.dt * (R[c3][c] * ir0 - gp[c3][c]);
        stgv(outs[c3] + m, res);
      }
    }
    cp_wait<0>();
  }
}
}  // namespace

template <typename T>
bool pcol_eligible(const Grid<T>& g) {
  return g.nx % kTW<T> == 0 && g.ny % PR == 0 && g.nz >= 2;
}

// runs of z-planes per column.  With fewer columns than half a wave of
// resident blocks (kMinBlocks per SM), as many runs as one wave holds: a
// partial second wave would leave most SMs idle for a whole run (on a
// 128 x 128 grid, 9 runs of 11 planes ran both predictors 1.2x faster than
// 16 runs of 6).  With more, at least two waves, which keeps the last,
// partial wave short (512 x 512: two runs per column 5 % faster than one).
template <typename T>
long long pcol_runs(int nz, long long ncol, int nsm) {
  const long long slots = (long long)kMinBlocks<T> * std::max(1, nsm);
  const long long c = std::max<long long>(1, ncol);
  const long long nw = 2 * c < slots ? slots / c : (2 * slots + c - 1) / c;
  return std::max<long long>(1, std::min<long long>((long long)nz, nw));
}

template <typename T>
cudaError_t launch_scalar_col(const StageArgs<T>& a, int nsm, const T* u, const T* v, const T* w, const T* b,
                              const T* thk, const T* qtk, const T* thh, const T* qth, const T* srad, T* th_out,
                              T* qt_out) {
  ScaCol<T> r;
  r.g = a.g;
  r.ph = a.ph;
  r.ntx = a.g.nx / kTW<T>;
  r.nty = a.g.ny / PR;
  const long long ncol = (long long)r.ntx * r.nty;
  const long long nw = pcol_runs<T>(a.g.nz, ncol, nsm);
  r.zrun = (int)((a.g.nz + nw - 1) / nw);
  r.nchunk = (a.g.nz + r.zrun - 1) / r.zrun;
  r.u = u, r.v = v, r.w = w, r.b = b;
  r.thk = thk, r.qtk = qtk, r.thh = thh, r.qth = qth, r.srad = srad;
  r.tho = th_out, r.qto = qt_out;
  const size_t smem = ScaSmem<T>::bytes();
  constexpr unsigned kDry = LES_PHYS_ADV | LES_PHYS_SGS;  // the dry Taylor-Green set
  auto kern = a.ph.advection == LES_ADV_WENO3 ? k_scalar_col<T, LES_ADV_WENO3, 0u>
              : a.ph.flags == kDry             ? k_scalar_col<T, LES_ADV_QUICK, kDry>
                                               : k_scalar_col<T, LES_ADV_QUICK, 0u>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long nblk = ncol * r.nchunk;
  const unsigned grid = (unsigned)std::min<long long>(nblk, 1LL << 20);
  ProfScope ps(a.prof, KI_SCALAR, a.st);
  kern<<<grid, PW * PWARP, smem, a.st>>>(r);
  return cudaGetLastError();
}

template bool pcol_eligible<float>(const Grid<float>&);
template bool pcol_eligible<double>(const Grid<double>&);
template cudaError_t launch_scalar_col<float>(const StageArgs<float>&, int, const float*, const float*, const float*,
                                              const float*, const float*, const float*, const float*, const float*,
                                              const float*, float*, float*);
template cudaError_t launch_scalar_col<double>(const StageArgs<double>&, int, const double*, const double*,
                                               const double*, const double*, const double*, const double*,
                                               const double*, const double*, const double*, double*, double*);


template <typename T>
cudaError_t launch_momentum_col(const StageArgs<T>& a, int nsm, const T* uk, const T* vk, const T* wk, const T* un,
                                const T* vn, const T* wn, const T* p, const T* b, T* ou, T* ov, T* ow) {
  MomCol<T> r;
  r.g = a.g;
  r.ph = a.ph;
  r.ntx = a.g.nx / kTW<T>;
  r.nty = a.g.ny / PR;
  const long long ncol = (long long)r.ntx * r.nty;
  const long long nw = pcol_runs<T>(a.g.nz, ncol, nsm);
  r.zrun = (int)((a.g.nz + nw - 1) / nw);
  r.nchunk = (a.g.nz + r.zrun - 1) / r.zrun;
  r.uk = uk, r.vk = vk, r.wk = wk, r.un = un, r.vn = vn, r.wn = wn, r.p = p, r.b = b;
  r.ou = ou, r.ov = ov, r.ow = ow;
  const size_t smem = MomSmem<T>::bytes();
  constexpr unsigned kDry = LES_PHYS_ADV | LES_PHYS_SGS;
  auto kern = a.ph.advection == LES_ADV_WENO3 ? k_momentum_col<T, LES_ADV_WENO3, 0u>
              : a.ph.flags == kDry             ? k_momentum_col<T, LES_ADV_QUICK, kDry>
                                               : k_momentum_col<T, LES_ADV_QUICK, 0u>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long nblk = ncol * r.nchunk;
  const unsigned grid = (unsigned)std::min<long long>(nblk, 1LL << 20);
  ProfScope ps(a.prof, KI_MOMENTUM, a.st);
  kern<<<grid, PW * PWARP, smem, a.st>>>(r);
  return cudaGetLastError();
}

template cudaError_t launch_momentum_col<float>(const StageArgs<float>&, int, const float*, const float*,
                                                const float*, const float*, const float*, const float*, const float*,
                                                const float*, float*, float*, float*);
template cudaError_t launch_momentum_col<double>(const StageArgs<double>&, int, const double*, const double*,
                                                 const double*, const double*, const double*, const double*,
                                                 const double*, const double*, double*, double*, double*);

}  // namespace les
