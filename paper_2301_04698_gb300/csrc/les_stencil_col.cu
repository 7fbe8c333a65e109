// les_stencil_col.cu -- the per-sub-iteration stencil passes as column marches
// over 16-byte lanes (Sec. 2.4): the correction of Eq. pressure_correction and
// the Poisson right side with the Appendix A term.
//
// A block of 8 warps owns a tile of 32 lanes x 8 rows; a lane holds V
// consecutive x nodes of its row (V = 4 floats or 2 doubles: one 16-byte
// load or store per field), so a tile is 32 V nodes wide.  The block marches
// its tile up a run of z-planes.  Neighbours in z are register windows that
// roll with the march; neighbours in x come from the adjacent lanes by warp
// shuffles (the two lanes at the tile's edges load the node beyond it);
// neighbours in y are 16-byte loads of the adjacent rows, which the warps
// of the block load as their own rows, so they are mostly L1 hits.  Every
// wrap and ghost rule is resolved once per row or plane, not per node.
// Eligible grids: nx a multiple of 32 V, ny a multiple of 8.
#include <algorithm>

#include "les_internal.h"

namespace les {
namespace {

constexpr int CW = 32;  // lanes per row
constexpr int CR = 8;   // rows (warps) per tile
constexpr unsigned FULL = 0xffffffffu;

template <typename T>
constexpr int kV = 16 / (int)sizeof(T);

template <typename T>
struct Lane {
  T v[kV<T>];
};

template <typename T>
__device__ __forceinline__ Lane<T> ldv(const T* __restrict__ p) {
  Lane<T> r;
  if constexpr (sizeof(T) == 4) {
    const float4 q = __ldg(reinterpret_cast<const float4*>(p));
    r.v[0] = q.x, r.v[1] = q.y, r.v[2] = q.z, r.v[3] = q.w;
  } else {
    const double2 q = __ldg(reinterpret_cast<const double2*>(p));
    r.v[0] = q.x, r.v[1] = q.y;
  }
  return r;
}
// streaming load of a field read once (does not allocate in L1)
template <typename T>
__device__ __forceinline__ Lane<T> ldv_once(const T* __restrict__ p) {
  Lane<T> r;
  if constexpr (sizeof(T) == 4) {
    const float4 q = __ldcs(reinterpret_cast<const float4*>(p));
    r.v[0] = q.x, r.v[1] = q.y, r.v[2] = q.z, r.v[3] = q.w;
  } else {
    const double2 q = __ldcs(reinterpret_cast<const double2*>(p));
    r.v[0] = q.x, r.v[1] = q.y;
  }
  return r;
}
template <typename T>
__device__ __forceinline__ void stv(T* __restrict__ p, const Lane<T>& r) {
  if constexpr (sizeof(T) == 4) {
    __stcs(reinterpret_cast<float4*>(p), make_float4(r.v[0], r.v[1], r.v[2], r.v[3]));
  } else {
    __stcs(reinterpret_cast<double2*>(p), make_double2(r.v[0], r.v[1]));
  }
}

__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// plane holding global level kk under ghost rule gh, and the sign of the rule
// (walls: mirror across the surface k = -1/2 and the lid k = nz - 1/2;
// periodic: wrap).  |kk| stays within two planes of the domain.
template <typename T>
__device__ __forceinline__ int zplane(const Grid<T>& g, int kk, int gh, T& sgn) {
  sgn = T(1);
  if (!g.walls) return kk < 0 ? kk + g.nz : (kk >= g.nz ? kk - g.nz : kk);
  if (kk < 0) {
    if (gh == G_ODD) sgn = T(-1);
    return -1 - kk;
  }
  if (kk >= g.nz) {
    if (gh != G_EVEN) sgn = T(-1);
    return 2 * g.nz - 1 - kk;
  }
  return kk;
}

// Lane values extended by H nodes on each side: e[H + c] is the lane's node
// c; e[H - 1 - q] and e[H + V + q] are the nodes q + 1 beyond its left and
// right ends, from the neighbouring lanes (or, at the tile's edges, the
// values `lo` / `hi` loaded by lanes 0 and 31).
template <typename T, int H>
struct Ext {
  T e[kV<T> + 2 * H];
};
template <typename T, int H>
__device__ __forceinline__ Ext<T, H> extend(const Lane<T>& c, int lane, const T (&lo)[H], const T (&hi)[H]) {
  constexpr int V = kV<T>;
  Ext<T, H> x;
#pragma unroll
  for (int q = 0; q < V; ++q) x.e[H + q] = c.v[q];
#pragma unroll
  for (int q = 0; q < H; ++q) {
    const T l = __shfl_up_sync(FULL, c.v[V - 1 - q], 1);
    const T r = __shfl_down_sync(FULL, c.v[q], 1);
    x.e[H - 1 - q] = lane == 0 ? lo[q] : l;
    x.e[H + V + q] = lane == CW - 1 ? hi[q] : r;
  }
  return x;
}

// runs of z-planes: at least `want` (tile, run) blocks, runs as long as possible
inline void col_runs(int nz, long long ncol, long long want, int& zrun, int& nchunk) {
  const long long w = std::max<long long>(1, std::min<long long>((long long)nz, (want + ncol - 1) / ncol));
  zrun = (int)((nz + w - 1) / w);
  nchunk = (nz + zrun - 1) / zrun;
}

template <typename T>
struct ColArgs {
  Grid<T> g;
  Phys<T> ph;
  int zrun, nchunk, ntx, nty;
  int op;
  const T *ou, *ov, *ow, *psi;
  T *u, *v, *w, *p, *rhs;
};

// ---- a7: correction (Sec. 2.4) ------------------------------------------------
// u_c = u^_c - dt G_c(psi), p += rho0 psi; the z neighbours of psi roll in
// registers.
template <typename T>
__global__ void __launch_bounds__(CW* CR) k_correct_col(ColArgs<T> a) {
  constexpr int V = kV<T>;
  const Grid<T>& g = a.g;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const size_t plane = (size_t)g.nx * g.ny;
  const long long ncol = (long long)a.ntx * a.nty;
  const long long nblk = ncol * a.nchunk;
  const T hx = T(0.5) * g.idx, hy = T(0.5) * g.idy, hz = T(0.5) * g.idz;
  for (long long blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    const int col = (int)(blk % ncol), chunk = (int)(blk / ncol);
    const int x0 = (col % a.ntx) * (CW * V), j = (col / a.ntx) * CR + wid;
    const int i = x0 + lane * V;
    const int k0 = chunk * a.zrun, k1 = min(k0 + a.zrun, g.nz);
    const size_t row = (size_t)j * g.nx, rowm = (size_t)wrapi(j - 1, g.ny) * g.nx,
                 rowp = (size_t)wrapi(j + 1, g.ny) * g.nx;
    const int xe = lane == 0 ? wrapi(x0 - 1, g.nx) : wrapi(x0 + CW * V, g.nx);
    const bool edge = lane == 0 || lane == CW - 1;
    T sg;
    Lane<T> pm = ldv(a.psi + (size_t)zplane(g, k0 - 1, G_EVEN, sg) * plane + row + i);
    Lane<T> pc = ldv(a.psi + (size_t)k0 * plane + row + i);
    for (int k = k0; k < k1; ++k) {
      const size_t pk = (size_t)k * plane;
      const Lane<T> pp = ldv(a.psi + (size_t)zplane(g, k + 1, G_EVEN, sg) * plane + row + i);
      const Lane<T> ym = ldv(a.psi + pk + rowm + i), yp = ldv(a.psi + pk + rowp + i);
      T eg[1] = {edge ? __ldg(a.psi + pk + row + xe) : T(0)};
      const Lane<T> uh = ldv_once(a.ou + pk + row + i), vh = ldv_once(a.ov + pk + row + i),
                    wh = ldv_once(a.ow + pk + row + i);
      Lane<T> pr = ldv_once(a.p + pk + row + i);
      const Ext<T, 1> x = extend<T, 1>(pc, lane, eg, eg);
      const T r0 = a.ph.rho0[k];
      Lane<T> ou, ov, ow;
#pragma unroll
      for (int c = 0; c < V; ++c) {
        const T gx = (x.e[c + 2] - x.e[c]) * hx;
        const T gy = (yp.v[c] - ym.v[c]) * hy;
        const T gz = (pp.v[c] - pm.v[c]) * hz;
        ou.v[c] = uh.v[c] - a.ph.dt * gx;
        ov.v[c] = vh.v[c] - a.ph.dt * gy;
        ow.v[c] = wh.v[c] - a.ph.dt * gz;
        pr.v[c] += r0 * pc.v[c];
      }
      stv(a.u + pk + row + i, ou);
      stv(a.v + pk + row + i, ov);
      stv(a.w + pk + row + i, ow);
      stv(a.p + pk + row + i, pr);
      pm = pc;
      pc = pp;
    }
  }
}

// ---- a4 (second half): Poisson right side (Eq. pressure_correction, App. A) ----
// rhs = (alpha0 / dt) D(rho0 u^) - C(psi) (compact operator) or D(rho0 u^) / dt
// (consistent operator); D central, C the fourth difference
// sum_l [psi_{+2} - 4 psi_{+1} + 6 psi - 4 psi_{-1} + psi_{-2}] / (4 Delta_l^2).
// The z windows are w^ on planes k-1 .. k+1 and psi on k-2 .. k+2.
template <typename T>
__global__ void __launch_bounds__(CW* CR) k_rhs_col(ColArgs<T> a) {
  constexpr int V = kV<T>;
  const Grid<T>& g = a.g;
  const Phys<T>& ph = a.ph;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const size_t plane = (size_t)g.nx * g.ny;
  const long long ncol = (long long)a.ntx * a.nty;
  const long long nblk = ncol * a.nchunk;
  const T hx = T(0.5) * g.idx, hy = T(0.5) * g.idy, hz = T(0.5) * g.idz;
  const T c4x = T(0.25) * g.idx * g.idx, c4y = T(0.25) * g.idy * g.idy, c4z = T(0.25) * g.idz * g.idz;
  const bool compact = a.op == LES_OP_COMPACT;
  for (long long blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    const int col = (int)(blk % ncol), chunk = (int)(blk / ncol);
    const int x0 = (col % a.ntx) * (CW * V), j = (col / a.ntx) * CR + wid;
    const int i = x0 + lane * V;
    const int k0 = chunk * a.zrun, k1 = min(k0 + a.zrun, g.nz);
    const size_t row = (size_t)j * g.nx;
    const size_t rm1 = (size_t)wrapi(j - 1, g.ny) * g.nx, rp1 = (size_t)wrapi(j + 1, g.ny) * g.nx;
    const size_t rm2 = (size_t)wrapi(j - 2, g.ny) * g.nx, rp2 = (size_t)wrapi(j + 2, g.ny) * g.nx;
    // the two nodes beyond each end of the tile, for the edge lanes
    const int xa = lane == 0 ? wrapi(x0 - 2, g.nx) : wrapi(x0 + CW * V, g.nx);
    const int xb = lane == 0 ? wrapi(x0 - 1, g.nx) : wrapi(x0 + CW * V + 1, g.nx);
    const bool edge = lane == 0 || lane == CW - 1;
    Lane<T> ps[5], wz[3];
    T sg;
#pragma unroll
    for (int q = 0; q < 4; ++q)
      ps[q] = compact ? ldv(a.psi + (size_t)zplane(g, k0 - 2 + q, G_EVEN, sg) * plane + row + i) : Lane<T>{};
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      wz[q] = ldv(a.ow + (size_t)zplane(g, k0 - 1 + q, G_ODD, sg) * plane + row + i);
#pragma unroll
      for (int c = 0; c < V; ++c) wz[q].v[c] *= sg;
    }
    // the next plane's own-row inputs are loaded one step ahead, so that
    // their latency overlaps a step of arithmetic
    T sw;
    Lane<T> wn = ldv(a.ow + (size_t)zplane(g, k0 + 1, G_ODD, sw) * plane + row + i);
    Lane<T> pn = compact ? ldv(a.psi + (size_t)zplane(g, k0 + 2, G_EVEN, sg) * plane + row + i) : Lane<T>{};
    Lane<T> un = ldv(a.ou + (size_t)k0 * plane + row + i);
    T swn = sw;
    for (int k = k0; k < k1; ++k) {
      const size_t pk = (size_t)k * plane;
      wz[2] = wn;
#pragma unroll
      for (int c = 0; c < V; ++c) wz[2].v[c] *= swn;
      if (compact) ps[4] = pn;
      // u^ with one node beyond each lane end; v^ on the rows j -+ 1
      const Lane<T> uc = un;
      if (k + 1 < k1) {
        wn = ldv(a.ow + (size_t)zplane(g, k + 2, G_ODD, sw) * plane + row + i);
        swn = sw;
        if (compact) pn = ldv(a.psi + (size_t)zplane(g, k + 3, G_EVEN, sg) * plane + row + i);
        un = ldv(a.ou + pk + plane + row + i);
      }
      T ue_lo[1] = {edge ? __ldg(a.ou + pk + row + xb) : T(0)};
      T ue_hi[1] = {edge ? __ldg(a.ou + pk + row + xa) : T(0)};
      const Lane<T> vm = ldv(a.ov + pk + rm1 + i), vp = ldv(a.ov + pk + rp1 + i);
      const Ext<T, 1> ux = extend<T, 1>(uc, lane, ue_lo, ue_hi);
      const T r0 = g.prof(ph.rho0, k), rzm = g.prof(ph.rho0, k - 1), rzp = g.prof(ph.rho0, k + 1);
      Lane<T> out;
      if (compact) {
        T pe_lo[2] = {edge ? __ldg(a.psi + pk + row + xb) : T(0), edge ? __ldg(a.psi + pk + row + xa) : T(0)};
        const Lane<T> qm1 = ldv(a.psi + pk + rm1 + i), qp1 = ldv(a.psi + pk + rp1 + i);
        const Lane<T> qm2 = ldv(a.psi + pk + rm2 + i), qp2 = ldv(a.psi + pk + rp2 + i);
        // lanes 0 and 31 hold the two nodes beyond their tile end in pe_lo:
        // lane 0 (x0 - 1, x0 - 2), lane 31 (x0 + 32V + 1, x0 + 32V)
        T lo[2] = {pe_lo[0], pe_lo[1]};
        T hi[2] = {pe_lo[1], pe_lo[0]};
        const Ext<T, 2> px = extend<T, 2>(ps[2], lane, lo, hi);
        const T a0dt = __ldg(ph.alpha0 + k) / ph.dt;
#pragma unroll
        for (int c = 0; c < V; ++c) {
          T div = (r0 * ux.e[c + 2] - r0 * ux.e[c]) * hx;
          div += (r0 * vp.v[c] - r0 * vm.v[c]) * hy;
          div += (rzp * wz[2].v[c] - rzm * wz[0].v[c]) * hz;
          const T cc = px.e[c + 2];
          T C = (px.e[c + 4] - T(4) * px.e[c + 3] + T(6) * cc - T(4) * px.e[c + 1] + px.e[c]) * c4x;
          C += (qp2.v[c] - T(4) * qp1.v[c] + T(6) * cc - T(4) * qm1.v[c] + qm2.v[c]) * c4y;
          C += (ps[4].v[c] - T(4) * ps[3].v[c] + T(6) * cc - T(4) * ps[1].v[c] + ps[0].v[c]) * c4z;
          out.v[c] = a0dt * div - C;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) ps[q] = ps[q + 1];
      } else {
#pragma unroll
        for (int c = 0; c < V; ++c) {
          T div = (r0 * ux.e[c + 2] - r0 * ux.e[c]) * hx;
          div += (r0 * vp.v[c] - r0 * vm.v[c]) * hy;
          div += (rzp * wz[2].v[c] - rzm * wz[0].v[c]) * hz;
          out.v[c] = div / ph.dt;
        }
      }
      stv(a.rhs + pk + row + i, out);
      wz[0] = wz[1];
      wz[1] = wz[2];
    }
  }
}

template <typename T>
ColArgs<T> col_args(const StageArgs<T>& a, int max_blocks) {
  ColArgs<T> c{};
  c.g = a.g;
  c.ph = a.ph;
  c.ntx = a.g.nx / (CW * kV<T>);
  c.nty = a.g.ny / CR;
  // max_blocks is eight blocks per SM: at least two waves of (tile, run) blocks
  col_runs(a.g.nz, (long long)c.ntx * c.nty, 2LL * max_blocks, c.zrun, c.nchunk);
  return c;
}

template <typename T>
unsigned col_grid(const ColArgs<T>& c) {
  return (unsigned)std::min<long long>((long long)c.ntx * c.nty * c.nchunk, 1LL << 20);
}

}  // namespace

template <typename T>
bool col_eligible(const Grid<T>& g) {
  return g.nx % (CW * kV<T>) == 0 && g.ny % CR == 0 && g.nz >= 2;
}

template <typename T>
cudaError_t launch_correct_col(const StageArgs<T>& a, int max_blocks, const T* ou, const T* ov, const T* ow,
                               const T* psi, T* u, T* v, T* w, T* p) {
  ColArgs<T> c = col_args(a, max_blocks);
  c.ou = ou, c.ov = ov, c.ow = ow, c.psi = psi;
  c.u = u, c.v = v, c.w = w, c.p = p;
  ProfScope ps(a.prof, KI_CORRECT, a.st);
  k_correct_col<T><<<col_grid(c), CW * CR, 0, a.st>>>(c);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_rhs_col(const StageArgs<T>& a, int max_blocks, int op, const T* ou, const T* ov, const T* ow,
                           const T* psi, T* rhs) {
  ColArgs<T> c = col_args(a, max_blocks);
  c.op = op;
  c.ou = ou, c.ov = ov, c.ow = ow, c.psi = psi;
  c.rhs = rhs;
  ProfScope ps(a.prof, KI_RHS, a.st);
  k_rhs_col<T><<<col_grid(c), CW * CR, 0, a.st>>>(c);
  return cudaGetLastError();
}

#define LES_COL_INSTANTIATE(T)                                                                                 \
  template bool col_eligible<T>(const Grid<T>&);                                                               \
  template cudaError_t launch_correct_col<T>(const StageArgs<T>&, int, const T*, const T*, const T*, const T*, \
                                             T*, T*, T*, T*);                                                  \
  template cudaError_t launch_rhs_col<T>(const StageArgs<T>&, int, int, const T*, const T*, const T*,          \
                                         const T*, T*);
LES_COL_INSTANTIATE(float)
LES_COL_INSTANTIATE(double)

}  // namespace les
