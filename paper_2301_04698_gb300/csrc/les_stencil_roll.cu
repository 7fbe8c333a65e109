// les_stencil_roll.cu -- momentum and scalar predictors (and the Poisson
// right side) as 2.5-D z-marches with ring buffers (Sec. 2.3-2.4: QUICK advection, Smagorinsky-Lilly
// viscosity with f_B, SGS stress and diffusion, buoyancy, Coriolis, sponge,
// pressure gradient, subsidence, radiation and surface fluxes).
//
// A 32 x 8 thread block owns a 32 x 8 column and marches a run of z-planes.
// Shared memory holds five-plane rings (x / y halo of two nodes) of
// u^{n+1/2} = (u^k + u^n)/2, b and alpha0 p', and a three-plane ring (halo one)
// of nu_t.  Each step stages one new plane of every input -- so no plane is
// read twice within a run -- computes nu_t on the plane above the output plane
// and then the output plane itself.  The wrap, ghost rules and sign of every
// staged value are applied once, at staging time.
#include "les_internal.h"

namespace les {
namespace {

constexpr int RX = 32, RY = 8, RH = 2;
constexpr int PX = RX + 2 * RH, PY = RY + 2 * RH, PN = PX * PY;  // halo-2 plane
constexpr int NX = RX + 2, NY = RY + 2, NNP = NX * NY;            // halo-1 nu plane
constexpr int NRING = 5;

__device__ __forceinline__ double r_sqrt(double a) { return sqrt(a); }
__device__ __forceinline__ float r_sqrt(float a) { return sqrtf(a); }
__device__ __forceinline__ double r_sin(double a) { return sin(a); }
__device__ __forceinline__ float r_sin(float a) { return sinf(a); }

__device__ __forceinline__ int wrap_any(int i, int n) {
  while (i < 0) i += n;
  while (i >= n) i -= n;
  return i;
}
__device__ __forceinline__ int slot5(int k) { return ((k % NRING) + NRING) % NRING; }
__device__ __forceinline__ int slot3(int k) { return ((k % 3) + 3) % 3; }
// in-plane index of local (x, y), x in [-2, 34), y in [-2, 10)
__device__ __forceinline__ int pidx(int x, int y) { return (y + RH) * PX + (x + RH); }
__device__ __forceinline__ int nidx1(int x, int y) { return (y + 1) * NX + (x + 1); }

// global plane and sign of plane gk under ghost rule gh
template <typename T>
__device__ __forceinline__ int zsrc_roll(const Grid<T>& g, int gk, int gh, T& sgn) {
  sgn = T(1);
  if (!g.walls) return wrap_any(gk, g.nz);
  if (gk < 0) {
    gk = -1 - gk;
    if (gh == G_ODD) sgn = T(-1);
  } else if (gk >= g.nz) {
    gk = 2 * g.nz - 1 - gk;
    if (gh != G_EVEN) sgn = T(-1);
  }
  return gk < 0 ? 0 : (gk >= g.nz ? g.nz - 1 : gk);  // planes beyond one mirror: any valid data (unused)
}


template <typename T>
struct MomRoll {
  Grid<T> g;
  Phys<T> ph;
  int zrun, nchunk, ntx, nty;
  const T *uk, *vk, *wk, *un, *vn, *wn, *p, *b;
  T *ou, *ov, *ow;
};

template <typename T, int ADV>
__global__ void __launch_bounds__(RX* RY) k_momentum_roll(MomRoll<T> a) {
  extern __shared__ unsigned char smraw[];
  T* U = reinterpret_cast<T*>(smraw);  // [NRING][PN] each
  T* V = U + NRING * PN;
  T* W = V + NRING * PN;
  T* Bb = W + NRING * PN;
  T* AP = Bb + NRING * PN;
  T* NU = AP + NRING * PN;  // [3][NNP]
  const Grid<T>& g = a.g;
  const Phys<T>& ph = a.ph;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + RX * ty;
  const long long ncol = (long long)a.ntx * a.nty;
  const long long nblk = ncol * a.nchunk;
  const size_t plane = (size_t)g.nx * g.ny;
  for (long long blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    const int col = (int)(blk % ncol), chunk = (int)(blk / ncol);
    const int x0 = (col % a.ntx) * RX, y0 = (col / a.ntx) * RY;
    const int k0 = chunk * a.zrun, k1 = min(k0 + a.zrun, g.nz);
    // this thread's two staging slots of a plane: in-plane offsets of the wrapped node
    int soff[2];
    bool sok[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int e = tid + q * RX * RY;
      sok[q] = e < PN;
      const int bx = e % PX, by = e / PX;
      soff[q] = sok[q] ? wrap_any(y0 - RH + by, g.ny) * g.nx + wrap_any(x0 - RH + bx, g.nx) : 0;
    }
    // stage global plane kk (any integer) into its ring slot
    auto stage = [&](int kk) {
      const int s = slot5(kk);
      T su, sv, sw;  // sign of the ghost rule per component
      int gzu, gzw, gze;
      {
        T sg;
        gzu = zsrc_roll(g, kk, G_UV, sg);
        su = sg;
        sv = sg;
        gzw = zsrc_roll(g, kk, G_ODD, sg);
        sw = sg;
        gze = zsrc_roll(g, kk, G_EVEN, sg);
      }
      const T a0 = __ldg(ph.alpha0 + gze);
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        if (!sok[q]) continue;
        const int e = tid + q * RX * RY;
        const size_t mu = (size_t)gzu * plane + soff[q];
        const size_t mw = (size_t)gzw * plane + soff[q];
        const size_t me = (size_t)gze * plane + soff[q];
        U[s * PN + e] = su * T(0.5) * (__ldg(a.uk + mu) + __ldg(a.un + mu));
        V[s * PN + e] = sv * T(0.5) * (__ldg(a.vk + mu) + __ldg(a.vn + mu));
        W[s * PN + e] = sw * T(0.5) * (__ldg(a.wk + mw) + __ldg(a.wn + mw));
        Bb[s * PN + e] = __ldg(a.b + me);
        AP[s * PN + e] = a0 * __ldg(a.p + me);
      }
    };
    // nu_t on global plane kk from the staged planes kk-1 .. kk+1
    auto nu_plane = [&](int kk) {
      const int s = slot3(kk);
      const bool cst = ph.flags & LES_PHYS_CONST_NU, sgs = ph.flags & LES_PHYS_SGS;
      for (int e = tid; e < NNP; e += RX * RY) {
        const int x = e % NX - 1, y = e / NX - 1;
        T val;
        if (cst) {
          val = ph.nu_const;
        } else if (!sgs) {
          val = T(0);
        } else {
          const T* vel[3] = {U, V, W};
          const int sm1 = slot5(kk - 1), s0 = slot5(kk), sp1 = slot5(kk + 1);
          T gr[3][3];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const T* f = vel[c];
            gr[c][0] = (f[s0 * PN + pidx(x + 1, y)] - f[s0 * PN + pidx(x - 1, y)]) * (T(0.5) * g.idx);
            gr[c][1] = (f[s0 * PN + pidx(x, y + 1)] - f[s0 * PN + pidx(x, y - 1)]) * (T(0.5) * g.idy);
            gr[c][2] = (f[sp1 * PN + pidx(x, y)] - f[sm1 * PN + pidx(x, y)]) * (T(0.5) * g.idz);
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
          if ((ph.flags & LES_PHYS_FB) && S2 > T(0)) {
            const T N2 = (Bb[sp1 * PN + pidx(x, y)] - Bb[sm1 * PN + pidx(x, y)]) * (T(0.5) * g.idz);
            T q = T(1) - N2 / (T(1) / ph.inv_pr * S2);
            q = q < T(0) ? T(0) : (q > T(1) ? T(1) : q);
            fB = r_sqrt(q);
          }
          val = ph.cs2d2 * fB * r_sqrt(S2);
        }
        NU[s * NNP + e] = val;
      }
    };
    // a ghost plane of nu_t mirrors an interior plane (walls)
    auto nu_mirror = [&](int kk, int src) {
      for (int e = tid; e < NNP; e += RX * RY) NU[slot3(kk) * NNP + e] = NU[slot3(src) * NNP + e];
    };
    auto nu_any = [&](int kk) {
      if (g.walls && kk < 0) nu_mirror(kk, -1 - kk);
      else if (g.walls && kk >= g.nz) nu_mirror(kk, 2 * g.nz - 1 - kk);
      else nu_plane(kk);
    };

    __syncthreads();  // the previous run's readers are done with the rings
    for (int kk = k0 - 2; kk <= k0 + 1; ++kk) stage(kk);
    __syncthreads();
    if (g.walls && k0 == 0) {
      nu_plane(0);
      __syncthreads();
      nu_mirror(-1, 0);
    } else {
      nu_plane(k0 - 1);
      nu_plane(k0);
    }
    const int i = x0 + tx, j = y0 + ty;
    const bool own = i < g.nx && j < g.ny;
    const T target[3] = {ph.ug, ph.vg, T(0)};
    const T ih[3] = {g.idx, g.idy, g.idz};
    T* const out[3] = {a.ou, a.ov, a.ow};
    for (int k = k0; k < k1; ++k) {
      const size_t m = (size_t)k * plane + (size_t)j * g.nx + i;
      // global loads of this node, issued before the staging so that their
      // latency overlaps it
      T un[3] = {T(0), T(0), T(0)};
      if (own) {
        un[0] = __ldg(a.un + m);
        un[1] = __ldg(a.vn + m);
        un[2] = __ldg(a.wn + m);
      }
      const T rho[3] = {g.prof(ph.rho0, k - 1), g.prof(ph.rho0, k), g.prof(ph.rho0, k + 1)};
      __syncthreads();  // plane k-3 and nu plane k-2 are no longer read
      stage(k + 2);
      __syncthreads();
      nu_any(k + 1);
      __syncthreads();
      if (!own) continue;
      // ring planes at this node for dz = -2 .. 2; staged field f (0 u, 1 v,
      // 2 w, 3 b, 4 alpha0 p') at offset (ox, oy, oz) is one shared load at a
      // constant offset from one of five bases
      const T* pl[5];
#pragma unroll
      for (int q = 0; q < 5; ++q) pl[q] = U + slot5(k - 2 + q) * PN + pidx(tx, ty);
      const T* nl[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) nl[q] = NU + slot3(k - 1 + q) * NNP + nidx1(tx, ty);
      auto S = [&](int f, int ox, int oy, int oz) { return pl[oz + 2][f * (NRING * PN) + oy * PX + ox]; };
      auto N = [&](int ox, int oy, int oz) { return nl[oz + 1][oy * NX + ox]; };
      const T r0 = rho[1];
      const T zc = (T(k) + T(0.5)) * g.dz;
      // the six faces of the cell: mass flux F = rho0 u_d and rho0 nu_t,
      // shared by the three components
      T Ff[3][2], Kf[3][2];
      bool adv_on[3][2], flux_on[3][2];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const int di = d == 0, dj = d == 1, dk = d == 2;
#pragma unroll
        for (int side = 0; side < 2; ++side) {
          const int lx = side ? 0 : -di, ly = side ? 0 : -dj, lz = side ? 0 : -dk;
          const int gkl = k + lz;
          const T rl = rho[1 + lz], ru = rho[1 + lz + dk];
          flux_on[d][side] = !g.surface_face(d, gkl);  // free slip: no momentum flux
          adv_on[d][side] = (ph.flags & LES_PHYS_ADV) && !g.wall_face(d, gkl);
          Ff[d][side] = T(0.5) * (rl * S(d, lx, ly, lz) + ru * S(d, lx + di, ly + dj, lz + dk));
          const T nuf = T(0.5) * (N(lx, ly, lz) + N(lx + di, ly + dj, lz + dk));
          const T rhof = T(0.5) * (rl + ru);
          Kf[d][side] = rhof * nuf;
        }
      }
      T res[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int ci = c == 0, cj = c == 1, ck = c == 2;
        T R = T(0);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const int di = d == 0, dj = d == 1, dk = d == 2;
#pragma unroll
          for (int side = 0; side < 2; ++side) {
            if (!flux_on[d][side]) continue;
            const int lx = side ? 0 : -di, ly = side ? 0 : -dj, lz = side ? 0 : -dk;
            const int ux = lx + di, uy = ly + dj, uz = lz + dk;
            const T cl = S(c, lx, ly, lz), cu = S(c, ux, uy, uz);
            T adv = T(0);
            if (adv_on[d][side]) {
              const T F = Ff[d][side];
              adv = F * face_value(ADV, F, S(c, lx - di, ly - dj, lz - dk), cl, cu, S(c, ux + di, uy + dj, uz + dk));
            }
            const T dn = (cu - cl) * ih[d];
            T dtg;
            if (c == d) {
              dtg = dn;
            } else {
              const T g0 = S(d, lx + ci, ly + cj, lz + ck) - S(d, lx - ci, ly - cj, lz - ck);
              const T g1 = S(d, ux + ci, uy + cj, uz + ck) - S(d, ux - ci, uy - cj, uz - ck);
              dtg = T(0.25) * (g0 + g1) * ih[c];
            }
            const T fl = -adv + Kf[d][side] * (dn + dtg);
            R += (side ? fl : -fl) * ih[d];
          }
        }
        const T uc = S(c, 0, 0, 0);
        if ((ph.flags & LES_PHYS_BUOY) && c == 2) R += r0 * S(3, 0, 0, 0);
        if (ph.flags & LES_PHYS_CORIOLIS) {
          if (c == 0) R += ph.f_cor * r0 * (S(1, 0, 0, 0) - ph.vg);
          if (c == 1) R -= ph.f_cor * r0 * (S(0, 0, 0, 0) - ph.ug);
        }
        if ((ph.flags & LES_PHYS_SPONGE) && zc > ph.sponge_zs) {
          const T sn = r_sin(T(1.5707963267948966) * (zc - ph.sponge_zs) / (ph.sponge_h - ph.sponge_zs));
          R -= ph.sponge_rate * sn * sn * r0 * (uc - target[c]);
        }
        const T gp = (S(4, ci, cj, ck) - S(4, -ci, -cj, -ck)) * (T(0.5) * ih[c]);
        res[c] = (r0 * un[c] + ph.dt * (-r0 * gp + R)) / r0;
      }
      // stores after every shared-memory read of the node
#pragma unroll
      for (int c = 0; c < 3; ++c) out[c][m] = res[c];
    }
  }
}


// ---- a3: scalar predictor as a rolling z-march ----------------------------------
template <typename T>
struct ScaRoll {
  Grid<T> g;
  Phys<T> ph;
  int zrun, nchunk, ntx, nty;
  const T *u, *v, *w, *b, *thk, *qtk, *thh, *qth, *srad;
  T *tho, *qto;
};

template <typename T, int ADV>
__global__ void __launch_bounds__(RX* RY) k_scalar_roll(ScaRoll<T> a) {
  extern __shared__ unsigned char smraw[];
  T* U = reinterpret_cast<T*>(smraw);  // u^k rings
  T* V = U + NRING * PN;
  T* W = V + NRING * PN;
  T* Bb = W + NRING * PN;
  T* P0 = Bb + NRING * PN;  // phibar theta_l
  T* P1 = P0 + NRING * PN;  // phibar q_t
  T* NU = P1 + NRING * PN;
  const Grid<T>& g = a.g;
  const Phys<T>& ph = a.ph;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + RX * ty;
  const long long ncol = (long long)a.ntx * a.nty;
  const long long nblk = ncol * a.nchunk;
  const size_t plane = (size_t)g.nx * g.ny;
  const bool fb = ph.flags & LES_PHYS_FB;
  for (long long blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    const int col = (int)(blk % ncol), chunk = (int)(blk / ncol);
    const int x0 = (col % a.ntx) * RX, y0 = (col / a.ntx) * RY;
    const int k0 = chunk * a.zrun, k1 = min(k0 + a.zrun, g.nz);
    int soff[2];
    bool sok[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int e = tid + q * RX * RY;
      sok[q] = e < PN;
      const int bx = e % PX, by = e / PX;
      soff[q] = sok[q] ? wrap_any(y0 - RH + by, g.ny) * g.nx + wrap_any(x0 - RH + bx, g.nx) : 0;
    }
    auto stage = [&](int kk) {
      const int s = slot5(kk);
      T suv, sw, se;
      const int gzu = zsrc_roll(g, kk, G_UV, suv);
      const int gzw = zsrc_roll(g, kk, G_ODD, sw);
      const int gze = zsrc_roll(g, kk, G_EVEN, se);
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        if (!sok[q]) continue;
        const int e = tid + q * RX * RY;
        const size_t mu = (size_t)gzu * plane + soff[q];
        const size_t mw = (size_t)gzw * plane + soff[q];
        const size_t me = (size_t)gze * plane + soff[q];
        U[s * PN + e] = suv * __ldg(a.u + mu);
        V[s * PN + e] = suv * __ldg(a.v + mu);
        W[s * PN + e] = sw * __ldg(a.w + mw);
        if (fb) Bb[s * PN + e] = __ldg(a.b + me);
        P0[s * PN + e] = T(0.5) * (__ldg(a.thk + me) + __ldg(a.thh + me));
        P1[s * PN + e] = T(0.5) * (__ldg(a.qtk + me) + __ldg(a.qth + me));
      }
    };
    auto nu_plane = [&](int kk) {
      const int s = slot3(kk);
      const bool cst = ph.flags & LES_PHYS_CONST_NU, sgs = ph.flags & LES_PHYS_SGS;
      for (int e = tid; e < NNP; e += RX * RY) {
        const int x = e % NX - 1, y = e / NX - 1;
        T val;
        if (cst) {
          val = ph.nu_const;
        } else if (!sgs) {
          val = T(0);
        } else {
          const T* vel[3] = {U, V, W};
          const int sm1 = slot5(kk - 1), s0 = slot5(kk), sp1 = slot5(kk + 1);
          T gr[3][3];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const T* f = vel[c];
            gr[c][0] = (f[s0 * PN + pidx(x + 1, y)] - f[s0 * PN + pidx(x - 1, y)]) * (T(0.5) * g.idx);
            gr[c][1] = (f[s0 * PN + pidx(x, y + 1)] - f[s0 * PN + pidx(x, y - 1)]) * (T(0.5) * g.idy);
            gr[c][2] = (f[sp1 * PN + pidx(x, y)] - f[sm1 * PN + pidx(x, y)]) * (T(0.5) * g.idz);
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
            const T N2 = (Bb[sp1 * PN + pidx(x, y)] - Bb[sm1 * PN + pidx(x, y)]) * (T(0.5) * g.idz);
            T q = T(1) - N2 / (T(1) / ph.inv_pr * S2);
            q = q < T(0) ? T(0) : (q > T(1) ? T(1) : q);
            fB = r_sqrt(q);
          }
          val = ph.cs2d2 * fB * r_sqrt(S2);
        }
        NU[s * NNP + e] = val;
      }
    };
    auto nu_mirror = [&](int kk, int src) {
      for (int e = tid; e < NNP; e += RX * RY) NU[slot3(kk) * NNP + e] = NU[slot3(src) * NNP + e];
    };
    auto nu_any = [&](int kk) {
      if (g.walls && kk < 0) nu_mirror(kk, -1 - kk);
      else if (g.walls && kk >= g.nz) nu_mirror(kk, 2 * g.nz - 1 - kk);
      else nu_plane(kk);
    };
    __syncthreads();
    for (int kk = k0 - 2; kk <= k0 + 1; ++kk) stage(kk);
    __syncthreads();
    if (g.walls && k0 == 0) {
      nu_plane(0);
      __syncthreads();
      nu_mirror(-1, 0);
    } else {
      nu_plane(k0 - 1);
      nu_plane(k0);
    }
    const int i = x0 + tx, j = y0 + ty;
    const bool own = i < g.nx && j < g.ny;
    const T inv_s[2] = {ph.inv_pr, ph.inv_sc};
    const T sflux[2] = {ph.sflux_th, ph.sflux_qt};
    const T ih[3] = {g.idx, g.idy, g.idz};
    for (int k = k0; k < k1; ++k) {
      const size_t m = (size_t)k * plane + (size_t)j * g.nx + i;
      // global loads of this node, issued before the staging
      T half[2] = {T(0), T(0)}, rad = T(0);
      if (own) {
        half[0] = __ldg(a.thh + m);
        half[1] = __ldg(a.qth + m);
        if (ph.flags & LES_PHYS_RAD) rad = __ldg(a.srad + m);
      }
      const T rho[3] = {g.prof(ph.rho0, k - 1), g.prof(ph.rho0, k), g.prof(ph.rho0, k + 1)};
      __syncthreads();
      stage(k + 2);
      __syncthreads();
      nu_any(k + 1);
      __syncthreads();
      if (!own) continue;
      // ring planes at this node for dz = -2 .. 2; field f: 0 u, 1 v, 2 w,
      // 3 b, 4 phibar theta_l, 5 phibar q_t
      const T* pl[5];
#pragma unroll
      for (int q = 0; q < 5; ++q) pl[q] = U + slot5(k - 2 + q) * PN + pidx(tx, ty);
      const T* nl[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) nl[q] = NU + slot3(k - 1 + q) * NNP + nidx1(tx, ty);
      auto S = [&](int f, int ox, int oy, int oz) { return pl[oz + 2][f * (NRING * PN) + oy * PX + ox]; };
      auto N = [&](int ox, int oy, int oz) { return nl[oz + 1][oy * NX + ox]; };
      const T r0 = rho[1];
      T tend[2] = {T(0), T(0)};
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const int di = d == 0, dj = d == 1, dk = d == 2;
#pragma unroll
        for (int side = 0; side < 2; ++side) {
          const int lx = side ? 0 : -di, ly = side ? 0 : -dj, lz = side ? 0 : -dk;
          const int ux = lx + di, uy = ly + dj, uz = lz + dk;
          const int gkl = k + lz;
          T fl[2];
          if (g.wall_face(d, gkl)) {
            const bool sfc = g.surface_face(d, gkl) && (ph.flags & LES_PHYS_SFC);
            fl[0] = sfc ? -sflux[0] : T(0);
            fl[1] = sfc ? -sflux[1] : T(0);
          } else {
            const T rl = rho[1 + lz], ru = rho[1 + lz + dk];
            T F = T(0);
            if (ph.flags & LES_PHYS_ADV) F = T(0.5) * (rl * S(d, lx, ly, lz) + ru * S(d, ux, uy, uz));
            const T nuf = T(0.5) * (N(lx, ly, lz) + N(ux, uy, uz));
            const T rhof = T(0.5) * (rl + ru);
            const T K = rhof * nuf;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
              const T b0 = S(4 + q, lx, ly, lz), b1 = S(4 + q, ux, uy, uz);
              T adv = T(0);
              if (ph.flags & LES_PHYS_ADV)
                adv = F * face_value(ADV, F, S(4 + q, lx - di, ly - dj, lz - dk), b0, b1, S(4 + q, ux + di, uy + dj, uz + dk));
              fl[q] = -adv + K * inv_s[q] * (b1 - b0) * ih[d];
            }
          }
#pragma unroll
          for (int q = 0; q < 2; ++q) tend[q] += (side ? fl[q] : -fl[q]) * ih[d];
        }
      }
      if (ph.flags & LES_PHYS_SUBS) {
        const T wsub = ph.subs_div * (T(k) + T(0.5)) * g.dz;
#pragma unroll
        for (int q = 0; q < 2; ++q) tend[q] += r0 * wsub * (S(4 + q, 0, 0, 1) - S(4 + q, 0, 0, 0)) * g.idz;
      }
      if (ph.flags & LES_PHYS_RAD) tend[0] += rad;
      a.tho[m] = (r0 * half[0] + ph.dt * tend[0]) / r0;
      a.qto[m] = (r0 * half[1] + ph.dt * tend[1]) / r0;
    }
  }
}

// ---- a4 (second half): Poisson right side as per-column z-marches ----------------
// rhs = (alpha0 / dt) D(rho0 u^) - C(psi) (compact operator, Appendix A) or
// D(rho0 u^) / dt (consistent operator).  One thread per column: the z
// neighbours of w^ and psi live in register windows that roll with k; the
// x / y neighbours are plain loads that the L1 serves for the warp's row.
template <typename T>
struct RhsRoll {
  Grid<T> g;
  Phys<T> ph;
  int op, zrun, nchunk;
  const T *ou, *ov, *ow, *psi;
  T* rhs;
};

template <typename T>
__global__ void __launch_bounds__(256) k_rhs_roll(RhsRoll<T> a) {
  const Grid<T>& g = a.g;
  const Phys<T>& ph = a.ph;
  const long long ncol = (long long)g.nx * g.ny;
  const long long nitem = ncol * a.nchunk;
  const size_t plane = (size_t)ncol;
  const T hx = T(0.5) * g.idx, hy = T(0.5) * g.idy, hz = T(0.5) * g.idz;
  const T c4x = T(0.25) * g.idx * g.idx, c4y = T(0.25) * g.idy * g.idy, c4z = T(0.25) * g.idz * g.idz;
  for (long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x; it < nitem;
       it += (long long)gridDim.x * blockDim.x) {
    const long long col = it % ncol;
    const int chunk = (int)(it / ncol);
    const int i = (int)(col % g.nx), j = (int)(col / g.nx);
    const int k0 = chunk * a.zrun, k1 = min(k0 + a.zrun, g.nz);
    const int xm1 = wrap_any(i - 1, g.nx), xp1 = wrap_any(i + 1, g.nx);
    const int xm2 = wrap_any(i - 2, g.nx), xp2 = wrap_any(i + 2, g.nx);
    const size_t rj = (size_t)j * g.nx;
    const size_t ym1 = (size_t)wrap_any(j - 1, g.ny) * g.nx, yp1 = (size_t)wrap_any(j + 1, g.ny) * g.nx;
    const size_t ym2 = (size_t)wrap_any(j - 2, g.ny) * g.nx, yp2 = (size_t)wrap_any(j + 2, g.ny) * g.nx;
    // psi on planes k-2 .. k+2 and w^ on planes k-1 .. k+1 of this column
    T ps[5], wz[3];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      T sg;
      ps[q] = __ldg(a.psi + (size_t)zsrc_roll(g, k0 - 2 + q, G_EVEN, sg) * plane + rj + i);
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      T sg;
      const int kk = zsrc_roll(g, k0 - 1 + q, G_ODD, sg);
      wz[q] = sg * __ldg(a.ow + (size_t)kk * plane + rj + i);
    }
    for (int k = k0; k < k1; ++k) {
      const size_t pk = (size_t)k * plane;
      const T r0 = g.prof(ph.rho0, k);
      T div = (r0 * __ldg(a.ou + pk + rj + xp1) - r0 * __ldg(a.ou + pk + rj + xm1)) * hx;
      div += (r0 * __ldg(a.ov + pk + yp1 + i) - r0 * __ldg(a.ov + pk + ym1 + i)) * hy;
      div += (g.prof(ph.rho0, k + 1) * wz[2] - g.prof(ph.rho0, k - 1) * wz[0]) * hz;
      T val;
      if (a.op == LES_OP_COMPACT) {
        const T* pp = a.psi + pk;
        const T c = ps[2];
        T C = (__ldg(pp + rj + xp2) - T(4) * __ldg(pp + rj + xp1) + T(6) * c - T(4) * __ldg(pp + rj + xm1) +
               __ldg(pp + rj + xm2)) * c4x;
        C += (__ldg(pp + yp2 + i) - T(4) * __ldg(pp + yp1 + i) + T(6) * c - T(4) * __ldg(pp + ym1 + i) +
              __ldg(pp + ym2 + i)) * c4y;
        C += (ps[4] - T(4) * ps[3] + T(6) * c - T(4) * ps[1] + ps[0]) * c4z;
        val = __ldg(ph.alpha0 + k) / ph.dt * div - C;
      } else {
        val = div / ph.dt;
      }
      a.rhs[pk + rj + i] = val;
      // roll the windows up one plane
#pragma unroll
      for (int q = 0; q < 4; ++q) ps[q] = ps[q + 1];
      wz[0] = wz[1];
      wz[1] = wz[2];
      if (k + 1 < k1) {
        T sg;
        ps[4] = __ldg(a.psi + (size_t)zsrc_roll(g, k + 3, G_EVEN, sg) * plane + rj + i);
        const int kk = zsrc_roll(g, k + 2, G_ODD, sg);
        wz[2] = sg * __ldg(a.ow + (size_t)kk * plane + rj + i);
      }
    }
  }
}

// z-runs: at least `blocks` (column, run) items to fill the GPU, runs as
// long as possible
inline void roll_runs(int nx, int ny, int nz, long long blocks, int& ntx, int& nty, int& zrun, int& nchunk) {
  ntx = (nx + RX - 1) / RX;
  nty = (ny + RY - 1) / RY;
  const long long ncol = (long long)ntx * nty;
  const int want = (int)std::max<long long>(1, std::min<long long>((long long)nz, (blocks + ncol - 1) / ncol));
  zrun = (nz + want - 1) / want;
  nchunk = (nz + zrun - 1) / zrun;
}

}  // namespace

template <typename T>
cudaError_t launch_rhs_roll(const StageArgs<T>& a, int max_blocks, int op, const T* ou, const T* ov, const T* ow,
                            const T* psi, T* rhs) {
  RhsRoll<T> r;
  r.g = a.g;
  r.ph = a.ph;
  r.op = op;
  r.ou = ou;
  r.ov = ov;
  r.ow = ow;
  r.psi = psi;
  r.rhs = rhs;
  // one thread per (column, z-run): enough threads for four 256-thread
  // blocks per SM (max_blocks is eight per SM), runs as long as possible
  const long long ncol = (long long)a.g.nx * a.g.ny;
  const long long want = (long long)(max_blocks / 2) * 256;
  const long long nch = std::max<long long>(1, std::min<long long>(a.g.nz, (want + ncol - 1) / ncol));
  r.zrun = (int)((a.g.nz + nch - 1) / nch);
  r.nchunk = (a.g.nz + r.zrun - 1) / r.zrun;
  const long long nitem = ncol * r.nchunk;
  const unsigned grid = (unsigned)std::min<long long>((nitem + 255) / 256, 1LL << 20);
  ProfScope ps(a.prof, KI_RHS, a.st);
  k_rhs_roll<T><<<grid, 256, 0, a.st>>>(r);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_scalar_roll(const StageArgs<T>& a, int max_blocks, const T* u, const T* v, const T* w,
                               const T* b, const T* thk, const T* qtk, const T* thh, const T* qth, const T* srad,
                               T* th_out, T* qt_out) {
  ScaRoll<T> r;
  r.g = a.g;
  r.ph = a.ph;
  // max_blocks is eight blocks per SM: aim at four resident per SM
  roll_runs(a.g.nx, a.g.ny, a.g.nz, max_blocks / 2, r.ntx, r.nty, r.zrun, r.nchunk);
  r.u = u;
  r.v = v;
  r.w = w;
  r.b = b;
  r.thk = thk;
  r.qtk = qtk;
  r.thh = thh;
  r.qth = qth;
  r.srad = srad;
  r.tho = th_out;
  r.qto = qt_out;
  const size_t smem = (size_t)(6 * NRING * PN + 3 * NNP) * sizeof(T);
  // the advection scheme is a template parameter: no per-face branch on it
  auto kern = a.ph.advection == LES_ADV_WENO3 ? k_scalar_roll<T, LES_ADV_WENO3> : k_scalar_roll<T, LES_ADV_QUICK>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long nblk = (long long)r.ntx * r.nty * r.nchunk;
  const unsigned grid = (unsigned)std::min<long long>(nblk, (long long)max_blocks * 4);
  ProfScope ps(a.prof, KI_SCALAR, a.st);
  kern<<<grid, dim3(RX, RY), smem, a.st>>>(r);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_momentum_roll(const StageArgs<T>& a, int max_blocks, const T* uk, const T* vk, const T* wk,
                                 const T* un, const T* vn, const T* wn, const T* p, const T* b, T* ou, T* ov,
                                 T* ow) {
  MomRoll<T> m;
  m.g = a.g;
  m.ph = a.ph;
  roll_runs(a.g.nx, a.g.ny, a.g.nz, max_blocks / 2, m.ntx, m.nty, m.zrun, m.nchunk);
  const long long ncol = (long long)m.ntx * m.nty;
  m.uk = uk;
  m.vk = vk;
  m.wk = wk;
  m.un = un;
  m.vn = vn;
  m.wn = wn;
  m.p = p;
  m.b = b;
  m.ou = ou;
  m.ov = ov;
  m.ow = ow;
  const size_t smem = (size_t)(5 * NRING * PN + 3 * NNP) * sizeof(T);
  auto kern = a.ph.advection == LES_ADV_WENO3 ? k_momentum_roll<T, LES_ADV_WENO3> : k_momentum_roll<T, LES_ADV_QUICK>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long nblk = ncol * m.nchunk;
  const unsigned grid = (unsigned)std::min<long long>(nblk, (long long)max_blocks * 4);
  ProfScope ps(a.prof, KI_MOMENTUM, a.st);
  kern<<<grid, dim3(RX, RY), smem, a.st>>>(m);
  return cudaGetLastError();
}

template cudaError_t launch_rhs_roll<float>(const StageArgs<float>&, int, int, const float*, const float*,
                                            const float*, const float*, float*);
template cudaError_t launch_rhs_roll<double>(const StageArgs<double>&, int, int, const double*, const double*,
                                             const double*, const double*, double*);
template cudaError_t launch_scalar_roll<float>(const StageArgs<float>&, int, const float*, const float*,
                                               const float*, const float*, const float*, const float*, const float*,
                                               const float*, const float*, float*, float*);
template cudaError_t launch_scalar_roll<double>(const StageArgs<double>&, int, const double*, const double*,
                                                const double*, const double*, const double*, const double*,
                                                const double*, const double*, const double*, double*, double*);
template cudaError_t launch_momentum_roll<float>(const StageArgs<float>&, int, const float*, const float*,
                                                 const float*, const float*, const float*, const float*,
                                                 const float*, const float*, float*, float*, float*);
template cudaError_t launch_momentum_roll<double>(const StageArgs<double>&, int, const double*, const double*,
                                                  const double*, const double*, const double*, const double*,
                                                  const double*, const double*, double*, double*, double*);

}  // namespace les
