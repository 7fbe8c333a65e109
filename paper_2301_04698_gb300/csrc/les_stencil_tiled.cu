// les_stencil_tiled.cu -- shared-memory tiled scalar and momentum predictors.
//
// Same discretisation as les_stencil.cu (Sec. 2.3-2.4: QUICK advection,
// Smagorinsky-Lilly viscosity with f_B, 2nd-order central SGS fluxes,
// buoyancy, Coriolis, sponge, subsidence, radiation and surface fluxes), laid
// out for the GPU: a 32 x 8 thread block owns a 32 x 8 x TZ tile and first
// stages each input over the tile plus a halo of two nodes in shared memory,
// applying the periodic wrap and the wall ghost rules once while loading;
// u^{n+1/2} = (u^k + u^n)/2 and phibar = (phi^k + phi^{n+1/2})/2 are formed
// on load.  nu_t is then computed for the tile plus a halo of one node from
// the staged velocities (never stored in HBM), and every flux reads shared
// memory at fixed offsets.
#include "les_internal.h"

namespace les {
namespace {

constexpr int BTX = 32, BTY = 8, BTZ = 4, BH = 2;
constexpr int BX = BTX + 2 * BH, BY = BTY + 2 * BH, BZ = BTZ + 2 * BH;
constexpr int BN = BX * BY * BZ;  // nodes of a halo-2 box
constexpr int NX1 = BTX + 2, NY1 = BTY + 2, NZ1 = BTZ + 2;
constexpr int NN = NX1 * NY1 * NZ1;  // nodes of the halo-1 nu box

__device__ __forceinline__ double mx_sqrt(double a) { return sqrt(a); }
__device__ __forceinline__ float mx_sqrt(float a) { return sqrtf(a); }
__device__ __forceinline__ double mx_sin(double a) { return sin(a); }
__device__ __forceinline__ float mx_sin(float a) { return sinf(a); }

// halo-2 box index of local node (x, y, z), x in [-2, BTX+2) ...
__device__ __forceinline__ int bidx(int x, int y, int z) { return ((z + BH) * BY + (y + BH)) * BX + (x + BH); }
// halo-1 nu box index
__device__ __forceinline__ int nidx(int x, int y, int z) { return ((z + 1) * NY1 + (y + 1)) * NX1 + (x + 1); }

__device__ __forceinline__ int wrapm(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

// global plane and sign of box plane gk under ghost rule g
template <typename T>
__device__ __forceinline__ int zsrc(const Grid<T>& g, int gk, int gh, T& sgn) {
  sgn = T(1);
  if (!g.walls) return wrapm(gk, g.nz);
  if (gk < 0) {
    gk = -1 - gk;
    if (gh == G_ODD) sgn = T(-1);
  } else if (gk >= g.nz) {
    gk = 2 * g.nz - 1 - gk;
    if (gh != G_EVEN) sgn = T(-1);
  }
  return gk < 0 ? 0 : (gk >= g.nz ? g.nz - 1 : gk);  // far planes: any valid data (unused)
}

// stage f (or (f + f2)/2) over the halo-2 box of the tile at (x0, y0, k0)
template <typename T>
__device__ __forceinline__ void load_box(T* __restrict__ s, const Grid<T>& g, const T* __restrict__ f,
                                         const T* __restrict__ f2, int gh, int x0, int y0, int k0) {
  const int tid = threadIdx.x + BTX * threadIdx.y;
  for (int e = tid; e < BN; e += BTX * BTY) {
    const int bx = e % BX, by = (e / BX) % BY, bz = e / (BX * BY);
    const int gx = wrapm(x0 - BH + bx, g.nx), gy = wrapm(y0 - BH + by, g.ny);
    T sgn;
    const int gz = zsrc(g, k0 - BH + bz, gh, sgn);
    const size_t m = ((size_t)gz * g.ny + gy) * g.nx + gx;
    T v = __ldg(f + m);
    if (f2) v = T(0.5) * (v + __ldg(f2 + m));
    s[e] = sgn * v;
  }
}

// local z of the node whose nu a ghost plane mirrors (walls), else z itself
template <typename T>
__device__ __forceinline__ int nu_src_z(const Grid<T>& g, int k0, int lz) {
  if (!g.walls) return lz;
  const int gk = k0 + lz;
  if (gk < 0) return -1 - gk - k0;
  if (gk >= g.nz) return 2 * g.nz - 1 - gk - k0;
  return lz;
}

// nu_t over the halo-1 box from the staged velocities and buoyancy
template <typename T>
__device__ __forceinline__ void nu_box(T* __restrict__ nu, const T* __restrict__ U, const T* __restrict__ V,
                                       const T* __restrict__ W, const T* __restrict__ B, const Grid<T>& g,
                                       const Phys<T>& ph, int k0) {
  const int tid = threadIdx.x + BTX * threadIdx.y;
  const bool cst = ph.flags & LES_PHYS_CONST_NU;
  const bool sgs = ph.flags & LES_PHYS_SGS;
  for (int e = tid; e < NN; e += BTX * BTY) {
    const int x = e % NX1 - 1, y = (e / NX1) % NY1 - 1, z0 = e / (NX1 * NY1) - 1;
    T val;
    if (cst) {
      val = ph.nu_const;
    } else if (!sgs) {
      val = T(0);
    } else {
      const int z = nu_src_z(g, k0, z0);
      const T* vel[3] = {U, V, W};
      T gr[3][3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        gr[c][0] = (vel[c][bidx(x + 1, y, z)] - vel[c][bidx(x - 1, y, z)]) * (T(0.5) * g.idx);
        gr[c][1] = (vel[c][bidx(x, y + 1, z)] - vel[c][bidx(x, y - 1, z)]) * (T(0.5) * g.idy);
        gr[c][2] = (vel[c][bidx(x, y, z + 1)] - vel[c][bidx(x, y, z - 1)]) * (T(0.5) * g.idz);
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
        const T N2 = (B[bidx(x, y, z + 1)] - B[bidx(x, y, z - 1)]) * (T(0.5) * g.idz);
        T q = T(1) - N2 / (T(1) / ph.inv_pr * S2);
        q = q < T(0) ? T(0) : (q > T(1) ? T(1) : q);
        fB = mx_sqrt(q);
      }
      val = ph.cs2d2 * fB * mx_sqrt(S2);
    }
    nu[e] = val;
  }
}


template <typename T>
__device__ __forceinline__ void tile_of(const Grid<T>& g, long long t, int& x0, int& y0, int& k0) {
  const int ntx = (g.nx + BTX - 1) / BTX, nty = (g.ny + BTY - 1) / BTY;
  x0 = (int)(t % ntx) * BTX;
  const long long r = t / ntx;
  y0 = (int)(r % nty) * BTY;
  k0 = (int)(r / nty) * BTZ;
}

// ---- a3: scalar predictor --------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(BTX* BTY)
    k_scalar_tiled(Grid<T> g, Phys<T> ph, long long ntiles, const T* __restrict__ u, const T* __restrict__ v,
                   const T* __restrict__ w, const T* __restrict__ b, const T* __restrict__ thk,
                   const T* __restrict__ qtk, const T* __restrict__ thh, const T* __restrict__ qth,
                   const T* __restrict__ srad, T* __restrict__ tho, T* __restrict__ qto) {
  extern __shared__ unsigned char smraw[];
  T* U = reinterpret_cast<T*>(smraw);
  T* V = U + BN;
  T* W = V + BN;
  T* Bb = W + BN;
  T* P0 = Bb + BN;  // phibar theta_l
  T* P1 = P0 + BN;  // phibar q_t
  T* NU = P1 + BN;
  const T* vel[3] = {U, V, W};
  const T* bar[2] = {P0, P1};
  const T inv_s[2] = {ph.inv_pr, ph.inv_sc};
  const T sflux[2] = {ph.sflux_th, ph.sflux_qt};
  const T ih[3] = {g.idx, g.idy, g.idz};
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    int x0, y0, k0;
    tile_of(g, t, x0, y0, k0);
    __syncthreads();
    load_box(U, g, u, (const T*)nullptr, G_UV, x0, y0, k0);
    load_box(V, g, v, (const T*)nullptr, G_UV, x0, y0, k0);
    load_box(W, g, w, (const T*)nullptr, G_ODD, x0, y0, k0);
    if (ph.flags & LES_PHYS_FB) load_box(Bb, g, b, (const T*)nullptr, G_EVEN, x0, y0, k0);
    load_box(P0, g, thk, thh, G_EVEN, x0, y0, k0);
    load_box(P1, g, qtk, qth, G_EVEN, x0, y0, k0);
    __syncthreads();
    nu_box(NU, U, V, W, Bb, g, ph, k0);
    __syncthreads();
    const int x = threadIdx.x, y = threadIdx.y;
    const int i = x0 + x, j = y0 + y;
    if (i >= g.nx || j >= g.ny) continue;
    for (int z = 0; z < BTZ; ++z) {
      const int k = k0 + z;
      if (k >= g.nz) break;
      T tend[2] = {T(0), T(0)};
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const int di = d == 0, dj = d == 1, dk = d == 2;
#pragma unroll
        for (int side = 0; side < 2; ++side) {
          const int lx = x - (side ? 0 : di), ly = y - (side ? 0 : dj), lz = z - (side ? 0 : dk);
          const int ux = lx + di, uy = ly + dj, uz = lz + dk;
          const int gkl = k0 + lz;
          T fl[2];
          if (g.wall_face(d, gkl)) {
            const bool sfc = g.surface_face(d, gkl) && (ph.flags & LES_PHYS_SFC);
            fl[0] = sfc ? -sflux[0] : T(0);
            fl[1] = sfc ? -sflux[1] : T(0);
          } else {
            T F = T(0);
            if (ph.flags & LES_PHYS_ADV)
              F = T(0.5) * (g.prof(ph.rho0, gkl) * vel[d][bidx(lx, ly, lz)] +
                            g.prof(ph.rho0, gkl + dk) * vel[d][bidx(ux, uy, uz)]);
            const T nuf = T(0.5) * (NU[nidx(lx, ly, lz)] + NU[nidx(ux, uy, uz)]);
            const T rhof = T(0.5) * (g.prof(ph.rho0, gkl) + g.prof(ph.rho0, gkl + dk));
#pragma unroll
            for (int q = 0; q < 2; ++q) {
              const T b0 = bar[q][bidx(lx, ly, lz)], b1 = bar[q][bidx(ux, uy, uz)];
              T adv = T(0);
              if (ph.flags & LES_PHYS_ADV)
                adv = F * face_value(ph.advection, F, bar[q][bidx(lx - di, ly - dj, lz - dk)], b0, b1,
                                 bar[q][bidx(ux + di, uy + dj, uz + dk)]);
              fl[q] = -adv + rhof * nuf * inv_s[q] * (b1 - b0) * ih[d];
            }
          }
#pragma unroll
          for (int q = 0; q < 2; ++q) tend[q] += (side ? fl[q] : -fl[q]) * ih[d];
        }
      }
      const size_t m = g.lin(i, j, k);
      const T r0 = ph.rho0[k];
      if (ph.flags & LES_PHYS_SUBS) {
        const T wsub = ph.subs_div * (T(k) + T(0.5)) * g.dz;
#pragma unroll
        for (int q = 0; q < 2; ++q)
          tend[q] += r0 * wsub * (bar[q][bidx(x, y, z + 1)] - bar[q][bidx(x, y, z)]) * g.idz;
      }
      if (ph.flags & LES_PHYS_RAD) tend[0] += srad[m];
      tho[m] = (r0 * thh[m] + ph.dt * tend[0]) / r0;
      qto[m] = (r0 * qth[m] + ph.dt * tend[1]) / r0;
    }
  }
}

// ---- a4: momentum predictor ------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(BTX* BTY)
    k_momentum_tiled(Grid<T> g, Phys<T> ph, long long ntiles, const T* __restrict__ uk, const T* __restrict__ vk,
                     const T* __restrict__ wk, const T* __restrict__ un, const T* __restrict__ vn,
                     const T* __restrict__ wn, const T* __restrict__ p, const T* __restrict__ b,
                     T* __restrict__ ou, T* __restrict__ ov, T* __restrict__ ow) {
  extern __shared__ unsigned char smraw[];
  T* U = reinterpret_cast<T*>(smraw);  // u^{n+1/2}
  T* V = U + BN;
  T* W = V + BN;
  T* Bb = W + BN;
  T* AP = Bb + BN;  // alpha0 p
  T* NU = AP + BN;
  const T* vel[3] = {U, V, W};
  const T* veln[3] = {un, vn, wn};
  T* out[3] = {ou, ov, ow};
  const T target[3] = {ph.ug, ph.vg, T(0)};
  const T ih[3] = {g.idx, g.idy, g.idz};
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    int x0, y0, k0;
    tile_of(g, t, x0, y0, k0);
    __syncthreads();
    load_box(U, g, uk, un, G_UV, x0, y0, k0);
    load_box(V, g, vk, vn, G_UV, x0, y0, k0);
    load_box(W, g, wk, wn, G_ODD, x0, y0, k0);
    load_box(Bb, g, b, (const T*)nullptr, G_EVEN, x0, y0, k0);
    {
      // alpha0 p' with the pressure's mirror ghosts
      const int tid = threadIdx.x + BTX * threadIdx.y;
      for (int e = tid; e < BN; e += BTX * BTY) {
        const int bx = e % BX, by = (e / BX) % BY, bz = e / (BX * BY);
        const int gx = wrapm(x0 - BH + bx, g.nx), gy = wrapm(y0 - BH + by, g.ny);
        T sgn;
        const int gz = zsrc(g, k0 - BH + bz, G_EVEN, sgn);
        AP[e] = __ldg(ph.alpha0 + gz) * __ldg(p + ((size_t)gz * g.ny + gy) * g.nx + gx);
      }
    }
    __syncthreads();
    nu_box(NU, U, V, W, Bb, g, ph, k0);
    __syncthreads();
    const int x = threadIdx.x, y = threadIdx.y;
    const int i = x0 + x, j = y0 + y;
    if (i >= g.nx || j >= g.ny) continue;
    for (int z = 0; z < BTZ; ++z) {
      const int k = k0 + z;
      if (k >= g.nz) break;
      const size_t m = g.lin(i, j, k);
      const T r0 = ph.rho0[k];
      const T zc = (T(k) + T(0.5)) * g.dz;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int ci = c == 0, cj = c == 1, ck = c == 2;
        T R = T(0);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const int di = d == 0, dj = d == 1, dk = d == 2;
#pragma unroll
          for (int side = 0; side < 2; ++side) {
            const int lx = x - (side ? 0 : di), ly = y - (side ? 0 : dj), lz = z - (side ? 0 : dk);
            const int ux = lx + di, uy = ly + dj, uz = lz + dk;
            const int gkl = k0 + lz;
            if (g.surface_face(d, gkl)) continue;  // free slip, no momentum flux
            T adv = T(0);
            if ((ph.flags & LES_PHYS_ADV) && !g.wall_face(d, gkl)) {
              const T F = T(0.5) * (g.prof(ph.rho0, gkl) * vel[d][bidx(lx, ly, lz)] +
                                    g.prof(ph.rho0, gkl + dk) * vel[d][bidx(ux, uy, uz)]);
              adv = F * face_value(ph.advection, F, vel[c][bidx(lx - di, ly - dj, lz - dk)], vel[c][bidx(lx, ly, lz)],
                               vel[c][bidx(ux, uy, uz)], vel[c][bidx(ux + di, uy + dj, uz + dk)]);
            }
            const T dn = (vel[c][bidx(ux, uy, uz)] - vel[c][bidx(lx, ly, lz)]) * ih[d];
            T dtg;
            if (c == d) {
              dtg = dn;
            } else {
              const T g0 = vel[d][bidx(lx + ci, ly + cj, lz + ck)] - vel[d][bidx(lx - ci, ly - cj, lz - ck)];
              const T g1 = vel[d][bidx(ux + ci, uy + cj, uz + ck)] - vel[d][bidx(ux - ci, uy - cj, uz - ck)];
              dtg = T(0.25) * (g0 + g1) * ih[c];
            }
            const T nuf = T(0.5) * (NU[nidx(lx, ly, lz)] + NU[nidx(ux, uy, uz)]);
            const T rhof = T(0.5) * (g.prof(ph.rho0, gkl) + g.prof(ph.rho0, gkl + dk));
            const T fl = -adv + rhof * nuf * (dn + dtg);
            R += (side ? fl : -fl) * ih[d];
          }
        }
        const T uc = vel[c][bidx(x, y, z)];
        if ((ph.flags & LES_PHYS_BUOY) && c == 2) R += r0 * Bb[bidx(x, y, z)];
        if (ph.flags & LES_PHYS_CORIOLIS) {
          if (c == 0) R += ph.f_cor * r0 * (vel[1][bidx(x, y, z)] - ph.vg);
          if (c == 1) R -= ph.f_cor * r0 * (vel[0][bidx(x, y, z)] - ph.ug);
        }
        if ((ph.flags & LES_PHYS_SPONGE) && zc > ph.sponge_zs) {
          const T s = mx_sin(T(1.5707963267948966) * (zc - ph.sponge_zs) / (ph.sponge_h - ph.sponge_zs));
          R -= ph.sponge_rate * s * s * r0 * (uc - target[c]);
        }
        const T gp = (AP[bidx(x + ci, y + cj, z + ck)] - AP[bidx(x - ci, y - cj, z - ck)]) * (T(0.5) * ih[c]);
        out[c][m] = (r0 * veln[c][m] + ph.dt * (-r0 * gp + R)) / r0;
      }
    }
  }
}

template <typename T>
LaunchCfg tiled_launch(const Grid<T>& g, int max_blocks, long long& ntiles) {
  const long long ntx = (g.nx + BTX - 1) / BTX, nty = (g.ny + BTY - 1) / BTY, ntz = (g.nz + BTZ - 1) / BTZ;
  ntiles = ntx * nty * ntz;
  LaunchCfg lc;
  lc.block = dim3(BTX, BTY, 1);
  lc.grid = dim3((unsigned)std::min<long long>(ntiles, (long long)max_blocks), 1, 1);
  return lc;
}

}  // namespace

template <typename T>
cudaError_t launch_scalar_tiled(const StageArgs<T>& a, int max_blocks, const T* u, const T* v, const T* w,
                                const T* b, const T* thk, const T* qtk, const T* thh, const T* qth,
                                const T* srad, T* th_out, T* qt_out) {
  long long ntiles = 0;
  const LaunchCfg lc = tiled_launch(a.g, max_blocks, ntiles);
  const size_t smem = (size_t)(6 * BN + NN) * sizeof(T);
  cudaError_t e = cudaFuncSetAttribute(k_scalar_tiled<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  ProfScope ps(a.prof, KI_SCALAR, a.st);
  k_scalar_tiled<T><<<lc.grid, lc.block, smem, a.st>>>(a.g, a.ph, ntiles, u, v, w, b, thk, qtk, thh, qth, srad,
                                                       th_out, qt_out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_momentum_tiled(const StageArgs<T>& a, int max_blocks, const T* uk, const T* vk, const T* wk,
                                  const T* un, const T* vn, const T* wn, const T* p, const T* b, T* ou, T* ov,
                                  T* ow) {
  long long ntiles = 0;
  const LaunchCfg lc = tiled_launch(a.g, max_blocks, ntiles);
  const size_t smem = (size_t)(5 * BN + NN) * sizeof(T);
  cudaError_t e =
      cudaFuncSetAttribute(k_momentum_tiled<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  ProfScope ps(a.prof, KI_MOMENTUM, a.st);
  k_momentum_tiled<T><<<lc.grid, lc.block, smem, a.st>>>(a.g, a.ph, ntiles, uk, vk, wk, un, vn, wn, p, b, ou, ov,
                                                         ow);
  return cudaGetLastError();
}

template cudaError_t launch_scalar_tiled<float>(const StageArgs<float>&, int, const float*, const float*,
                                                const float*, const float*, const float*, const float*,
                                                const float*, const float*, const float*, float*, float*);
template cudaError_t launch_scalar_tiled<double>(const StageArgs<double>&, int, const double*, const double*,
                                                 const double*, const double*, const double*, const double*,
                                                 const double*, const double*, const double*, double*, double*);
template cudaError_t launch_momentum_tiled<float>(const StageArgs<float>&, int, const float*, const float*,
                                                  const float*, const float*, const float*, const float*,
                                                  const float*, const float*, float*, float*, float*);
template cudaError_t launch_momentum_tiled<double>(const StageArgs<double>&, int, const double*, const double*,
                                                   const double*, const double*, const double*, const double*,
                                                   const double*, const double*, double*, double*, double*);

}  // namespace les
