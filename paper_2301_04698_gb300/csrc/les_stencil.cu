// les_stencil.cu -- explicit stencil stages of one LES time step on sm_103a.
//
// Sec. 2.1-2.3 (thermodynamics, buoyancy, Smagorinsky-Lilly viscosity, sponge)
// and Sec. 2.4 (QUICK advection, 2nd-order central diffusion, the momentum and
// scalar predictors of the iterative predictor-corrector scheme, the Poisson
// right side with the Appendix A fourth-difference term, the correction).
//
// Every kernel walks 32x8-thread tiles grid-stride and marches each thread
// through a run of z-planes; all loads go through the read-only path so that
// the stencil neighbours of a tile are served from L1 / L2.  Templated on the
// field precision T (float or double); every sum that leaves a kernel is FP64.
#include "les_gridsync.cuh"
#include "les_internal.h"

namespace les {

// ---- precision-generic math -------------------------------------------------
__device__ __forceinline__ double m_pow(double a, double b) { return pow(a, b); }
__device__ __forceinline__ float m_pow(float a, float b) { return powf(a, b); }
__device__ __forceinline__ double m_exp(double a) { return exp(a); }
__device__ __forceinline__ float m_exp(float a) { return expf(a); }
__device__ __forceinline__ double m_sqrt(double a) { return sqrt(a); }
__device__ __forceinline__ float m_sqrt(float a) { return sqrtf(a); }
__device__ __forceinline__ double m_sin(double a) { return sin(a); }
__device__ __forceinline__ float m_sin(float a) { return sinf(a); }

__device__ __forceinline__ int vghost(int c) { return c == 2 ? G_ODD : G_UV; }

// ---- Sec. 2.1-2.2: moist thermodynamics at one level -------------------------
template <typename T>
struct Thermo {
  T p0, p00;
  __device__ __forceinline__ T rm(T qt, T ql) const { return (T(1) - qt) * T(kRd) + (qt - ql) * T(kRv); }
  __device__ __forceinline__ T cpm(T qt, T ql) const {
    return (T(1) - qt) * T(kCpd) + (qt - ql) * T(kCpv) + ql * T(kCl);
  }
  // Exner function (p0 / p00)^(R_m / c_pm)
  __device__ __forceinline__ T exner(T qt, T ql) const { return m_pow(p0 / p00, rm(qt, ql) / cpm(qt, ql)); }
  // saturation specific humidity (Clausius-Clapeyron, constant L_v0)
  __device__ __forceinline__ T qvs(T temp) const {
    T es = T(kEtr) * m_exp(T(kLv0 / kRv) * (T(1.0 / kTtr) - T(1) / temp));
    const T eps = T(kRd / kRv);
    return eps * es / (p0 - (T(1) - eps) * es);
  }
  // theta_l(T, q_l*(T)) with q_l* = max(0, q_t - q_v*)
  __device__ __forceinline__ T theta_l_sat(T temp, T qt) const {
    T ql = qt - qvs(temp);
    ql = ql > T(0) ? ql : T(0);
    return temp / exner(qt, ql) * (T(1) - T(kLv0) * ql / (cpm(qt, ql) * temp));
  }
  // secant solve of theta_l*(T) = theta_l, liquid only (Sec. 2.2)
  __device__ void adjust(T th, T qt, T tol, int maxit, T& temp, T& ql) const {
    T T1 = exner(qt, T(0)) * th;
    T qs1 = qvs(T1);
    if (qt <= qs1) {
      temp = T1;
      ql = T(0);
      return;
    }
    T Ta = T1, Tb = T1 + T(kLv0) * (qt - qs1) / cpm(qt, T(0));
    T fa = theta_l_sat(Ta, qt) - th;
    T fb = theta_l_sat(Tb, qt) - th;
    for (int it = 0; it < maxit; ++it) {
      if (fabs(fb) < tol || fb == fa) break;
      T Tc = Tb - fb * (Tb - Ta) / (fb - fa);
      Ta = Tb;
      fa = fb;
      Tb = Tc;
      fb = theta_l_sat(Tb, qt) - th;
    }
    temp = Tb;
    ql = qt - qvs(Tb);
    ql = ql > T(0) ? ql : T(0);
  }
};

// a1: T, q_l and buoyancy b = g (alpha - alpha0) / alpha0, alpha = R_m T / p0
template <typename T>
__global__ void __launch_bounds__(NTHREADS) k_thermo_cells(Grid<T> g, Phys<T> ph, const T* __restrict__ th,
                                                           const T* __restrict__ qt, T* __restrict__ temp,
                                                           T* __restrict__ ql, T* __restrict__ b,
                                                           T* __restrict__ srad) {
  for (long long t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
    int i, j, k0, k1;
    tile_origin(g, t, i, j, k0, k1);
    if (i >= g.nx || j >= g.ny) continue;
    for (int k = k0; k < k1; ++k) {
      const size_t m = g.lin(i, j, k);
      Thermo<T> td{ph.p0[k], ph.p00};
      const T thc = th[m], qtc = qt[m];
      T tc, qlc;
      if (ph.flags & LES_PHYS_MOIST) {
        td.adjust(thc, qtc, ph.sat_tol, ph.sat_maxit, tc, qlc);
      } else {
        qlc = T(0);
        tc = td.exner(qtc, T(0)) * thc;
      }
      temp[m] = tc;
      ql[m] = qlc;
      if (ph.flags & LES_PHYS_BUOY) {
        const T a0 = ph.alpha0[k];
        const T alpha = td.rm(qtc, qlc) * tc / td.p0;
        b[m] = T(kGrav) * (alpha - a0) / a0;
      } else {
        b[m] = T(0);
      }
      srad[m] = T(0);
    }
  }
}

// a1 (radiation): per column, longwave flux through the faces
//   F(k+1/2) = F0 exp(-kappa LWP above) + F1 exp(-kappa LWP below),
// and the source -(1 / (c_pm Pi)) dF/dz of rho0 theta_l.  A block holds 32
// columns (threadIdx.x) x RZ segments of each column (threadIdx.y): every
// thread sums rho0 q_l dz over its segment, a shared-memory scan over the
// segments gives each one the liquid water below it and the column total,
// and the thread then forms the face fluxes of its own levels.
constexpr int RZ = 8;
template <typename T>
__global__ void __launch_bounds__(32 * RZ) k_radiation(Grid<T> g, Phys<T> ph, const T* __restrict__ qt,
                                                      const T* __restrict__ ql, T* __restrict__ srad) {
  __shared__ T seg[RZ][32];
  const int i = blockIdx.x * 32 + threadIdx.x;
  const int j = blockIdx.y;
  const int zs = threadIdx.y;
  const bool col = i < g.nx;
  const int per = (g.nz + RZ - 1) / RZ;
  const int ka = min(zs * per, g.nz), kb = min(ka + per, g.nz);
  const T dz = g.dz;
  T part = T(0);
  if (col)
    for (int k = ka; k < kb; ++k) part += ph.rho0[k] * ql[g.lin(i, j, k)] * dz;
  seg[zs][threadIdx.x] = part;
  __syncthreads();
  if (!col) return;
  T below = T(0), total = T(0);
  for (int q = 0; q < RZ; ++q) {
    const T v = seg[q][threadIdx.x];
    if (q < zs) below += v;
    total += v;
  }
  // flux through the face below this segment's first level
  T Fm = ph.rad_f0 * m_exp(-ph.rad_kappa * (total - below)) + ph.rad_f1 * m_exp(-ph.rad_kappa * below);
  for (int k = ka; k < kb; ++k) {
    const size_t m = g.lin(i, j, k);
    const T qlc = ql[m], qtc = qt[m];
    below += ph.rho0[k] * qlc * dz;
    const T above = total - below;
    const T Fp = ph.rad_f0 * m_exp(-ph.rad_kappa * above) + ph.rad_f1 * m_exp(-ph.rad_kappa * below);
    Thermo<T> td{ph.p0[k], ph.p00};
    srad[m] = -(Fp - Fm) / dz / (td.cpm(qtc, qlc) * td.exner(qtc, qlc));
    Fm = Fp;
  }
}

// ---- Sec. 2.3: Smagorinsky-Lilly viscosity at a node ----------------------------
// nu_t = (c_s Delta)^2 f_B S, S = sqrt(2 S_ij S_ij) from nodal central
// differences, f_B = sqrt(clip(1 - N^2 / (Pr S^2), 0, 1)), N^2 = db/dz.
template <typename T, bool HALF>
struct VelView {
  const T* u[3];
  const T* un[3];
  __device__ __forceinline__ T operator()(const Grid<T>& g, int c, int i, int j, int k) const {
    T a = g.at(u[c], i, j, k, vghost(c));
    if (HALF) a = T(0.5) * (a + g.at(un[c], i, j, k, vghost(c)));
    return a;
  }
};

template <typename T, bool HALF>
__device__ __forceinline__ T nu_node(const Grid<T>& g, const Phys<T>& ph, const VelView<T, HALF>& V,
                                     const T* __restrict__ b, int i, int j, int k) {
  if (ph.flags & LES_PHYS_CONST_NU) return ph.nu_const;
  if (!(ph.flags & LES_PHYS_SGS)) return T(0);
  T gr[3][3];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int di = d == 0, dj = d == 1, dk = d == 2;
      gr[c][d] = (V(g, c, i + di, j + dj, k + dk) - V(g, c, i - di, j - dj, k - dk)) * (T(0.5) * g.ih(d));
    }
  T S2 = T(0);
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const T s = T(0.5) * (gr[c][d] + gr[d][c]);
      S2 += T(2) * s * s;
    }
  T fB = T(1);
  if ((ph.flags & LES_PHYS_FB) && S2 > T(0)) {
    const T N2 = (g.at(b, i, j, k + 1, G_EVEN) - g.at(b, i, j, k - 1, G_EVEN)) * (T(0.5) * g.idz);
    T x = T(1) - N2 / (T(1) / ph.inv_pr * S2);
    x = x < T(0) ? T(0) : (x > T(1) ? T(1) : x);
    fB = m_sqrt(x);
  }
  return ph.cs2d2 * fB * m_sqrt(S2);
}

template <typename T, bool HALF>
__global__ void __launch_bounds__(NTHREADS) k_nu(Grid<T> g, Phys<T> ph, VelView<T, HALF> V,
                                                 const T* __restrict__ b, T* __restrict__ uh,
                                                 T* __restrict__ vh, T* __restrict__ wh,
                                                 T* __restrict__ nu) {
  for (long long t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
    int i, j, k0, k1;
    tile_origin(g, t, i, j, k0, k1);
    if (i >= g.nx || j >= g.ny) continue;
    for (int k = k0; k < k1; ++k) {
      const size_t m = g.lin(i, j, k);
      if (HALF) {
        uh[m] = V(g, 0, i, j, k);
        vh[m] = V(g, 1, i, j, k);
        wh[m] = V(g, 2, i, j, k);
      }
      nu[m] = nu_node<T, HALF>(g, ph, V, b, i, j, k);
    }
  }
}

// QUICK face value between node n and n + e_d (Sec. 2.4): for F >= 0
// (-f[n-1] + 6 f[n] + 3 f[n+1]) / 8, otherwise (3 f[n] + 6 f[n+1] - f[n+2]) / 8

// ---- a3: scalar predictor (Eq. scalar_prediction_step) -----------------------
// rho0 phi^{k+1} = rho0 phi^{n+1/2} + dt [ -div(rho0 u^k phibar)
//   + div(rho0 nu_t / Pr grad phibar) + S ],  phibar = (phi^k + phi^{n+1/2}) / 2
template <typename T>
__global__ void __launch_bounds__(NTHREADS)
    k_scalar(Grid<T> g, Phys<T> ph, const T* __restrict__ u, const T* __restrict__ v,
             const T* __restrict__ w, const T* __restrict__ nu, const T* __restrict__ thk,
             const T* __restrict__ qtk, const T* __restrict__ thh, const T* __restrict__ qth,
             const T* __restrict__ srad, T* __restrict__ tho, T* __restrict__ qto) {
  const T* vel[3] = {u, v, w};
  const T* phk[2] = {thk, qtk};
  const T* phh[2] = {thh, qth};
  const T inv_s[2] = {ph.inv_pr, ph.inv_sc};
  const T sflux[2] = {ph.sflux_th, ph.sflux_qt};
  for (long long t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
    int i, j, k0, k1;
    tile_origin(g, t, i, j, k0, k1);
    if (i >= g.nx || j >= g.ny) continue;
    for (int k = k0; k < k1; ++k) {
      auto bar = [&](int q, int ii, int jj, int kk) -> T {
        return T(0.5) * (g.at(phk[q], ii, jj, kk, G_EVEN) + g.at(phh[q], ii, jj, kk, G_EVEN));
      };
      T tend[2] = {T(0), T(0)};
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const int di = d == 0, dj = d == 1, dk = d == 2;
        const T ihd = g.ih(d);
#pragma unroll
        for (int side = 0; side < 2; ++side) {
          const int li = i - (side ? 0 : di), lj = j - (side ? 0 : dj), lk = k - (side ? 0 : dk);
          const int ui = li + di, uj = lj + dj, uk = lk + dk;
          T fl[2];
          if (g.wall_face(d, lk)) {
            const bool sfc = g.surface_face(d, lk) && (ph.flags & LES_PHYS_SFC);
            fl[0] = sfc ? -sflux[0] : T(0);
            fl[1] = sfc ? -sflux[1] : T(0);
          } else {
            T F = T(0);
            if (ph.flags & LES_PHYS_ADV) {
              F = T(0.5) * (g.prof(ph.rho0, lk) * g.at(vel[d], li, lj, lk, vghost(d)) +
                            g.prof(ph.rho0, uk) * g.at(vel[d], ui, uj, uk, vghost(d)));
            }
            const T nuf = T(0.5) * (g.at(nu, li, lj, lk, G_EVEN) + g.at(nu, ui, uj, uk, G_EVEN));
            const T rhof = T(0.5) * (g.prof(ph.rho0, lk) + g.prof(ph.rho0, uk));
#pragma unroll
            for (int q = 0; q < 2; ++q) {
              const T b0 = bar(q, li, lj, lk), b1 = bar(q, ui, uj, uk);
              T adv = T(0);
              if (ph.flags & LES_PHYS_ADV) {
                const T bm = bar(q, li - di, lj - dj, lk - dk);
                const T b2 = bar(q, ui + di, uj + dj, uk + dk);
                adv = F * face_value(ph.advection, F, bm, b0, b1, b2);
              }
              fl[q] = -adv + rhof * nuf * inv_s[q] * (b1 - b0) * ihd;
            }
          }
#pragma unroll
          for (int q = 0; q < 2; ++q) tend[q] += (side ? fl[q] : -fl[q]) * ihd;
        }
      }
      const size_t m = g.lin(i, j, k);
      const T r0 = ph.rho0[k];
      if (ph.flags & LES_PHYS_SUBS) {
        // sinking at D z: d phi / dz taken upwind, from the level above
        const T wsub = ph.subs_div * (T(k) + T(0.5)) * g.dz;
#pragma unroll
        for (int q = 0; q < 2; ++q) tend[q] += r0 * wsub * (bar(q, i, j, k + 1) - bar(q, i, j, k)) * g.idz;
      }
      if (ph.flags & LES_PHYS_RAD) tend[0] += srad[m];
      tho[m] = (r0 * thh[m] + ph.dt * tend[0]) / r0;
      qto[m] = (r0 * qth[m] + ph.dt * tend[1]) / r0;
    }
  }
}

// ---- a4: momentum predictor (Eq. momentum_prediction_step) ---------------------
// rho0 u^ = rho0 u^n + dt [ -rho0 G(alpha0 p^k) + R ],  R at u^{n+1/2}:
// -div(rho0 u (x) u) (QUICK) + div(rho0 nu_t (grad u + grad u^T)) + rho0 b k
// - f k x rho0 (u - u_g) - sponge.
template <typename T>
__global__ void __launch_bounds__(NTHREADS)
    k_momentum(Grid<T> g, Phys<T> ph, const T* __restrict__ uh, const T* __restrict__ vh,
               const T* __restrict__ wh, const T* __restrict__ un, const T* __restrict__ vn,
               const T* __restrict__ wn, const T* __restrict__ nu, const T* __restrict__ p,
               const T* __restrict__ b, T* __restrict__ ou, T* __restrict__ ov, T* __restrict__ ow) {
  const T* vel[3] = {uh, vh, wh};
  const T* veln[3] = {un, vn, wn};
  T* out[3] = {ou, ov, ow};
  const T target[3] = {ph.ug, ph.vg, T(0)};
  for (long long t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
    int i, j, k0, k1;
    tile_origin(g, t, i, j, k0, k1);
    if (i >= g.nx || j >= g.ny) continue;
    for (int k = k0; k < k1; ++k) {
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
          const T ihd = g.ih(d);
#pragma unroll
          for (int side = 0; side < 2; ++side) {
            const int li = i - (side ? 0 : di), lj = j - (side ? 0 : dj), lk = k - (side ? 0 : dk);
            const int ui = li + di, uj = lj + dj, uk = lk + dk;
            if (g.surface_face(d, lk)) continue;  // free slip, no momentum flux
            T adv = T(0);
            if ((ph.flags & LES_PHYS_ADV) && !g.wall_face(d, lk)) {
              const T F = T(0.5) * (g.prof(ph.rho0, lk) * g.at(vel[d], li, lj, lk, vghost(d)) +
                                    g.prof(ph.rho0, uk) * g.at(vel[d], ui, uj, uk, vghost(d)));
              adv = F * face_value(ph.advection, F, g.at(vel[c], li - di, lj - dj, lk - dk, vghost(c)),
                              g.at(vel[c], li, lj, lk, vghost(c)), g.at(vel[c], ui, uj, uk, vghost(c)),
                              g.at(vel[c], ui + di, uj + dj, uk + dk, vghost(c)));
            }
            // SGS stress on the face: compact normal derivative, tangential
            // derivative = mean of the two nodal central differences
            const T dn = (g.at(vel[c], ui, uj, uk, vghost(c)) - g.at(vel[c], li, lj, lk, vghost(c))) * ihd;
            T dtg;
            if (c == d) {
              dtg = dn;
            } else {
              const T g0 = g.at(vel[d], li + ci, lj + cj, lk + ck, vghost(d)) -
                           g.at(vel[d], li - ci, lj - cj, lk - ck, vghost(d));
              const T g1 = g.at(vel[d], ui + ci, uj + cj, uk + ck, vghost(d)) -
                           g.at(vel[d], ui - ci, uj - cj, uk - ck, vghost(d));
              dtg = T(0.25) * (g0 + g1) * g.ih(c);
            }
            const T nuf = T(0.5) * (g.at(nu, li, lj, lk, G_EVEN) + g.at(nu, ui, uj, uk, G_EVEN));
            const T rhof = T(0.5) * (g.prof(ph.rho0, lk) + g.prof(ph.rho0, uk));
            const T fl = -adv + rhof * nuf * (dn + dtg);
            R += (side ? fl : -fl) * ihd;
          }
        }
        const T uc = g.at(vel[c], i, j, k, vghost(c));
        if ((ph.flags & LES_PHYS_BUOY) && c == 2) R += r0 * b[m];
        if (ph.flags & LES_PHYS_CORIOLIS) {
          if (c == 0) R += ph.f_cor * r0 * (vh[m] - ph.vg);
          if (c == 1) R -= ph.f_cor * r0 * (uh[m] - ph.ug);
        }
        if ((ph.flags & LES_PHYS_SPONGE) && zc > ph.sponge_zs) {
          const T x = m_sin(T(1.5707963267948966) * (zc - ph.sponge_zs) / (ph.sponge_h - ph.sponge_zs));
          R -= ph.sponge_rate * x * x * r0 * (uc - target[c]);
        }
        const T gp = (g.prof(ph.alpha0, k + ck) * g.at(p, i + ci, j + cj, k + ck, G_EVEN) -
                      g.prof(ph.alpha0, k - ck) * g.at(p, i - ci, j - cj, k - ck, G_EVEN)) *
                     (T(0.5) * g.ih(c));
        out[c][m] = (r0 * veln[c][m] + ph.dt * (-r0 * gp + R)) / r0;
      }
    }
  }
}

// ---- Poisson right side (Eq. pressure_correction with Appendix A) -------------
// compact: rhs = alpha0 / dt D(rho0 u^) - C(psi^k),
//   C = sum_l [psi_{l+2} - 4 psi_{l+1} + 6 psi_l - 4 psi_{l-1} + psi_{l-2}] / (4 Delta_l^2)
// wide:    rhs = D(rho0 u^) / dt
template <typename T>
__global__ void __launch_bounds__(NTHREADS)
    k_rhs(Grid<T> g, Phys<T> ph, int op, const T* __restrict__ ou, const T* __restrict__ ov,
          const T* __restrict__ ow, const T* __restrict__ psi, T* __restrict__ rhs) {
  const T* hat[3] = {ou, ov, ow};
  for (long long t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
    int i, j, k0, k1;
    tile_origin(g, t, i, j, k0, k1);
    if (i >= g.nx || j >= g.ny) continue;
    for (int k = k0; k < k1; ++k) {
      T div = T(0);
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const int di = d == 0, dj = d == 1, dk = d == 2;
        div += (g.prof(ph.rho0, k + dk) * g.at(hat[d], i + di, j + dj, k + dk, vghost(d)) -
                g.prof(ph.rho0, k - dk) * g.at(hat[d], i - di, j - dj, k - dk, vghost(d))) *
               (T(0.5) * g.ih(d));
      }
      T val;
      if (op == LES_OP_COMPACT) {
        T C = T(0);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const int di = d == 0, dj = d == 1, dk = d == 2;
          const T ih = g.ih(d);
          C += (g.at(psi, i + 2 * di, j + 2 * dj, k + 2 * dk, G_EVEN) -
                T(4) * g.at(psi, i + di, j + dj, k + dk, G_EVEN) + T(6) * g.at(psi, i, j, k, G_EVEN) -
                T(4) * g.at(psi, i - di, j - dj, k - dk, G_EVEN) +
                g.at(psi, i - 2 * di, j - 2 * dj, k - 2 * dk, G_EVEN)) *
               (T(0.25) * ih * ih);
        }
        val = ph.alpha0[k] / ph.dt * div - C;
      } else {
        val = div / ph.dt;
      }
      rhs[g.lin(i, j, k)] = val;
    }
  }
}

// ---- a7: correction (Sec. 2.4) ----------------------------------------------
// u^{k+1} = u^ - dt G(psi), p^{k+1} = p^k + rho0 psi, psi = alpha0 dp
template <typename T>
__global__ void __launch_bounds__(NTHREADS)
    k_correct(Grid<T> g, Phys<T> ph, const T* __restrict__ ou, const T* __restrict__ ov,
              const T* __restrict__ ow, const T* __restrict__ psi, T* __restrict__ u,
              T* __restrict__ v, T* __restrict__ w, T* __restrict__ p) {
  const T* hat[3] = {ou, ov, ow};
  T* vel[3] = {u, v, w};
  for (long long t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
    int i, j, k0, k1;
    tile_origin(g, t, i, j, k0, k1);
    if (i >= g.nx || j >= g.ny) continue;
    for (int k = k0; k < k1; ++k) {
      const size_t m = g.lin(i, j, k);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int ci = c == 0, cj = c == 1, ck = c == 2;
        const T gr = (g.at(psi, i + ci, j + cj, k + ck, G_EVEN) - g.at(psi, i - ci, j - cj, k - ck, G_EVEN)) *
                     (T(0.5) * g.ih(c));
        vel[c][m] = hat[c][m] - ph.dt * gr;
      }
      p[m] += ph.rho0[k] * psi[m];
    }
  }
}

// ---- a8: diagnostics with FP64 totals -------------------------------------------
// sum rho0 theta_l dV, sum rho0 q_t dV, sum rho0 u_c dV (3), kinetic energy,
// max Courant number, max |D(rho0 u)|, non-finite values, sum rho0 q_l dV.
// FP64 fields accumulate in FP64.  FP32 fields form each thread's sums in
// FP32 over runs of 16 nodes, folded into compensated FP32 pairs (FP64 on
// this GPU costs tens of FP32 operations per node), with dV applied to the
// FP64 totals; maxima and the count in FP32.
template <typename T>
__global__ void __launch_bounds__(NTHREADS)
    k_diag(Grid<T> g, Phys<T> ph, const T* __restrict__ u, const T* __restrict__ v,
           const T* __restrict__ w, const T* __restrict__ p, const T* __restrict__ th,
           const T* __restrict__ qt, const T* __restrict__ ql, double* partials, SolverCtl* ctl,
           double* out) {
  const T* vel[3] = {u, v, w};
  double acc[LES_NDIAG];
#pragma unroll
  for (int q = 0; q < LES_NDIAG; ++q) acc[q] = 0.0;
  const double dV = (double)g.dx * (double)g.dy * (double)g.dz;
  if constexpr (sizeof(T) == 4) {
    constexpr int NS = 7;  // the sums: 0 theta, 1 q_t, 2-4 u, 5 2 x kinetic energy, 6 q_l
    F2 sum[NS];
    float run[NS];
#pragma unroll
    for (int q = 0; q < NS; ++q) {
      sum[q] = F2{0.f, 0.f};
      run[q] = 0.f;
    }
    float cmax = 0.f, dmax = 0.f, bad = 0.f;
    int cnt = 0;
    for (long long t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
      int i, j, k0, k1;
      tile_origin(g, t, i, j, k0, k1);
      if (i >= g.nx || j >= g.ny) continue;
      for (int k = k0; k < k1; ++k) {
        const size_t m = g.lin(i, j, k);
        const float r0 = ph.rho0[k];
        const float uc[3] = {u[m], v[m], w[m]};
        run[0] += r0 * th[m];
        run[1] += r0 * qt[m];
        float ke = 0.f, cfl = 0.f, div = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const int ci = c == 0, cj = c == 1, ck = c == 2;
          run[2 + c] += r0 * uc[c];
          ke += uc[c] * uc[c];
          cfl += fabsf(uc[c]) * g.ih(c);
          div += (g.prof(ph.rho0, k + ck) * g.at(vel[c], i + ci, j + cj, k + ck, vghost(c)) -
                  g.prof(ph.rho0, k - ck) * g.at(vel[c], i - ci, j - cj, k - ck, vghost(c))) *
                 (0.5f * g.ih(c));
        }
        run[5] += r0 * ke;
        run[6] += r0 * ql[m];
        cmax = fmaxf(cmax, cfl * ph.dt);
        dmax = fmaxf(dmax, fabsf(div));
        const float vals[6] = {uc[0], uc[1], uc[2], p[m], th[m], qt[m]};
#pragma unroll
        for (int q = 0; q < 6; ++q)
          if (!isfinite(vals[q])) bad += 1.f;
        if ((++cnt & 15) == 0)
#pragma unroll
          for (int q = 0; q < NS; ++q) {
            f2_acc(sum[q], run[q]);
            run[q] = 0.f;
          }
      }
    }
#pragma unroll
    for (int q = 0; q < NS; ++q) f2_acc(sum[q], run[q]);
    acc[0] = f2_value(sum[0]);
    acc[1] = f2_value(sum[1]);
    acc[2] = f2_value(sum[2]);
    acc[3] = f2_value(sum[3]);
    acc[4] = f2_value(sum[4]);
    acc[5] = 0.5 * f2_value(sum[5]);
    acc[6] = cmax;
    acc[7] = dmax;
    acc[8] = bad;
    acc[9] = f2_value(sum[6]);
  } else {
    for (long long t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
      int i, j, k0, k1;
      tile_origin(g, t, i, j, k0, k1);
      if (i >= g.nx || j >= g.ny) continue;
      for (int k = k0; k < k1; ++k) {
        const size_t m = g.lin(i, j, k);
        const double r0 = (double)ph.rho0[k];
        acc[0] += r0 * (double)th[m];
        acc[1] += r0 * (double)qt[m];
        double ke = 0.0, cfl = 0.0, div = 0.0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const int ci = c == 0, cj = c == 1, ck = c == 2;
          const double uc = (double)vel[c][m];
          acc[2 + c] += r0 * uc;
          ke += uc * uc;
          cfl += fabs(uc) * (double)g.ih(c);
          div += ((double)g.prof(ph.rho0, k + ck) * (double)g.at(vel[c], i + ci, j + cj, k + ck, vghost(c)) -
                  (double)g.prof(ph.rho0, k - ck) * (double)g.at(vel[c], i - ci, j - cj, k - ck, vghost(c))) *
                 (0.5 * (double)g.ih(c));
        }
        acc[5] += 0.5 * r0 * ke;
        acc[6] = fmax(acc[6], cfl * (double)ph.dt);
        acc[7] = fmax(acc[7], fabs(div));
        const double vals[6] = {(double)u[m], (double)v[m], (double)w[m], (double)p[m], (double)th[m], (double)qt[m]};
#pragma unroll
        for (int q = 0; q < 6; ++q)
          if (!isfinite(vals[q])) acc[8] += 1.0;
        acc[9] += r0 * (double)ql[m];
      }
    }
  }
  // the cell volume, applied once per thread
#pragma unroll
  for (int q : {0, 1, 2, 3, 4, 5, 9}) acc[q] *= dV;
  double res[LES_NDIAG];
  if (grid_reduce<LES_NDIAG>(acc, (1u << 6) | (1u << 7), partials, &ctl->tickets[TK_DIAG], res)) {
#pragma unroll
    for (int q = 0; q < LES_NDIAG; ++q) out[q] = res[q];
  }
}

// max over cells of |u|/dx + |v|/dy + |w|/dz (Courant-number step)
template <typename T>
__global__ void __launch_bounds__(NTHREADS)
    k_cfl(Grid<T> g, const T* __restrict__ u, const T* __restrict__ v, const T* __restrict__ w,
          double* partials, SolverCtl* ctl) {
  double acc[1] = {0.0};
  for (long long t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
    int i, j, k0, k1;
    tile_origin(g, t, i, j, k0, k1);
    if (i >= g.nx || j >= g.ny) continue;
    for (int k = k0; k < k1; ++k) {
      const size_t m = g.lin(i, j, k);
      const double c = fabs((double)u[m]) / (double)g.dx + fabs((double)v[m]) / (double)g.dy +
                       fabs((double)w[m]) / (double)g.dz;
      acc[0] = fmax(acc[0], c);
    }
  }
  double res[1];
  if (grid_reduce<1>(acc, 1u, partials, &ctl->tickets[TK_MAX], res)) ctl->scal = res[0];
}

// ---- host launchers -------------------------------------------------------------
template <typename T>
cudaError_t launch_thermo(const StageArgs<T>& a, const T* th, const T* qt, T* temp, T* ql, T* b, T* srad) {
  {
    ProfScope ps(a.prof, KI_THERMO, a.st);
    k_thermo_cells<T><<<a.lc.grid, a.lc.block, 0, a.st>>>(a.g, a.ph, th, qt, temp, ql, b, srad);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !(a.ph.flags & LES_PHYS_RAD)) return e;
  dim3 grid((a.g.nx + 31) / 32, a.g.ny);
  {
    ProfScope ps(a.prof, KI_RADIATION, a.st);
    k_radiation<T><<<grid, dim3(32, RZ), 0, a.st>>>(a.g, a.ph, qt, ql, srad);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_nu(const StageArgs<T>& a, const T* u, const T* v, const T* w, const T* un, const T* vn,
                      const T* wn, const T* b, T* uh, T* vh, T* wh, T* nu) {
  if (un) {
    VelView<T, true> V{{u, v, w}, {un, vn, wn}};
    ProfScope ps(a.prof, KI_NU_HALF, a.st);
    k_nu<T, true><<<a.lc.grid, a.lc.block, 0, a.st>>>(a.g, a.ph, V, b, uh, vh, wh, nu);
  } else {
    VelView<T, false> V{{u, v, w}, {u, v, w}};
    ProfScope ps(a.prof, KI_NU, a.st);
    k_nu<T, false><<<a.lc.grid, a.lc.block, 0, a.st>>>(a.g, a.ph, V, b, nullptr, nullptr, nullptr, nu);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_scalar(const StageArgs<T>& a, const T* u, const T* v, const T* w, const T* nu,
                          const T* thk, const T* qtk, const T* thh, const T* qth, const T* srad, T* th_out,
                          T* qt_out) {
  ProfScope ps(a.prof, KI_SCALAR, a.st);
  k_scalar<T><<<a.lc.grid, a.lc.block, 0, a.st>>>(a.g, a.ph, u, v, w, nu, thk, qtk, thh, qth, srad, th_out,
                                                   qt_out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_momentum(const StageArgs<T>& a, const T* uh, const T* vh, const T* wh, const T* un,
                            const T* vn, const T* wn, const T* nu, const T* p, const T* b, T* ou, T* ov, T* ow) {
  ProfScope ps(a.prof, KI_MOMENTUM, a.st);
  k_momentum<T><<<a.lc.grid, a.lc.block, 0, a.st>>>(a.g, a.ph, uh, vh, wh, un, vn, wn, nu, p, b, ou, ov, ow);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_rhs(const StageArgs<T>& a, int op, const T* ou, const T* ov, const T* ow, const T* psi,
                       T* rhs) {
  ProfScope ps(a.prof, KI_RHS, a.st);
  k_rhs<T><<<a.lc.grid, a.lc.block, 0, a.st>>>(a.g, a.ph, op, ou, ov, ow, psi, rhs);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_correct(const StageArgs<T>& a, const T* ou, const T* ov, const T* ow, const T* psi, T* u,
                           T* v, T* w, T* p) {
  ProfScope ps(a.prof, KI_CORRECT, a.st);
  k_correct<T><<<a.lc.grid, a.lc.block, 0, a.st>>>(a.g, a.ph, ou, ov, ow, psi, u, v, w, p);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_diag(const StageArgs<T>& a, const T* u, const T* v, const T* w, const T* p, const T* th,
                        const T* qt, const T* ql, double* partials, SolverCtl* ctl, double* out_dev) {
  ProfScope ps(a.prof, KI_DIAG, a.st);
  k_diag<T><<<a.lc.grid, a.lc.block, 0, a.st>>>(a.g, a.ph, u, v, w, p, th, qt, ql, partials, ctl, out_dev);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cfl_max(const StageArgs<T>& a, const T* u, const T* v, const T* w, double* partials,
                           SolverCtl* ctl) {
  ProfScope ps(a.prof, KI_CFL, a.st);
  k_cfl<T><<<a.lc.grid, a.lc.block, 0, a.st>>>(a.g, u, v, w, partials, ctl);
  return cudaGetLastError();
}

#define LES_INSTANTIATE(T)                                                                                  \
  template cudaError_t launch_thermo<T>(const StageArgs<T>&, const T*, const T*, T*, T*, T*, T*);          \
  template cudaError_t launch_nu<T>(const StageArgs<T>&, const T*, const T*, const T*, const T*, const T*, \
                                    const T*, const T*, T*, T*, T*, T*);                                   \
  template cudaError_t launch_scalar<T>(const StageArgs<T>&, const T*, const T*, const T*, const T*,       \
                                        const T*, const T*, const T*, const T*, const T*, T*, T*);         \
  template cudaError_t launch_momentum<T>(const StageArgs<T>&, const T*, const T*, const T*, const T*,     \
                                          const T*, const T*, const T*, const T*, const T*, T*, T*, T*);   \
  template cudaError_t launch_rhs<T>(const StageArgs<T>&, int, const T*, const T*, const T*, const T*, T*); \
  template cudaError_t launch_correct<T>(const StageArgs<T>&, const T*, const T*, const T*, const T*, T*, \
                                         T*, T*, T*);                                                      \
  template cudaError_t launch_diag<T>(const StageArgs<T>&, const T*, const T*, const T*, const T*,         \
                                      const T*, const T*, const T*, double*, SolverCtl*, double*);         \
  template cudaError_t launch_cfl_max<T>(const StageArgs<T>&, const T*, const T*, const T*, double*,       \
                                         SolverCtl*);

LES_INSTANTIATE(float)
LES_INSTANTIATE(double)

}  // namespace les
