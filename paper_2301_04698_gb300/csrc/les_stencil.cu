// les_stencil.cu -- the pointwise and column stages of one LES time step on
// sm_103a: thermodynamics and buoyancy (Sec. 2.1-2.2), the longwave radiation
// source, the correction of Sec. 2.4 on grids the column kernel does not
// take, and the FP64 diagnostics.
//
// The tile kernels walk 32x8-thread tiles grid-stride and march each thread
// through a run of z-planes; the thermodynamics streams 16-byte chunks where
// the rows allow.  Templated on the field precision T (float or double);
// every sum that leaves a kernel is FP64.
#include <type_traits>

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

// a1 at one node of level k: T, q_l and buoyancy b = g (alpha - alpha0) /
// alpha0, alpha = R_m T / p0
template <typename T>
__device__ __forceinline__ void thermo_node(const Phys<T>& ph, int k, T thc, T qtc, T& tc, T& qlc, T& bc) {
  Thermo<T> td{ph.p0[k], ph.p00};
  if (ph.flags & LES_PHYS_MOIST) {
    td.adjust(thc, qtc, ph.sat_tol, ph.sat_maxit, tc, qlc);
  } else {
    qlc = T(0);
    tc = td.exner(qtc, T(0)) * thc;
  }
  if (ph.flags & LES_PHYS_BUOY) {
    const T a0 = ph.alpha0[k];
    const T alpha = td.rm(qtc, qlc) * tc / td.p0;
    bc = T(kGrav) * (alpha - a0) / a0;
  } else {
    bc = T(0);
  }
}

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
      T tc, qlc, bc;
      thermo_node(ph, k, th[m], qt[m], tc, qlc, bc);
      temp[m] = tc;
      ql[m] = qlc;
      b[m] = bc;
      srad[m] = T(0);
    }
  }
}

// The same as a stream of 16-byte chunks (V nodes of one row; nx a multiple
// of V): each thread loads its chunks of theta_l and q_t with 16-byte loads,
// many in flight across the grid, and writes the four outputs likewise.
template <typename T>
__global__ void __launch_bounds__(256) k_thermo_vec(Grid<T> g, Phys<T> ph, const T* __restrict__ th,
                                                    const T* __restrict__ qt, T* __restrict__ temp,
                                                    T* __restrict__ ql, T* __restrict__ b, T* __restrict__ srad) {
  constexpr int V = 16 / (int)sizeof(T);
  using V16 = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  const long long pc = (long long)g.nx * g.ny / V;  // chunks per plane
  const long long nc = pc * g.nz;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < nc; c += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(c / pc);
    const V16 tv = __ldcs(reinterpret_cast<const V16*>(th) + c), qv = __ldcs(reinterpret_cast<const V16*>(qt) + c);
    const T* tp = reinterpret_cast<const T*>(&tv);
    const T* qp = reinterpret_cast<const T*>(&qv);
    V16 to, lo, bo, zo;
    T* top = reinterpret_cast<T*>(&to);
    T* lop = reinterpret_cast<T*>(&lo);
    T* bop = reinterpret_cast<T*>(&bo);
    T* zop = reinterpret_cast<T*>(&zo);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      thermo_node(ph, k, tp[v], qp[v], top[v], lop[v], bop[v]);
      zop[v] = T(0);
    }
    __stcs(reinterpret_cast<V16*>(temp) + c, to);
    __stcs(reinterpret_cast<V16*>(ql) + c, lo);
    __stcs(reinterpret_cast<V16*>(b) + c, bo);
    __stcs(reinterpret_cast<V16*>(srad) + c, zo);
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

// a8 for FP32 fields as a stream of 16-byte chunks (four nodes of a row),
// with the per-node arithmetic of k_diag: the fields at the chunk's nodes by
// 16-byte loads, the divergence's neighbours along y as the chunks of the
// rows beside it and along z as the chunks of the planes above and below
// (their ghost rule resolved once per chunk), along x from the chunk and
// its two edge nodes.  nx a multiple of 4, every field 16-byte aligned.
__global__ void __launch_bounds__(NTHREADS)
    k_diag_vec(Grid<float> g, Phys<float> ph, const float* __restrict__ u, const float* __restrict__ v,
               const float* __restrict__ w, const float* __restrict__ p, const float* __restrict__ th,
               const float* __restrict__ qt, const float* __restrict__ ql, double* partials, SolverCtl* ctl,
               double* out) {
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
  const int cpr = g.nx / 4;
  const long long pc = (long long)cpr * g.ny, nc = pc * g.nz;
  const int nthr = blockDim.x * blockDim.y;
  const long long t0 = (long long)blockIdx.x * nthr + threadIdx.x + blockDim.x * threadIdx.y;
  auto ld4 = [](const float* q) { return __ldg(reinterpret_cast<const float4*>(q)); };
  auto el = [](const float4& a, int n) { return n == 0 ? a.x : (n == 1 ? a.y : (n == 2 ? a.z : a.w)); };
  for (long long c = t0; c < nc; c += (long long)gridDim.x * nthr) {
    const int k = (int)(c / pc);
    const int rem = (int)(c - (long long)k * pc);
    const int j = rem / cpr, i0 = (rem - j * cpr) * 4;
    const size_t m = (size_t)c * 4;
    const size_t plane = (size_t)g.nx * g.ny;
    const float4 u4 = ld4(u + m), v4 = ld4(v + m), w4 = ld4(w + m);
    const float4 p4 = ld4(p + m), t4 = ld4(th + m), q4 = ld4(qt + m), l4 = ld4(ql + m);
    const float ul = g.at(u, i0 - 1, j, k, G_UV), ur = g.at(u, i0 + 4, j, k, G_UV);
    const size_t row = (size_t)k * plane + (size_t)i0;
    const float4 vm = ld4(v + row + (size_t)g.wrap(j - 1, g.ny) * g.nx);
    const float4 vp = ld4(v + row + (size_t)g.wrap(j + 1, g.ny) * g.nx);
    // w on the planes k -+ 1 under the antisymmetric ghost rule
    int kzm = k - 1, kzp = k + 1;
    float szm = 1.f, szp = 1.f;
    if (g.walls) {
      if (kzm < 0) kzm = 0, szm = -1.f;
      if (kzp >= g.nz) kzp = g.nz - 1, szp = -1.f;
    } else {
      kzm = g.wrap(kzm, g.nz);
      kzp = g.wrap(kzp, g.nz);
    }
    const size_t col = (size_t)j * g.nx + i0;
    const float4 wm = ld4(w + (size_t)kzm * plane + col), wp = ld4(w + (size_t)kzp * plane + col);
    const float r0 = ph.rho0[k];
    const float rzm = g.prof(ph.rho0, k - 1), rzp = g.prof(ph.rho0, k + 1);
#pragma unroll
    for (int n = 0; n < 4; ++n) {
      const float uc[3] = {el(u4, n), el(v4, n), el(w4, n)};
      const float thn = el(t4, n), qtn = el(q4, n);
      run[0] += r0 * thn;
      run[1] += r0 * qtn;
      float ke = 0.f, cfl = 0.f;
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) {
        run[2 + cc] += r0 * uc[cc];
        ke += uc[cc] * uc[cc];
        cfl += fabsf(uc[cc]) * g.ih(cc);
      }
      const float xp = n == 3 ? ur : el(u4, n + 1), xm = n == 0 ? ul : el(u4, n - 1);
      float div = (r0 * xp - r0 * xm) * (0.5f * g.ih(0));
      div += (r0 * el(vp, n) - r0 * el(vm, n)) * (0.5f * g.ih(1));
      div += (rzp * (szp * el(wp, n)) - rzm * (szm * el(wm, n))) * (0.5f * g.ih(2));
      run[5] += r0 * ke;
      run[6] += r0 * el(l4, n);
      cmax = fmaxf(cmax, cfl * ph.dt);
      dmax = fmaxf(dmax, fabsf(div));
      const float vals[6] = {uc[0], uc[1], uc[2], el(p4, n), thn, qtn};
#pragma unroll
      for (int q = 0; q < 6; ++q)
        if (!isfinite(vals[q])) bad += 1.f;
    }
    if ((++cnt & 3) == 0)
#pragma unroll
      for (int q = 0; q < NS; ++q) {
        f2_acc(sum[q], run[q]);
        run[q] = 0.f;
      }
  }
#pragma unroll
  for (int q = 0; q < NS; ++q) f2_acc(sum[q], run[q]);
  double acc[LES_NDIAG];
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
  const double dV = (double)g.dx * (double)g.dy * (double)g.dz;
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
    constexpr int V = 16 / (int)sizeof(T);
    const bool vec = a.g.nx % V == 0 && ((uintptr_t)th | (uintptr_t)qt | (uintptr_t)temp | (uintptr_t)ql |
                                          (uintptr_t)b | (uintptr_t)srad) % 16 == 0;
    if (vec) {
      const long long nc = (long long)a.g.nx * a.g.ny * a.g.nz / V;
      const unsigned grid = (unsigned)std::max<long long>(1, std::min<long long>((nc + 255) / 256, 1LL << 20));
      k_thermo_vec<T><<<grid, 256, 0, a.st>>>(a.g, a.ph, th, qt, temp, ql, b, srad);
    } else {
      k_thermo_cells<T><<<a.lc.grid, a.lc.block, 0, a.st>>>(a.g, a.ph, th, qt, temp, ql, b, srad);
    }
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
  if constexpr (sizeof(T) == 4) {
    const bool vec = a.g.nx % 4 == 0 && ((uintptr_t)u | (uintptr_t)v | (uintptr_t)w | (uintptr_t)p |
                                          (uintptr_t)th | (uintptr_t)qt | (uintptr_t)ql) % 16 == 0;
    if (vec) {
      k_diag_vec<<<a.lc.grid, a.lc.block, 0, a.st>>>(a.g, a.ph, u, v, w, p, th, qt, ql, partials, ctl, out_dev);
      return cudaGetLastError();
    }
  }
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
  template cudaError_t launch_correct<T>(const StageArgs<T>&, const T*, const T*, const T*, const T*, T*, \
                                         T*, T*, T*);                                                      \
  template cudaError_t launch_diag<T>(const StageArgs<T>&, const T*, const T*, const T*, const T*,         \
                                      const T*, const T*, const T*, double*, SolverCtl*, double*);         \
  template cudaError_t launch_cfl_max<T>(const StageArgs<T>&, const T*, const T*, const T*, double*,       \
                                         SolverCtl*);

LES_INSTANTIATE(float)
LES_INSTANTIATE(double)

}  // namespace les
