/*
 * les_oracle.c -- FP64 CPU oracle of one time step of the anelastic LES of
 * Chammas et al., "Accelerating large-eddy simulations of clouds with Tensor
 * Processing Units" (arXiv 2301.04698).
 *
 * TEST INFRASTRUCTURE ONLY.  Plain loops in double precision that follow the
 * paper's statement of the discretised equations in the paper's order:
 *
 *   Sec. 2.1  reference state (Eqs. 1-4), theta_l, Exner function, R_m, c_pm,
 *             buoyancy b = g (alpha - alpha0) / alpha0, alpha = R_m T / p0
 *   Sec. 2.2  saturation adjustment theta_l*(T) - theta_l = 0 by the secant
 *             method, liquid only
 *   Sec. 2.3  nu_t = (c_s Delta)^2 f_B S, diffusivities nu_t / Pr, nu_t / Sc,
 *             sponge layer in the top of the domain
 *   Sec. 2.4  collocated finite differences, QUICK advection (or WENO3 with
 *             the local Lax-Friedrichs flux, the alternative scheme), 2nd-order
 *             central diffusion, the iterative predictor-corrector scheme
 *             (momentum prediction, pressure-correction Poisson equation,
 *             momentum / pressure correction, scalars staggered half a step)
 *   App. A    the fourth-difference correction C on the Poisson right side
 *
 * Points where the paper is silent are resolved by the readings written down
 * in the design notes of the repository; each is marked "reading:" below.
 * Nothing here is blocked, fused or reordered for speed.  Only the loops over
 * z-planes carry an OpenMP pragma; every sum is formed per plane and then
 * added plane by plane, so results do not depend on the thread count.
 */
#include "les_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ---- Table 1 constants ---------------------------------------------------- */
#define RD   287.0      /* gas constant of dry air                 */
#define RV   461.89     /* gas constant of water vapour            */
#define CPD  1004.5     /* isobaric heat capacity of dry air       */
#define CPV  1859.5     /* isobaric heat capacity of water vapour  */
#define CLQ  4181.0     /* heat capacity of liquid water           */
#define LV0  2.47e6     /* latent heat of vaporisation             */
#define GRAV 9.81       /* gravitational acceleration              */
/* reading: saturation vapour pressure by Clausius-Clapeyron with constant
 * L_v0 anchored at the triple point (the paper cites another work for q_v*). */
#define T_TRIPLE 273.16
#define E_TRIPLE 611.657

/* z-ghost rules at the surface (k < 0) and the lid (k >= nz) */
enum { GH_EVEN = 0,   /* mirror: scalars, pressure, rho0, nu_t, b          */
       GH_ODD  = 1,   /* antisymmetric: w and vertical mass flux            */
       GH_UV   = 2 }; /* horizontal velocity: free slip at the surface,
                         no slip at the lid (Sec. 4)                        */

typedef struct orc {
  orc_params p;
  int64_t n;
  double dt;
  int32_t step, sub;
  double *f[ORC_NFIELD];
  double **psi_prev;     /* K fields: solutions of the previous step        */
  double *rho0, *alpha0, *p0, *zc;
  double *tmp[8];        /* scratch fields                                  */
} orc;

static inline int64_t IDX(const orc *s, int i, int j, int k) {
  return ((int64_t)k * s->p.ny + j) * s->p.nx + i;
}
static inline int wrap(int i, int n) { i %= n; return i < 0 ? i + n : i; }

/* Value of field f at node (i,j,k) with periodic wrap in x, y and the ghost
 * rule `g` in z.  Reading: with walls, the surface and lid lie on the faces
 * k = -1/2 and k = nz - 1/2; ghost nodes mirror the interior. */
static double at(const orc *s, const double *f, int g, int i, int j, int k) {
  const int nz = s->p.nz;
  double sgn = 1.0;
  i = wrap(i, s->p.nx);
  j = wrap(j, s->p.ny);
  if (!s->p.walls) {
    k = wrap(k, nz);
  } else if (k < 0) {
    k = -1 - k;
    if (g == GH_ODD) sgn = -1.0;
  } else if (k >= nz) {
    k = 2 * nz - 1 - k;
    if (g == GH_ODD || g == GH_UV) sgn = -1.0;
  }
  return sgn * f[IDX(s, i, j, k)];
}

/* 1-D profile value at level k (mirror ghosts with walls, wrap otherwise) */
static double prof(const orc *s, const double *a, int k) {
  const int nz = s->p.nz;
  if (!s->p.walls) return a[wrap(k, nz)];
  if (k < 0) k = -1 - k;
  if (k >= nz) k = 2 * nz - 1 - k;
  return a[k];
}

static double spacing(const orc *s, int d) {
  return d == 0 ? s->p.dx : (d == 1 ? s->p.dy : s->p.dz);
}

/* ---- Sec. 2.1: reference state -------------------------------------------- */
static void reference_state(orc *s, const double *rho0_given) {
  const double th0 = s->p.theta0, p00 = s->p.p00;
  for (int k = 0; k < s->p.nz; ++k) {
    double z = (k + 0.5) * s->p.dz;
    s->zc[k] = z;
    /* p0 = p00 (1 - g z / (c_pd theta0))^(c_pd / R_d) */
    s->p0[k] = p00 * pow(1.0 - GRAV * z / (CPD * th0), CPD / RD);
    /* T0 = theta0 (p0 / p00)^(R_d / c_pd);  rho0 = p0 / (R_d T0) */
    double T0 = th0 * pow(s->p0[k] / p00, RD / CPD);
    s->rho0[k] = rho0_given ? rho0_given[k] : s->p0[k] / (RD * T0);
    s->alpha0[k] = 1.0 / s->rho0[k];
  }
}

/* ---- Sec. 2.1-2.2: moist thermodynamics ------------------------------------ */
static double gas_rm(double qt, double ql) { return (1.0 - qt) * RD + (qt - ql) * RV; }
static double heat_cpm(double qt, double ql) {
  return (1.0 - qt) * CPD + (qt - ql) * CPV + ql * CLQ;
}
static double exner(const orc *s, int k, double qt, double ql) {
  return pow(s->p0[k] / s->p.p00, gas_rm(qt, ql) / heat_cpm(qt, ql));
}
/* theta_l(T, q_l; p0) = T / Pi (1 - L_v0 q_l / (c_pm T))  (liquid only) */
static double theta_l_of(const orc *s, int k, double T, double qt, double ql) {
  return T / exner(s, k, qt, ql) * (1.0 - LV0 * ql / (heat_cpm(qt, ql) * T));
}
/* reading: e_s = e_tr exp[(L_v0/R_v)(1/T_tr - 1/T)],
 *          q_v* = (R_d/R_v) e_s / (p0 - (1 - R_d/R_v) e_s) */
static double qv_star(const orc *s, int k, double T) {
  double es = E_TRIPLE * exp(LV0 / RV * (1.0 / T_TRIPLE - 1.0 / T));
  double eps = RD / RV;
  return eps * es / (s->p0[k] - (1.0 - eps) * es);
}
/* theta_l at saturation: q_l* = max(0, q_t - q_v*(T, p0)) (Eq. e:liquid) */
static double theta_l_star(const orc *s, int k, double T, double qt) {
  double ql = fmax(0.0, qt - qv_star(s, k, T));
  return theta_l_of(s, k, T, qt, ql);
}

/* Sec. 2.2: solve theta_l*(T) - theta_l = 0 by the secant method.
 * reading: start at the unsaturated temperature T1 = Pi theta_l and at
 * T2 = T1 + L_v0 (q_t - q_v*(T1)) / c_pm; stop when |f| < sat_tol or after
 * sat_maxit secant updates; if q_t <= q_v*(T1) the air is unsaturated. */
static void saturation_adjust(const orc *s, int k, double th, double qt,
                              double *T_out, double *ql_out) {
  double T1 = exner(s, k, qt, 0.0) * th;
  double qs1 = qv_star(s, k, T1);
  if (qt <= qs1) { *T_out = T1; *ql_out = 0.0; return; }
  double Ta = T1, Tb = T1 + LV0 * (qt - qs1) / heat_cpm(qt, 0.0);
  double fa = theta_l_star(s, k, Ta, qt) - th;
  double fb = theta_l_star(s, k, Tb, qt) - th;
  for (int it = 0; it < s->p.sat_maxit; ++it) {
    if (fabs(fb) < s->p.sat_tol || fb == fa) break;
    double Tc = Tb - fb * (Tb - Ta) / (fb - fa);
    Ta = Tb; fa = fb;
    Tb = Tc; fb = theta_l_star(s, k, Tb, qt) - th;
  }
  *T_out = Tb;
  *ql_out = fmax(0.0, qt - qv_star(s, k, Tb));
}

/* ---- allocation ---------------------------------------------------------- */
void *orc_create(const orc_params *prm, const double *rho0) {
  orc *s = (orc *)calloc(1, sizeof(orc));
  if (!s) return NULL;
  s->p = *prm;
  s->n = (int64_t)prm->nx * prm->ny * prm->nz;
  s->dt = prm->dt;
  for (int f = 0; f < ORC_NFIELD; ++f) s->f[f] = (double *)calloc(s->n, sizeof(double));
  for (int t = 0; t < 8; ++t) s->tmp[t] = (double *)calloc(s->n, sizeof(double));
  int K = prm->K > 0 ? prm->K : 1;
  s->psi_prev = (double **)calloc(K, sizeof(double *));
  for (int k = 0; k < K; ++k) s->psi_prev[k] = (double *)calloc(s->n, sizeof(double));
  s->rho0 = (double *)calloc(prm->nz, sizeof(double));
  s->alpha0 = (double *)calloc(prm->nz, sizeof(double));
  s->p0 = (double *)calloc(prm->nz, sizeof(double));
  s->zc = (double *)calloc(prm->nz, sizeof(double));
  reference_state(s, rho0);
  return s;
}

void orc_destroy(void *vs) {
  orc *s = (orc *)vs;
  if (!s) return;
  for (int f = 0; f < ORC_NFIELD; ++f) free(s->f[f]);
  for (int t = 0; t < 8; ++t) free(s->tmp[t]);
  for (int k = 0; k < (s->p.K > 0 ? s->p.K : 1); ++k) free(s->psi_prev[k]);
  free(s->psi_prev);
  free(s->rho0); free(s->alpha0); free(s->p0); free(s->zc);
  free(s);
}

double *orc_field(void *vs, int id) {
  orc *s = (orc *)vs;
  return (id >= 0 && id < ORC_NFIELD) ? s->f[id] : NULL;
}
double orc_get_dt(void *vs) { return ((orc *)vs)->dt; }
void orc_set_dt(void *vs, double dt) { ((orc *)vs)->dt = dt; }
void orc_profiles(void *vs, double *rho0, double *p0) {
  orc *s = (orc *)vs;
  for (int k = 0; k < s->p.nz; ++k) { rho0[k] = s->rho0[k]; p0[k] = s->p0[k]; }
}

/* ---- Sec. 2.3: Smagorinsky-Lilly viscosity at every node ------------------- */
/* S = sqrt(2 S_ij S_ij) from nodal central differences (reading of "2-norm of
 * the strain rate tensor"); f_B = sqrt(clip(1 - N^2 / (Pr S^2), 0, 1)) with
 * N^2 = db/dz (reading of the moist buoyancy-frequency limiter). */
static double nu_node(const orc *s, const double *u, const double *v, const double *w,
                      const double *b, int i, int j, int k) {
  const uint32_t fl = s->p.flags;
  if (fl & ORC_CONST_NU) return s->p.nu_const;
  if (!(fl & ORC_SGS)) return 0.0;
  const double *vel[3] = {u, v, w};
  const int gh[3] = {GH_UV, GH_UV, GH_ODD};
  double g[3][3];
  for (int c = 0; c < 3; ++c)
    for (int d = 0; d < 3; ++d) {
      int di = d == 0, dj = d == 1, dk = d == 2;
      g[c][d] = (at(s, vel[c], gh[c], i + di, j + dj, k + dk) -
                 at(s, vel[c], gh[c], i - di, j - dj, k - dk)) / (2.0 * spacing(s, d));
    }
  double S2 = 0.0;
  for (int c = 0; c < 3; ++c)
    for (int d = 0; d < 3; ++d) {
      double Scd = 0.5 * (g[c][d] + g[d][c]);
      S2 += 2.0 * Scd * Scd;
    }
  double fB = 1.0;
  if ((fl & ORC_FB) && S2 > 0.0) {
    double N2 = (at(s, b, GH_EVEN, i, j, k + 1) - at(s, b, GH_EVEN, i, j, k - 1)) /
                (2.0 * s->p.dz);
    double x = 1.0 - N2 / (s->p.pr * S2);
    fB = sqrt(x < 0.0 ? 0.0 : (x > 1.0 ? 1.0 : x));
  }
  double delta = cbrt(s->p.dx * s->p.dy * s->p.dz);
  double cd = s->p.cs * delta;
  return cd * cd * fB * sqrt(S2);
}

void orc_nu_field(void *vs, const double *u, const double *v, const double *w,
                  const double *b, double *nu) {
  orc *s = (orc *)vs;
  const double *bb = b ? b : s->f[ORC_B];
#pragma omp parallel for schedule(static)
  for (int k = 0; k < s->p.nz; ++k)
    for (int j = 0; j < s->p.ny; ++j)
      for (int i = 0; i < s->p.nx; ++i)
        nu[IDX(s, i, j, k)] = nu_node(s, u, v, w, bb, i, j, k);
}

/* ---- Sec. 2.4: face quantities -------------------------------------------- */
/* The face "n + 1/2 in direction d" lies between node n and node n + e_d. */
static int is_surface_face(const orc *s, int d, int k) { return s->p.walls && d == 2 && k == -1; }
static int is_wall_face(const orc *s, int d, int k) {
  return s->p.walls && d == 2 && (k == -1 || k == s->p.nz - 1);
}

/* mass flux through the face: average of rho0 u_d at the two nodes */
static double mass_flux(const orc *s, const double *ud, int d, int i, int j, int k) {
  int di = d == 0, dj = d == 1, dk = d == 2;
  int g = d == 2 ? GH_ODD : GH_UV;
  return 0.5 * (prof(s, s->rho0, k) * at(s, ud, g, i, j, k) +
                prof(s, s->rho0, k + dk) * at(s, ud, g, i + di, j + dj, k + dk));
}

/* QUICK face value (Sec. 2.4): quadratic upstream interpolation.  F >= 0:
 * (-phi_{n-1} + 6 phi_n + 3 phi_{n+1}) / 8; F < 0: (3 phi_n + 6 phi_{n+1}
 * - phi_{n+2}) / 8. */
static double quick(const orc *s, const double *f, int g, double F, int d, int i, int j, int k) {
  int di = d == 0, dj = d == 1, dk = d == 2;
  double fm1 = at(s, f, g, i - di, j - dj, k - dk);
  double f0 = at(s, f, g, i, j, k);
  double f1 = at(s, f, g, i + di, j + dj, k + dk);
  double f2 = at(s, f, g, i + 2 * di, j + 2 * dj, k + 2 * dk);
  if (F >= 0.0) return (-fm1 + 6.0 * f0 + 3.0 * f1) / 8.0;
  return (3.0 * f0 + 6.0 * f1 - f2) / 8.0;
}

/* Third-order WENO face value with the local Lax-Friedrichs flux (Sec. 2.4,
 * the alternative advection scheme).  With the local speed |F| the
 * Lax-Friedrichs flux F (phi_L + phi_R) / 2 - |F| (phi_R - phi_L) / 2 takes
 * the reconstruction from the upwind side: for F >= 0 the left-biased one
 * from (phi_{n-1}, phi_n, phi_{n+1}), else the right-biased one from
 * (phi_n, phi_{n+1}, phi_{n+2}).  Each blends the two two-point candidates
 * (upwind extrapolation and centred average) with the ideal weights 1/3, 2/3
 * scaled by the inverse squared smoothness indicators; eps is our reading
 * (the paper gives none): 1e-6 times the squared largest magnitude of the
 * three values, plus 1e-18. */
static double weno3_side(double fa, double fb, double fc) {
  /* fa: the node two before the face on the upwind side, fb: the upwind
   * node, fc: the node across the face */
  const double q0 = 0.5 * (3.0 * fb - fa);
  const double q1 = 0.5 * (fb + fc);
  const double b0 = (fb - fa) * (fb - fa);
  const double b1 = (fc - fb) * (fc - fb);
  double m = fabs(fa);
  if (fabs(fb) > m) m = fabs(fb);
  if (fabs(fc) > m) m = fabs(fc);
  const double eps = 1e-6 * m * m + 1e-18;
  const double a0 = (1.0 / 3.0) / ((eps + b0) * (eps + b0));
  const double a1 = (2.0 / 3.0) / ((eps + b1) * (eps + b1));
  return (a0 * q0 + a1 * q1) / (a0 + a1);
}

static double weno3(const orc *s, const double *f, int g, double F, int d, int i, int j, int k) {
  int di = d == 0, dj = d == 1, dk = d == 2;
  double fm1 = at(s, f, g, i - di, j - dj, k - dk);
  double f0 = at(s, f, g, i, j, k);
  double f1 = at(s, f, g, i + di, j + dj, k + dk);
  double f2 = at(s, f, g, i + 2 * di, j + 2 * dj, k + 2 * dk);
  if (F >= 0.0) return weno3_side(fm1, f0, f1);
  return weno3_side(f2, f1, f0);
}

/* face value of the configured advection scheme */
static double face_value(const orc *s, const double *f, int g, double F, int d, int i, int j, int k) {
  return s->p.advection == 1 ? weno3(s, f, g, F, d, i, j, k) : quick(s, f, g, F, d, i, j, k);
}

/* ---- a1: thermodynamics once per step ------------------------------------- */
static void thermo(orc *s) {
  const double *th = s->f[ORC_THH], *qt = s->f[ORC_QTH];
  double *T = s->f[ORC_T], *ql = s->f[ORC_QL], *b = s->f[ORC_B], *srad = s->f[ORC_SRAD];
  const uint32_t fl = s->p.flags;
  const int nx = s->p.nx, ny = s->p.ny, nz = s->p.nz;
#pragma omp parallel for schedule(static)
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        int64_t c = IDX(s, i, j, k);
        double Tc, qlc;
        if (fl & ORC_MOIST) {
          saturation_adjust(s, k, th[c], qt[c], &Tc, &qlc);
        } else {
          qlc = 0.0;
          Tc = exner(s, k, qt[c], 0.0) * th[c];
        }
        T[c] = Tc;
        ql[c] = qlc;
        /* b = g (alpha - alpha0) / alpha0, alpha = R_m T / p0 */
        if (fl & ORC_BUOY) {
          double alpha = gas_rm(qt[c], qlc) * Tc / s->p0[k];
          b[c] = GRAV * (alpha - s->alpha0[k]) / s->alpha0[k];
        } else {
          b[c] = 0.0;
        }
        srad[c] = 0.0;
      }
  if (!(fl & ORC_RAD)) return;
  /* reading: longwave flux through the face above node k,
   *   F(k+1/2) = F0 exp(-kappa LWP(above)) + F1 exp(-kappa LWP(below)),
   * LWP = sum rho0 q_l dz; source -(1/(c_pm Pi)) dF/dz in the rho0 theta_l
   * equation (Eq. e:potential_temperature). */
  const double dz = s->p.dz;
#pragma omp parallel for schedule(static)
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      double total = 0.0;
      for (int k = 0; k < nz; ++k) total += s->rho0[k] * ql[IDX(s, i, j, k)] * dz;
      double below = 0.0;   /* LWP below the face under node k */
      double Fm = s->p.rad_f0 * exp(-s->p.rad_kappa * total) + s->p.rad_f1;
      for (int k = 0; k < nz; ++k) {
        int64_t c = IDX(s, i, j, k);
        below += s->rho0[k] * ql[c] * dz;
        double above = total - below;
        double Fp = s->p.rad_f0 * exp(-s->p.rad_kappa * above) +
                    s->p.rad_f1 * exp(-s->p.rad_kappa * below);
        double cpm = heat_cpm(qt[c], ql[c]);
        double Pi = exner(s, k, qt[c], ql[c]);
        srad[c] = -(Fp - Fm) / dz / (cpm * Pi);
        Fm = Fp;
      }
    }
}

int orc_begin_step(void *vs) {
  orc *s = (orc *)vs;
  const int64_t n = s->n;
  if (s->dt <= 0.0) {
    /* Courant-number time step from the initial field, then held fixed */
    double cmax = 0.0;
    for (int64_t c = 0; c < n; ++c) {
      double v = fabs(s->f[ORC_U][c]) / s->p.dx + fabs(s->f[ORC_V][c]) / s->p.dy +
                 fabs(s->f[ORC_W][c]) / s->p.dz;
      if (v > cmax) cmax = v;
    }
    if (!(cmax > 0.0)) return 1;
    s->dt = s->p.cfl / cmax;
  }
  /* reading: U^(0) = U^n, p^(0) = p^n, phi^(0) = phi^{n+1/2}, dp^(0) = 0 */
  memcpy(s->f[ORC_UN], s->f[ORC_U], n * sizeof(double));
  memcpy(s->f[ORC_VN], s->f[ORC_V], n * sizeof(double));
  memcpy(s->f[ORC_WN], s->f[ORC_W], n * sizeof(double));
  memcpy(s->f[ORC_THH], s->f[ORC_TH], n * sizeof(double));
  memcpy(s->f[ORC_QTH], s->f[ORC_QT], n * sizeof(double));
  memset(s->f[ORC_PSI], 0, n * sizeof(double));
  thermo(s);
  s->sub = 0;
  return 0;
}

/* ---- a3: scalar predictor (Eq. scalar_prediction_step) -------------------- */
/* (rho0 phi)^{k+1} = (rho0 phi)^{n+1/2} + dt [ -div((rho0 u)^{n+1} phi^{n+1})
 *     + div(rho0 D_phi grad phi^{n+1}) + S_phi ],
 * u^{n+1} = u^k, phi^{n+1} = (phi^k + phi^{n+1/2}) / 2, D_phi = nu_t / Pr or
 * nu_t / Sc. */
void orc_scalar_stage(void *vs) {
  orc *s = (orc *)vs;
  const uint32_t fl = s->p.flags;
  const int nx = s->p.nx, ny = s->p.ny, nz = s->p.nz;
  const double dt = s->dt;
  const double *u = s->f[ORC_U], *v = s->f[ORC_V], *w = s->f[ORC_W];
  const double *vel[3] = {u, v, w};
  double *nu = s->tmp[0];
  orc_nu_field(s, u, v, w, s->f[ORC_B], nu);
  memcpy(s->f[ORC_NU], nu, s->n * sizeof(double));

  for (int q = 0; q < 2; ++q) {
    double *phik = s->f[q == 0 ? ORC_TH : ORC_QT];
    const double *phih = s->f[q == 0 ? ORC_THH : ORC_QTH];
    double *bar = s->tmp[1], *out = s->tmp[2];
    const double schmidt = q == 0 ? s->p.pr : s->p.sc;
    /* surface flux rho0 (w' phi')_s: SHF / c_pd for theta_l, LHF / L_v0 for q_t */
    const double sflux = q == 0 ? s->p.shf / CPD : s->p.lhf / LV0;
    for (int64_t c = 0; c < s->n; ++c) bar[c] = 0.5 * (phik[c] + phih[c]);
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
          double tend = 0.0;
          for (int d = 0; d < 3; ++d) {
            int di = d == 0, dj = d == 1, dk = d == 2;
            double h = spacing(s, d);
            double flux[2];   /* total flux through faces -1/2 and +1/2 */
            for (int side = 0; side < 2; ++side) {
              int fi = i - (side == 0 ? di : 0), fj = j - (side == 0 ? dj : 0),
                  fk = k - (side == 0 ? dk : 0);
              double adv = 0.0, dif = 0.0;
              if (is_wall_face(s, d, fk)) {
                if (is_surface_face(s, d, fk) && (fl & ORC_SFC)) dif = -sflux;
              } else {
                if (fl & ORC_ADV) {
                  double F = mass_flux(s, vel[d], d, fi, fj, fk);
                  adv = F * face_value(s, bar, GH_EVEN, F, d, fi, fj, fk);
                }
                double nuf = 0.5 * (at(s, nu, GH_EVEN, fi, fj, fk) +
                                    at(s, nu, GH_EVEN, fi + di, fj + dj, fk + dk));
                double rhof = 0.5 * (prof(s, s->rho0, fk) + prof(s, s->rho0, fk + dk));
                dif = rhof * nuf / schmidt *
                      (at(s, bar, GH_EVEN, fi + di, fj + dj, fk + dk) -
                       at(s, bar, GH_EVEN, fi, fj, fk)) / h;
              }
              flux[side] = -adv + dif;
            }
            tend += (flux[1] - flux[0]) / h;
          }
          int64_t c = IDX(s, i, j, k);
          if (fl & ORC_SUBS) {
            /* reading: the paper's w_sub is the subsidence speed D z >= 0;
             * the air sinks, so dphi/dz is taken upwind (from above). */
            double wsub = s->p.subs_div * s->zc[k];
            double dphidz = (at(s, bar, GH_EVEN, i, j, k + 1) - bar[c]) / s->p.dz;
            tend += s->rho0[k] * wsub * dphidz;
          }
          if (q == 0 && (fl & ORC_RAD)) tend += s->f[ORC_SRAD][c];
          out[c] = (s->rho0[k] * phih[c] + dt * tend) / s->rho0[k];
        }
    memcpy(phik, out, s->n * sizeof(double));
  }
}

/* ---- a4: momentum predictor (Eq. momentum_prediction_step) ----------------- */
/* rho0 u^ = rho0 u^n + dt [ -rho0 G(alpha0 p^k) + R^{n+1/2} ],
 * R = -div(rho0 u (x) u) + div(rho0 sigma) + rho0 b k - f k x rho0 (u - u_g)
 *     - sponge, all at (.)^{n+1/2} = ((.)^k + (.)^n) / 2.
 * Then the Poisson right side (Eq. pressure_correction with App. A):
 * rhs = alpha0 / dt D(rho0 u^) - C^k. */
void orc_momentum_stage(void *vs) {
  orc *s = (orc *)vs;
  const uint32_t fl = s->p.flags;
  const int nx = s->p.nx, ny = s->p.ny, nz = s->p.nz;
  const double dt = s->dt;
  double *uh[3] = {s->tmp[3], s->tmp[4], s->tmp[5]};
  const double *un[3] = {s->f[ORC_UN], s->f[ORC_VN], s->f[ORC_WN]};
  const double *uk[3] = {s->f[ORC_U], s->f[ORC_V], s->f[ORC_W]};
  double *hat[3] = {s->f[ORC_UH], s->f[ORC_VH], s->f[ORC_WH]};
  const int gh[3] = {GH_UV, GH_UV, GH_ODD};
  for (int c = 0; c < 3; ++c)
    for (int64_t m = 0; m < s->n; ++m) uh[c][m] = 0.5 * (uk[c][m] + un[c][m]);
  double *nu = s->tmp[0];
  orc_nu_field(s, uh[0], uh[1], uh[2], s->f[ORC_B], nu);
  memcpy(s->f[ORC_NU], nu, s->n * sizeof(double));
  /* alpha0 p' with the pressure's mirror ghosts */
  double *ap = s->tmp[6];
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) ap[IDX(s, i, j, k)] = s->alpha0[k] * s->f[ORC_P][IDX(s, i, j, k)];

  const double H = nz * s->p.dz;
  const double zs = (1.0 - s->p.sponge_frac) * H;
  const double target[3] = {s->p.ug, s->p.vg, 0.0};

#pragma omp parallel for schedule(static)
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        int64_t m = IDX(s, i, j, k);
        double r0 = s->rho0[k];
        for (int c = 0; c < 3; ++c) {
          int ci = c == 0, cj = c == 1, ck = c == 2;
          double R = 0.0;
          for (int d = 0; d < 3; ++d) {
            int di = d == 0, dj = d == 1, dk = d == 2;
            double h = spacing(s, d);
            double flux[2];
            for (int side = 0; side < 2; ++side) {
              int fi = i - (side == 0 ? di : 0), fj = j - (side == 0 ? dj : 0),
                  fk = k - (side == 0 ? dk : 0);
              double adv = 0.0, tau = 0.0;
              if (is_surface_face(s, d, fk)) {
                /* reading: free-slip surface with zero momentum flux */
                flux[side] = 0.0;
                continue;
              }
              if ((fl & ORC_ADV) && !is_wall_face(s, d, fk)) {
                double F = mass_flux(s, uh[d], d, fi, fj, fk);
                adv = F * face_value(s, uh[c], gh[c], F, d, fi, fj, fk);
              }
              /* SGS stress rho0 nu_t (d_d u_c + d_c u_d) on the face: the normal
               * derivative is compact; the tangential one is the mean of the
               * two nodal central differences. */
              double dn = (at(s, uh[c], gh[c], fi + di, fj + dj, fk + dk) -
                           at(s, uh[c], gh[c], fi, fj, fk)) / h;
              double dtg;
              if (c == d) {
                dtg = dn;
              } else {
                double hc = spacing(s, c);
                double g0 = (at(s, uh[d], gh[d], fi + ci, fj + cj, fk + ck) -
                             at(s, uh[d], gh[d], fi - ci, fj - cj, fk - ck)) / (2.0 * hc);
                double g1 = (at(s, uh[d], gh[d], fi + di + ci, fj + dj + cj, fk + dk + ck) -
                             at(s, uh[d], gh[d], fi + di - ci, fj + dj - cj, fk + dk - ck)) /
                            (2.0 * hc);
                dtg = 0.5 * (g0 + g1);
              }
              double nuf = 0.5 * (at(s, nu, GH_EVEN, fi, fj, fk) +
                                  at(s, nu, GH_EVEN, fi + di, fj + dj, fk + dk));
              double rhof = 0.5 * (prof(s, s->rho0, fk) + prof(s, s->rho0, fk + dk));
              tau = rhof * nuf * (dn + dtg);
              flux[side] = -adv + tau;
            }
            R += (flux[1] - flux[0]) / h;
          }
          if ((fl & ORC_BUOY) && c == 2) R += r0 * s->f[ORC_B][m];
          if (fl & ORC_CORIOLIS) {
            /* -f k x rho0 (u - u_g) = (f rho0 (v - v_g), -f rho0 (u - u_g), 0) */
            if (c == 0) R += s->p.f_cor * r0 * (uh[1][m] - s->p.vg);
            if (c == 1) R -= s->p.f_cor * r0 * (uh[0][m] - s->p.ug);
          }
          if ((fl & ORC_SPONGE) && s->zc[k] > zs) {
            /* reading: Rayleigh rate rising as sin^2 from z_s to the lid */
            double x = sin(0.5 * M_PI * (s->zc[k] - zs) / (H - zs));
            R -= s->p.sponge_rate * x * x * r0 * (uh[c][m] - target[c]);
          }
          double hc = spacing(s, c);
          double gp = (at(s, ap, GH_EVEN, i + ci, j + cj, k + ck) -
                       at(s, ap, GH_EVEN, i - ci, j - cj, k - ck)) / (2.0 * hc);
          hat[c][m] = (r0 * un[c][m] + dt * (-r0 * gp + R)) / r0;
        }
      }

  orc_poisson_rhs(s);
}

/* The Poisson right side (Eq. pressure_correction with App. A) from the
 * predicted momentum u^ and the last increment psi:
 * rhs = alpha0 / dt D(rho0 u^) - C^k (compact operator), or D(rho0 u^) / dt. */
void orc_poisson_rhs(void *vs) {
  orc *s = (orc *)vs;
  const int nx = s->p.nx, ny = s->p.ny, nz = s->p.nz;
  const double dt = s->dt;
  const double *hat[3] = {s->f[ORC_UH], s->f[ORC_VH], s->f[ORC_WH]};
  const int gh[3] = {GH_UV, GH_UV, GH_ODD};
  double *rhs = s->f[ORC_RHS];
  const double *psi = s->f[ORC_PSI];
#pragma omp parallel for schedule(static)
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        double div = 0.0;
        for (int d = 0; d < 3; ++d) {
          int di = d == 0, dj = d == 1, dk = d == 2;
          div += (prof(s, s->rho0, k + dk) * at(s, hat[d], gh[d], i + di, j + dj, k + dk) -
                  prof(s, s->rho0, k - dk) * at(s, hat[d], gh[d], i - di, j - dj, k - dk)) /
                 (2.0 * spacing(s, d));
        }
        double val;
        if (s->p.op == 0) {
          /* App. A: C = sum_l [psi_{l+2} - 4 psi_{l+1} + 6 psi_l - 4 psi_{l-1}
           * + psi_{l-2}] / (4 Delta_l^2), subtracted from alpha0 / dt D(rho0 u^) */
          double C = 0.0;
          for (int d = 0; d < 3; ++d) {
            int di = d == 0, dj = d == 1, dk = d == 2;
            double h = spacing(s, d);
            C += (at(s, psi, GH_EVEN, i + 2 * di, j + 2 * dj, k + 2 * dk) -
                  4.0 * at(s, psi, GH_EVEN, i + di, j + dj, k + dk) +
                  6.0 * at(s, psi, GH_EVEN, i, j, k) -
                  4.0 * at(s, psi, GH_EVEN, i - di, j - dj, k - dk) +
                  at(s, psi, GH_EVEN, i - 2 * di, j - 2 * dj, k - 2 * dk)) / (4.0 * h * h);
          }
          val = s->alpha0[k] / dt * div - C;
        } else {
          val = div / dt;
        }
        rhs[IDX(s, i, j, k)] = val;
      }
}

/* ---- a5: the Poisson operator and its solvers ----------------------------- */
/* op 0: compact Laplacian L_c psi = sum_l (psi_{l+1} - 2 psi_l + psi_{l-1}) / Delta_l^2
 *       with homogeneous Neumann (mirror) ghosts at walls (Sec. 2.4, App. A);
 * op 1: D(rho0 G psi), the divergence of the gradient used by the correction. */
void orc_apply_poisson(void *vs, int32_t op, const double *x, double *y) {
  orc *s = (orc *)vs;
  const int nx = s->p.nx, ny = s->p.ny, nz = s->p.nz;
  if (op == 0) {
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
          double acc = 0.0;
          for (int d = 0; d < 3; ++d) {
            int di = d == 0, dj = d == 1, dk = d == 2;
            double h = spacing(s, d);
            acc += (at(s, x, GH_EVEN, i + di, j + dj, k + dk) - 2.0 * at(s, x, GH_EVEN, i, j, k) +
                    at(s, x, GH_EVEN, i - di, j - dj, k - dk)) / (h * h);
          }
          y[IDX(s, i, j, k)] = acc;
        }
    return;
  }
  double *g[3] = {s->tmp[7], s->tmp[1], s->tmp[2]};
  for (int d = 0; d < 3; ++d) {
    int di = d == 0, dj = d == 1, dk = d == 2;
    double h = spacing(s, d);
    for (int k = 0; k < nz; ++k)
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i)
          g[d][IDX(s, i, j, k)] = s->rho0[k] *
              (at(s, x, GH_EVEN, i + di, j + dj, k + dk) - at(s, x, GH_EVEN, i - di, j - dj, k - dk)) /
              (2.0 * h);
  }
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        double acc = 0.0;
        for (int d = 0; d < 3; ++d) {
          int di = d == 0, dj = d == 1, dk = d == 2;
          int gh = d == 2 ? GH_ODD : GH_UV;
          acc += (at(s, g[d], gh, i + di, j + dj, k + dk) - at(s, g[d], gh, i - di, j - dj, k - dk)) /
                 (2.0 * spacing(s, d));
        }
        y[IDX(s, i, j, k)] = acc;
      }
}

static double dot(const orc *s, const double *a, const double *b) {
  const int nz = s->p.nz;
  const int64_t plane = (int64_t)s->p.nx * s->p.ny;
  double *part = (double *)malloc(nz * sizeof(double));
#pragma omp parallel for schedule(static)
  for (int k = 0; k < nz; ++k) {
    double acc = 0.0;
    for (int64_t m = k * plane; m < (k + 1) * plane; ++m) acc += a[m] * b[m];
    part[k] = acc;
  }
  double sum = 0.0;
  for (int k = 0; k < nz; ++k) sum += part[k];
  free(part);
  return sum;
}

static double mean(const orc *s, const double *a) {
  const int nz = s->p.nz;
  const int64_t plane = (int64_t)s->p.nx * s->p.ny;
  double sum = 0.0;
  for (int k = 0; k < nz; ++k) {
    double acc = 0.0;
    for (int64_t m = k * plane; m < (k + 1) * plane; ++m) acc += a[m];
    sum += acc;
  }
  return sum / (double)s->n;
}

/* Solve A x = b for the mean-free x.  The mean of b is removed first (the
 * operator's null space holds the constants).  Conjugate gradient or weighted
 * Jacobi (x <- x + omega (b - A x) / diag(A), the paper's solver, Sec. 2.4),
 * both stopping at ||b - A x||_2 <= tol ||b||_2.  Returns 0 when converged. */
int orc_poisson(void *vs, int32_t op, int32_t solver, const double *b_in, double *x,
                double tol, int32_t maxit, int32_t *iters, double *res) {
  orc *s = (orc *)vs;
  const int64_t n = s->n;
  double *b = (double *)malloc(n * sizeof(double));
  double *r = (double *)malloc(n * sizeof(double));
  double *pv = (double *)malloc(n * sizeof(double));
  double *q = (double *)malloc(n * sizeof(double));
  double mb = mean(s, b_in);
  for (int64_t m = 0; m < n; ++m) b[m] = b_in[m] - mb;
  double bn = sqrt(dot(s, b, b));
  int it = 0, status = 0;
  double rel = 0.0;
  if (bn == 0.0) {
    memset(x, 0, n * sizeof(double));
  } else if (solver == 0) {
    orc_apply_poisson(s, op, x, q);
    for (int64_t m = 0; m < n; ++m) { r[m] = b[m] - q[m]; pv[m] = r[m]; }
    double rr = dot(s, r, r);
    rel = sqrt(rr) / bn;
    while (rel > tol && it < maxit) {
      orc_apply_poisson(s, op, pv, q);
      double alpha = rr / dot(s, pv, q);
      for (int64_t m = 0; m < n; ++m) { x[m] += alpha * pv[m]; r[m] -= alpha * q[m]; }
      double rr_new = dot(s, r, r);
      ++it;
      rel = sqrt(rr_new) / bn;
      double beta = rr_new / rr;
      rr = rr_new;
      for (int64_t m = 0; m < n; ++m) pv[m] = r[m] + beta * pv[m];
    }
    if (rel > tol) status = 1;
  } else {
    /* diagonal of the compact operator, with the mirror ghost folded in */
    const int nx = s->p.nx, ny = s->p.ny, nz = s->p.nz;
    double *diag = pv;
    for (int k = 0; k < nz; ++k) {
      double dzz = -2.0 / (s->p.dz * s->p.dz);
      if (s->p.walls && (k == 0 || k == nz - 1)) dzz = -1.0 / (s->p.dz * s->p.dz);
      if (s->p.walls && nz == 1) dzz = 0.0;
      double dg = -2.0 / (s->p.dx * s->p.dx) - 2.0 / (s->p.dy * s->p.dy) + dzz;
      for (int64_t m = (int64_t)k * nx * ny; m < (int64_t)(k + 1) * nx * ny; ++m) diag[m] = dg;
    }
    orc_apply_poisson(s, 0, x, q);
    for (int64_t m = 0; m < n; ++m) r[m] = b[m] - q[m];
    rel = sqrt(dot(s, r, r)) / bn;
    while (rel > tol && it < maxit) {
      for (int64_t m = 0; m < n; ++m) x[m] += s->p.omega * r[m] / diag[m];
      orc_apply_poisson(s, 0, x, q);
      for (int64_t m = 0; m < n; ++m) r[m] = b[m] - q[m];
      ++it;
      rel = sqrt(dot(s, r, r)) / bn;
    }
    if (rel > tol) status = 1;
  }
  /* gauge: the solution is taken with zero mean */
  double mx = mean(s, x);
  for (int64_t m = 0; m < n; ++m) x[m] -= mx;
  if (iters) *iters = it;
  if (res) *res = rel;
  free(b); free(r); free(pv); free(q);
  return status;
}

int orc_solve_stage(void *vs, int32_t *iters, double *res) {
  orc *s = (orc *)vs;
  double *psi = s->f[ORC_PSI];
  int k = s->sub < s->p.K ? s->sub : s->p.K - 1;
  if (s->p.warm == 1) memcpy(psi, s->psi_prev[k], s->n * sizeof(double));
  else memset(psi, 0, s->n * sizeof(double));
  int st = orc_poisson(s, s->p.op, s->p.solver, s->f[ORC_RHS], psi, s->p.tol, s->p.maxit,
                       iters, res);
  memcpy(s->psi_prev[k], psi, s->n * sizeof(double));
  return st;
}

/* ---- a7: correction (Sec. 2.4) --------------------------------------------- */
/* (rho0 u)^{k+1} = (rho0 u)^ - dt rho0 G(alpha0 dp);  p^{k+1} = p^k + dp */
void orc_correct_stage(void *vs) {
  orc *s = (orc *)vs;
  const int nx = s->p.nx, ny = s->p.ny, nz = s->p.nz;
  const double dt = s->dt;
  const double *psi = s->f[ORC_PSI];
  double *uk[3] = {s->f[ORC_U], s->f[ORC_V], s->f[ORC_W]};
  const double *hat[3] = {s->f[ORC_UH], s->f[ORC_VH], s->f[ORC_WH]};
#pragma omp parallel for schedule(static)
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        int64_t m = IDX(s, i, j, k);
        for (int c = 0; c < 3; ++c) {
          int ci = c == 0, cj = c == 1, ck = c == 2;
          double g = (at(s, psi, GH_EVEN, i + ci, j + cj, k + ck) -
                      at(s, psi, GH_EVEN, i - ci, j - cj, k - ck)) / (2.0 * spacing(s, c));
          uk[c][m] = (s->rho0[k] * hat[c][m] - dt * s->rho0[k] * g) / s->rho0[k];
        }
        /* dp = rho0 (alpha0 dp) */
        s->f[ORC_P][m] += s->rho0[k] * psi[m];
      }
  s->sub += 1;
}

void orc_end_step(void *vs) {
  orc *s = (orc *)vs;
  s->step += 1;
  s->sub = 0;
}

int orc_step(void *vs, int32_t nsteps, int32_t *iters_total) {
  orc *s = (orc *)vs;
  int status = 0, total = 0;
  for (int n = 0; n < nsteps; ++n) {
    if (orc_begin_step(s)) return 2;
    for (int k = 0; k < s->p.K; ++k) {
      orc_scalar_stage(s);
      orc_momentum_stage(s);
      int32_t it = 0;
      double res = 0.0;
      if (orc_solve_stage(s, &it, &res)) status = 1;
      total += it;
      orc_correct_stage(s);
    }
    orc_end_step(s);
  }
  if (iters_total) *iters_total = total;
  return status;
}

/* ---- single-cell thermodynamics for the pins ------------------------------ */
void orc_saturation(void *vs, int32_t k, double th, double qt, double *T, double *ql) {
  saturation_adjust((orc *)vs, k, th, qt, T, ql);
}
double orc_theta_l_star(void *vs, int32_t k, double T, double qt) {
  return theta_l_star((orc *)vs, k, T, qt);
}
double orc_qv_star(void *vs, int32_t k, double T) { return qv_star((orc *)vs, k, T); }

/* ---- a8: diagnostics -------------------------------------------------------- */
/* out: [0] sum rho0 theta_l dV, [1] sum rho0 q_t dV, [2..4] sum rho0 u_c dV,
 * [5] kinetic energy 1/2 sum rho0 |u|^2 dV, [6] max Courant number,
 * [7] max |D(rho0 u)|, [8] count of non-finite values, [9] sum rho0 q_l dV */
void orc_diagnostics(void *vs, double *out) {
  orc *s = (orc *)vs;
  const int nx = s->p.nx, ny = s->p.ny, nz = s->p.nz;
  const double dV = s->p.dx * s->p.dy * s->p.dz;
  const double *vel[3] = {s->f[ORC_U], s->f[ORC_V], s->f[ORC_W]};
  const int gh[3] = {GH_UV, GH_UV, GH_ODD};
  double acc[ORC_NDIAG] = {0};
  for (int k = 0; k < nz; ++k) {
    double pl[ORC_NDIAG] = {0};
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        int64_t m = IDX(s, i, j, k);
        double r0 = s->rho0[k];
        pl[0] += r0 * s->f[ORC_TH][m] * dV;
        pl[1] += r0 * s->f[ORC_QT][m] * dV;
        double ke = 0.0, cfl = 0.0, div = 0.0;
        for (int c = 0; c < 3; ++c) {
          int ci = c == 0, cj = c == 1, ck = c == 2;
          pl[2 + c] += r0 * vel[c][m] * dV;
          ke += vel[c][m] * vel[c][m];
          cfl += fabs(vel[c][m]) / spacing(s, c);
          div += (prof(s, s->rho0, k + ck) * at(s, vel[c], gh[c], i + ci, j + cj, k + ck) -
                  prof(s, s->rho0, k - ck) * at(s, vel[c], gh[c], i - ci, j - cj, k - ck)) /
                 (2.0 * spacing(s, c));
        }
        pl[5] += 0.5 * r0 * ke * dV;
        if (cfl * s->dt > pl[6]) pl[6] = cfl * s->dt;
        if (fabs(div) > pl[7]) pl[7] = fabs(div);
        for (int f = 0; f < ORC_NFIELD; ++f)
          if (!isfinite(s->f[f][m])) pl[8] += 1.0;
        pl[9] += r0 * s->f[ORC_QL][m] * dV;
      }
    for (int q = 0; q < ORC_NDIAG; ++q) {
      if (q == 6 || q == 7) acc[q] = pl[q] > acc[q] ? pl[q] : acc[q];
      else acc[q] += pl[q];
    }
  }
  for (int q = 0; q < ORC_NDIAG; ++q) out[q] = acc[q];
}
