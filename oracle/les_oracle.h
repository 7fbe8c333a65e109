/*
 * les_oracle.h -- FP64 CPU oracle of the anelastic LES time step.
 *
 * TEST INFRASTRUCTURE ONLY.  This header and les_oracle.c are a plain, slow,
 * obviously-correct restatement of the discretisation of Chammas et al.
 * (arXiv 2301.04698), Sec. 2.1-2.4 and Appendix A.  Only tests/, the package's
 * smoke() check and bench.py's CPU baseline may load it.  It shares no code,
 * header, constant table or helper with the CUDA path.
 *
 * Every field is a double array of nx*ny*nz values, x fastest:
 *   index(i,j,k) = (k*ny + j)*nx + i,  node i sits at x = (i+1/2) dx.
 */
#ifndef LES_ORACLE_H
#define LES_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* physics switches (bit flags) */
#define ORC_ADV       (1u << 0)   /* QUICK advection (Sec. 2.4) */
#define ORC_SGS       (1u << 1)   /* Smagorinsky-Lilly viscosity (Sec. 2.3) */
#define ORC_CONST_NU  (1u << 2)   /* constant viscosity instead of Smagorinsky */
#define ORC_MOIST     (1u << 3)   /* saturation adjustment (Sec. 2.2) */
#define ORC_BUOY      (1u << 4)   /* buoyancy rho0 b k (Eq. momentum) */
#define ORC_CORIOLIS  (1u << 5)   /* -f k x rho0 (u - u_g) */
#define ORC_SPONGE    (1u << 6)   /* Rayleigh sponge, top fraction of the domain */
#define ORC_RAD       (1u << 7)   /* longwave radiative flux divergence */
#define ORC_SUBS      (1u << 8)   /* large-scale subsidence */
#define ORC_SFC       (1u << 9)   /* prescribed surface fluxes of theta_l, q_t */
#define ORC_FB        (1u << 10)  /* buoyancy factor f_B in nu_t */

/* field ids */
enum {
  ORC_U = 0, ORC_V, ORC_W,        /* velocity u^k (u^n between steps)      */
  ORC_P,                          /* perturbation pressure p'^k             */
  ORC_TH, ORC_QT,                 /* scalars phi^k (phi^{n+1/2} at step 0)  */
  ORC_UN, ORC_VN, ORC_WN,         /* u^n                                    */
  ORC_THH, ORC_QTH,               /* phi^{n+1/2}                            */
  ORC_UH, ORC_VH, ORC_WH,         /* predicted velocity (rho0 u)^ / rho0    */
  ORC_RHS,                        /* Poisson right-hand side                */
  ORC_PSI,                        /* alpha0 * dp (Poisson unknown)          */
  ORC_B, ORC_QL, ORC_T,           /* buoyancy, liquid water, temperature    */
  ORC_SRAD,                       /* radiative source of rho0 theta_l       */
  ORC_NU,                         /* last nu_t computed (diagnostic)        */
  ORC_NFIELD
};

typedef struct orc_params {
  int32_t nx, ny, nz;
  int32_t walls;          /* 0: periodic in z; 1: surface + lid (Sec. 4)      */
  double dx, dy, dz;
  double dt;              /* > 0: fixed; 0: from cfl on the first step        */
  double cfl;
  int32_t K;              /* sub-iterations per step                          */
  int32_t solver;         /* 0 conjugate gradient, 1 weighted Jacobi          */
  int32_t op;             /* 0 compact Laplacian + Appendix A term, 1 D(rho0 G) */
  int32_t warm;           /* 0 zero, 1 previous step's solution               */
  double tol;             /* relative residual ||b - A x|| / ||b||            */
  int32_t maxit;
  double omega;           /* Jacobi weight                                    */
  uint32_t flags;
  double cs, pr, sc, nu_const;
  double f_cor, ug, vg;
  double sponge_frac, sponge_rate;
  double subs_div;        /* D in w_sub = D z                                 */
  double shf, lhf;        /* surface sensible / latent heat flux (W m^-2)     */
  double rad_f0, rad_f1, rad_kappa;
  double theta0, p00;
  double sat_tol;         /* secant stop |theta_l* - theta_l| (K)             */
  int32_t sat_maxit;
  int32_t advection;      /* 0 QUICK; 1 WENO3 with the local Lax-Friedrichs flux */
} orc_params;

void   *orc_create(const orc_params *prm, const double *rho0 /* nz or NULL */);
void    orc_destroy(void *s);
double *orc_field(void *s, int id);
double  orc_get_dt(void *s);
void    orc_set_dt(void *s, double dt);
void    orc_profiles(void *s, double *rho0, double *p0);

int  orc_begin_step(void *s);
void orc_scalar_stage(void *s);
void orc_momentum_stage(void *s);
void orc_poisson_rhs(void *s); /* the right side alone, from u^ and psi */
int  orc_solve_stage(void *s, int32_t *iters, double *res);
void orc_correct_stage(void *s);
void orc_end_step(void *s);
int  orc_step(void *s, int32_t nsteps, int32_t *iters_total);

/* building blocks exposed for the closed-form pins */
void orc_apply_poisson(void *s, int32_t op, const double *x, double *y);
int  orc_poisson(void *s, int32_t op, int32_t solver, const double *b, double *x,
                 double tol, int32_t maxit, int32_t *iters, double *res);
void orc_nu_field(void *s, const double *u, const double *v, const double *w,
                  const double *b, double *nu);
void orc_saturation(void *s, int32_t k, double th, double qt, double *T, double *ql);
double orc_theta_l_star(void *s, int32_t k, double T, double qt);
double orc_qv_star(void *s, int32_t k, double T);
void orc_diagnostics(void *s, double *out /* ORC_NDIAG */);
#define ORC_NDIAG 10

#ifdef __cplusplus
}
#endif
#endif
