/*
 * les.h -- C ABI of the GB300 LES time-step library (libles.so).
 *
 * One time step of the anelastic moist large-eddy simulation of Chammas et al.,
 * "Accelerating large-eddy simulations of clouds with Tensor Processing Units"
 * (arXiv 2301.04698): the explicit QUICK / Smagorinsky / thermodynamics stencil
 * updates and the pressure-correction Poisson solve of the iterative
 * predictor-corrector scheme (Sec. 2.1-2.4, Appendix A), on one CUDA device.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Grid: nx * ny * nz collocated nodes, node (i,j,k) at ((i+1/2)dx, (j+1/2)dy,
 *   (k+1/2)dz).  Every field is one contiguous array of nx*ny*nz values in the
 *   handle's precision (float for precision 32, double for 64), x fastest:
 *   element (i,j,k) is at offset (k*ny + j)*nx + i.  Periodic in x and y;
 *   periodic in z or bounded by a surface (k = -1/2) and a lid (k = nz - 1/2).
 * - Memory: the library allocates no device memory.  The caller supplies one
 *   device workspace of les_workspace_bytes() bytes (e.g. a torch uint8 tensor)
 *   that the handle borrows until les_destroy(); every field, solver vector and
 *   reduction scratch lives in it.  Host buffers passed to get/set are
 *   borrowed only for the duration of the call.
 * - Streams: all device work is issued on the handle's stream (cudaStream_t
 *   given as void*; NULL = legacy default stream).  Calls return when the work
 *   is enqueued, except where a result must come back to the host (solver
 *   status, diagnostics, host copies), which synchronise the stream.
 * - Errors: every call returns a status (LES_OK = 0).  No exception or abort
 *   crosses the ABI; les_last_error() gives a message for the handle.
 * - Threads: a handle must not be used from two threads at once.
 */
#ifndef LES_H
#define LES_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LES_ABI_VERSION 1

/* ---- status codes -------------------------------------------------------- */
#define LES_OK                 0
#define LES_ERR_INVALID_ARG    1  /* bad pointer, size, id or configuration  */
#define LES_ERR_CUDA           2  /* a CUDA runtime call or launch failed     */
#define LES_ERR_NOT_CONVERGED  3  /* Poisson solve hit maxit; state is valid  */
#define LES_ERR_NONFINITE      4  /* NaN / Inf detected in the state          */
#define LES_ERR_TIMEOUT        5  /* a bounded device wait gave up            */
#define LES_ERR_STATE          6  /* call out of order (e.g. stage sequence)  */
#define LES_ERR_NO_MODEL       7  /* learned warm start requested, none set   */

/* ---- physics switches (les_config.physics) -------------------------------- */
#define LES_PHYS_ADV       (1u << 0)  /* QUICK advection, Sec. 2.4             */
#define LES_PHYS_SGS       (1u << 1)  /* Smagorinsky-Lilly nu_t, Sec. 2.3      */
#define LES_PHYS_CONST_NU  (1u << 2)  /* constant viscosity const_nu instead   */
#define LES_PHYS_MOIST     (1u << 3)  /* saturation adjustment, Sec. 2.2       */
#define LES_PHYS_BUOY      (1u << 4)  /* rho0 b k in Eq. (momentum)            */
#define LES_PHYS_CORIOLIS  (1u << 5)  /* -f k x rho0 (u - u_g)                 */
#define LES_PHYS_SPONGE    (1u << 6)  /* Rayleigh sponge near the lid, Sec 2.3 */
#define LES_PHYS_RAD       (1u << 7)  /* longwave flux divergence (theta_l)    */
#define LES_PHYS_SUBS      (1u << 8)  /* large-scale subsidence                */
#define LES_PHYS_SFC       (1u << 9)  /* surface fluxes of theta_l and q_t     */
#define LES_PHYS_FB        (1u << 10) /* stratification factor f_B in nu_t    */

/* ---- enumerations -------------------------------------------------------- */
#define LES_BC_PERIODIC    0
#define LES_BC_WALLS       1          /* free-slip surface, no-slip lid (Sec 4) */
#define LES_SOLVER_CG      0          /* conjugate gradient, FP64 dot products  */
#define LES_SOLVER_JACOBI  1          /* weighted Jacobi, the paper's solver    */
#define LES_OP_COMPACT     0          /* L_c psi = rhs - C(psi^k), App. A       */
#define LES_OP_WIDE        1          /* D(rho0 G psi) = D(rho0 u^)/dt          */
#define LES_WARM_ZERO      0
#define LES_WARM_PREV      1          /* previous step's solve, same sub-iter   */
#define LES_WARM_LEARNED   2          /* learned network (les_set_warm_model)   */
/* advection scheme (Sec. 2.4): QUICK, or third-order WENO with the local
 * Lax-Friedrichs flux (upwind-side WENO3 reconstruction; its smoothness
 * regulariser eps = 1e-6 max|phi|^2 + 1e-18 over the three values is this
 * library's reading -- the paper gives none) */
#define LES_ADV_QUICK      0
#define LES_ADV_WENO3      1
/* preconditioner of the CG solve (not in the paper) */
#define LES_PRECOND_NONE    0
#define LES_PRECOND_LEARNED 1

/* field ids for get / set / offset */
enum les_field {
  LES_U = 0, LES_V, LES_W,        /* velocity (u^{n+1} between steps)          */
  LES_P,                          /* perturbation pressure p'                  */
  LES_THETA_L, LES_QT,            /* liquid potential temperature, total water */
  LES_UN, LES_VN, LES_WN,         /* u^n during a step                         */
  LES_THETA_L_HALF, LES_QT_HALF,  /* phi^{n+1/2} during a step                 */
  LES_UHAT, LES_VHAT, LES_WHAT,   /* predicted velocity (rho0 u)^ / rho0       */
  LES_RHS,                        /* Poisson right-hand side                   */
  LES_PSI,                        /* alpha0 * dp, the Poisson unknown          */
  LES_B, LES_QL, LES_T,           /* buoyancy, liquid water, temperature       */
  LES_SRAD,                       /* radiative source of rho0 theta_l          */
  LES_NFIELD
};

/* stages of one step, for les_stage(): BEGIN, then n_subiter times
 * (SCALAR, MOMENTUM, SOLVE, CORRECT), then END (Sec. 2.4) */
enum les_stage_id {
  LES_STAGE_BEGIN = 0,   /* dt (if 0), phi^{n+1/2} thermodynamics -> T, q_l, b,
                            radiative source; u^n, phi^{n+1/2} saved; dp = 0   */
  LES_STAGE_SCALAR,      /* Eq. (scalar_prediction_step) -> phi^{k+1}          */
  LES_STAGE_MOMENTUM,    /* Eq. (momentum_prediction_step) -> u^, and the
                            Poisson right side (Eq. pressure_correction, App. A) */
  LES_STAGE_SOLVE,       /* Poisson solve for psi = alpha0 dp                  */
  LES_STAGE_CORRECT,     /* (rho0 u)^{k+1} = (rho0 u)^ - dt rho0 G psi,
                            p^{k+1} = p^k + rho0 psi                           */
  LES_STAGE_END
};

/* Configuration.  Readings of points the paper leaves open are documented
 * with the library; defaults come from les_config_default(). */
typedef struct les_config {
  uint32_t struct_size;      /* sizeof(les_config), ABI check               */
  int32_t  precision;        /* 32 or 64                                    */
  int32_t  nx, ny, nz;       /* >= 3, >= 3, >= 2                            */
  int32_t  bc_z;             /* LES_BC_PERIODIC | LES_BC_WALLS              */
  double   dx, dy, dz;       /* spacings (m)                                */
  double   dt;               /* > 0 fixed; 0 = cfl / max(|u|/dx+|v|/dy+|w|/dz)
                                from the state at the first step, then held */
  double   cfl;
  int32_t  n_subiter;        /* K sub-iterations per step (>= 1)             */
  int32_t  solver;           /* LES_SOLVER_*                                */
  int32_t  poisson_op;       /* LES_OP_*                                    */
  int32_t  warm_start;       /* LES_WARM_*                                  */
  double   poisson_tol;      /* ||b - A x||_2 <= tol ||b||_2                */
  int32_t  poisson_maxit;
  uint32_t physics;          /* LES_PHYS_* bits                             */
  double   jacobi_omega;
  double   cs, pr, sc;       /* Smagorinsky constant, Prandtl, Schmidt      */
  double   const_nu;         /* viscosity with LES_PHYS_CONST_NU (m^2/s)    */
  double   f_cor, ug, vg;    /* Coriolis parameter, geostrophic wind        */
  double   sponge_frac;      /* sponge occupies the top fraction            */
  double   sponge_rate;      /* Rayleigh rate at the lid (1/s)              */
  double   subs_div;         /* D in the subsidence speed D z (1/s)         */
  double   shf, lhf;         /* surface sensible / latent heat flux (W/m^2) */
  double   rad_f0, rad_f1;   /* longwave flux amplitudes (W/m^2)            */
  double   rad_kappa;        /* absorption coefficient (m^2/kg)             */
  double   theta0, p00;      /* reference potential temperature, pressure   */
  double   sat_tol;          /* secant stop |theta_l* - theta_l| (K)        */
  int32_t  sat_maxit;
  int32_t  solver_path;      /* 0: one persistent cooperative launch per CG
                                solve when eligible (compact operator, nx a
                                multiple of 128 floats / 64 doubles, ny a
                                multiple of the tile rows), else 1;
                                1: one launch per CG phase               */
  int32_t  advection;        /* LES_ADV_QUICK (paper's default) |
                                LES_ADV_WENO3 (its alternative, Sec. 2.4)  */
  int32_t  precond;          /* LES_PRECOND_NONE (default) |
                                LES_PRECOND_LEARNED: flexible CG with the
                                attached network (les_set_warm_model) as
                                the preconditioner, z = net(r), or z = -r
                                where r.net(r) >= 0; CG and the compact
                                operator only; not in the paper        */
  double   reserved[3];
} les_config;

typedef struct les_step_stats {
  int32_t steps;             /* steps completed by the call                 */
  int32_t solves;            /* Poisson solves                              */
  int32_t iters_total;       /* solver iterations summed over the solves    */
  int32_t iters_max;         /* most iterations in one solve                */
  int32_t not_converged;     /* solves that stopped at maxit                */
  int32_t reserved0;
  double  res_max;           /* largest final relative residual             */
  double  dt;                /* the step size in use                        */
} les_step_stats;

#define LES_NDIAG 10
/* les_diagnostics() output, all accumulated in FP64 on the device:
 * [0] sum rho0 theta_l dV   [1] sum rho0 q_t dV    [2..4] sum rho0 u_c dV
 * [5] 1/2 sum rho0 |u|^2 dV [6] max Courant number [7] max |D(rho0 u)|
 * [8] number of non-finite values in u, v, w, p, theta_l, q_t
 * [9] sum rho0 q_l dV */

typedef struct les_handle les_handle;

/* Fill *cfg with the paper's Table 1 constants and library defaults for an
 * nx*ny*nz grid.  Never fails. */
void les_config_default(les_config *cfg, int32_t nx, int32_t ny, int32_t nz);

/* Bytes of device workspace that les_init needs for *cfg (256-B aligned
 * sub-buffers).  Returns LES_ERR_INVALID_ARG for an invalid configuration. */
int les_workspace_bytes(const les_config *cfg, size_t *bytes);

/* Create a handle.  rho0_z: optional host array of nz reference densities
 * (NULL = the hydrostatic adiabatic profile of Sec. 2.1, Eqs. 2-4).
 * workspace: device pointer (>= 256-B aligned) of at least
 * les_workspace_bytes() bytes, borrowed until les_destroy.  stream: a
 * cudaStream_t or NULL.  The state starts at zero. */
int les_init(const les_config *cfg, const double *rho0_z, void *workspace,
             size_t workspace_bytes, void *stream, les_handle **out);

/* Release the handle (not the workspace).  NULL is accepted. */
void les_destroy(les_handle *h);

/* Re-target all later work to another stream. */
int les_set_stream(les_handle *h, void *stream);

/* Copy nx*ny*nz values of the handle's precision into / out of a field.
 * The fields are the prognostic and diagnostic variables of Sec. 2.1
 * (u, v, w, p', theta_l, q_t; T, q_l and b of Sec. 2.1-2.2) and the
 * intermediate arrays of the scheme of Sec. 2.4 (u^n, phi^{n+1/2}, the
 * predicted velocity, the Poisson right side and psi = alpha0 dp), in the
 * layout above.  on_device != 0: src / dst is a device pointer
 * (stream-ordered copy); otherwise a host pointer (the call synchronises the
 * stream).  LES_ERR_INVALID_ARG for a bad id or a NULL pointer. */
int les_set_state(les_handle *h, int32_t field, const void *src, int32_t on_device);
int les_get_state(les_handle *h, int32_t field, void *dst, int32_t on_device);

/* les_set_state for count fields (fields[q] from srcs[q], all on the device
 * or all on the host): every copy is enqueued before the one synchronisation
 * that host sources need, so the uploads of a whole state follow each other
 * on the copy engine.  LES_ERR_INVALID_ARG (and nothing copied) for a bad
 * id, a NULL pointer or count < 0.  The paper has no counterpart: a
 * convenience for callers that hold the state on the host. */
int les_set_states(les_handle *h, int32_t count, const int32_t *fields, const void *const *srcs,
                   int32_t on_device);

/* Upload a state for a later step without waiting: the count (1 .. 8)
 * fields are copied from host memory srcs[q] (pinned, for the copies to run
 * asynchronously) into the caller's device buffer staging (16-byte aligned,
 * count * nx * ny * nz elements, field q at element q * nx * ny * nz) on
 * copy_stream, and the call returns.  The next BEGIN stage (les_step or
 * les_stage) makes the handle's stream wait for those copies and takes the
 * staged fields as the state (a device-to-device copy), so the upload of a
 * state overlaps the steps enqueued before that BEGIN.  Up to two prefetches
 * may be pending, each with its own staging buffer; each is consumed by one
 * BEGIN, oldest first.  Before copying, copy_stream waits for the BEGIN that
 * consumed the previous prefetch, so a staging buffer can be reused for the
 * prefetch after next.  The caller keeps srcs and staging alive until the
 * consuming BEGIN has run.  LES_ERR_STATE with two prefetches pending;
 * LES_ERR_INVALID_ARG for a bad or repeated id, a NULL pointer or a
 * misaligned staging buffer.  The paper has no counterpart: the input
 * pipeline of callers that step a stream of host-held states. */
int les_prefetch_states(les_handle *h, int32_t count, const int32_t *fields, const void *const *srcs,
                        void *staging, void *copy_stream);

/* Byte offset of a field's current buffer inside the workspace (buffers of
 * the scalars and u^n rotate between steps and sub-iterations). */
int les_field_offset(les_handle *h, int32_t field, size_t *offset);

/* Advance nsteps time steps (Sec. 2.4).  stats may be NULL.  Returns
 * LES_ERR_NOT_CONVERGED if any solve stopped at maxit (the state is still
 * advanced), LES_ERR_INVALID_ARG if dt = 0 and the fluid is at rest. */
int les_step(les_handle *h, int32_t nsteps, les_step_stats *stats);

/* Run one stage of the step (enum les_stage_id) in the documented order;
 * returns LES_ERR_STATE when called out of order.  stats may be NULL. */
int les_stage(les_handle *h, int32_t stage, les_step_stats *stats);

/* Solve A x = b with the handle's operator, boundary conditions and solver:
 * the pressure-correction equation of Sec. 2.4 (Eq. pressure_correction,
 * with the compact Laplacian of Appendix A: A = L_c, LES_OP_COMPACT) or the
 * consistent operator A = D(rho0 G .) (LES_OP_WIDE); the solver is CG or the
 * weighted Jacobi iteration the paper uses (Sec. 2.4).  b's mean is removed
 * first and x is returned with zero mean.  d_rhs, d_x: device arrays
 * of nx*ny*nz values, distinct from the handle's fields; x holds the initial
 * guess on entry.  rtol > 0, maxit >= 0.  iters / rel_res may be NULL.
 * Synchronises the stream.  LES_ERR_NOT_CONVERGED if maxit was reached. */
int les_poisson_solve(les_handle *h, const void *d_rhs, void *d_x, double rtol,
                      int32_t maxit, int32_t *iters, double *rel_res);

/* y = A x for op = LES_OP_COMPACT or LES_OP_WIDE (device arrays). */
int les_apply_poisson(les_handle *h, int32_t op, const void *d_x, void *d_y);

/* FP64 diagnostics of the current state (layout above); out: host array of
 * LES_NDIAG doubles.  Synchronises the stream. */
int les_diagnostics(les_handle *h, double *out);

/* ---- allocation-free Poisson solve --------------------------------------------
 * For callers that cannot allocate device memory, and so cannot provide the
 * workspace a handle needs: a plug-in whose host application owns all device
 * memory through its own pool allocator, or a latency-bound loop that must not
 * call cudaMalloc / cudaFree because they can synchronise the whole device.
 * The paper has no counterpart; the solve is the same as les_poisson_solve()
 * (same operator, boundary conditions, solver, mean removal and stop test),
 * configured by *cfg alone (no handle).
 *
 * Scratch: one file-scope __device__ array of 16 MiB + 256.25 KiB inside
 * libles.so, held by every GPU that loads the library until the process
 * exits.  Limit: nx*ny*nz <= 524288 cells at precision 64, <= 1048576 at
 * precision 32 (four work vectors of 16 MiB in total); larger grids are
 * rejected with LES_ERR_INVALID_ARG and a message in err.  No cudaMalloc,
 * cudaFree or allocating library routine is called.
 * Every call looks up the array's address in the current device's context
 * (cudaGetSymbolAddress, no allocation), so a context torn down and created
 * again in the same process gets its own copy.  Every call on a device
 * shares the one array,
 * which keeps the previous call's contents (the call clears the control
 * block it needs zeroed): calls that overlap on the GPU race, so issue them
 * on one stream or serialise them.
 * d_rho0: device array of nz reference densities in the field precision,
 * needed only for LES_OP_WIDE (may be NULL otherwise).  d_rhs, d_x: device
 * arrays of nx*ny*nz values, x holds the initial guess on entry.  stream: a
 * cudaStream_t or NULL.  err: optional host buffer of err_len bytes for a
 * message.  Synchronises the stream.  Returns LES_OK, LES_ERR_NOT_CONVERGED,
 * LES_ERR_INVALID_ARG or LES_ERR_CUDA. */
int les_poisson_solve_static(const les_config *cfg, const void *d_rho0, const void *d_rhs, void *d_x,
                             double rtol, int32_t maxit, void *stream, int32_t *iters,
                             double *rel_res, char *err, size_t err_len);

/* ---- device measurement ---------------------------------------------------------
 * The FMA rate of the current device in precision 32 or 64: every thread of
 * four waves of resident 1024-thread blocks runs eight independent FMA
 * chains for trips x 16 steps (one warm-up launch, then one launch timed with
 * CUDA events on stream).  The FP32 rate is the ALU bound against which the
 * kernels bound by instruction issue (the predictors) are judged, the FP64
 * rate the bound of the FP64 configurations; the method does not use them.
 * trips > 0; *tflops receives 2 x FMAs / time in TFLOP/s, *ms the timed
 * launch's duration.  Allocates and frees a few kilobytes on the stream
 * (cudaMallocAsync) and synchronises it.  Returns LES_OK, LES_ERR_INVALID_ARG
 * (trips <= 0, a precision other than 32 or 64, a null output) or
 * LES_ERR_CUDA. */
int les_measure_fma(void *stream, int32_t precision, int32_t trips, double *tflops, double *ms);

/* ---- domain decomposition of the Poisson solve --------------------------------
 * The paper runs its LES on many TPU cores by cutting the domain into
 * partitions, exchanging halos before every stencil pass and reducing the
 * iterative solver's sums over all partitions (Sec. 2.5; the partitionings of
 * Sec. 4.2).  These calls do that for the pressure-correction solve (Sec. 2.4,
 * compact operator of Appendix A), the part of the step that dominates its
 * time: the global nx x ny x nz grid of *cfg (periodic in x and y) is cut into
 * px x py sub-domains of (nx / px) x (ny / py) x nz nodes (the z columns stay
 * whole, as in every partitioning the paper reports), one per rank; rank
 * (rx, ry) owns the nodes x in [rx nx/px, (rx+1) nx/px), y likewise.
 * The solve is the standard CG to ||b - A x|| <= tol ||b|| with b's global mean
 * removed and x returned with zero global mean, the same iterates as
 * les_poisson_solve up to the order of the sums.  Per iteration it calls
 * ops->exchange once (the halo of the search direction) and ops->allreduce
 * once (four FP64 sums).  The caller implements both: NCCL send / receive and
 * all-reduce between GPUs, peer copies, or in-process copies between
 * sub-domains on one device. */
typedef struct les_dd les_dd;
typedef struct les_dd_ops {
  void *ctx;  /* passed back to both functions */
  /* Send the four face strips send[f] (device buffers of bytes[f] bytes;
   * f = 0 west: the nodes x = x0, 1 east: x = x0 + nx/px - 1, 2 south:
   * y = y0, 3 north: y = y0 + ny/py - 1; each strip ordered with the
   * in-face index fastest, then z) to the neighbour on that side, and receive
   * the neighbours' opposite strips into recv[f] (recv[0] from the west
   * neighbour's east strip, and so on; periodic neighbours wrap).  A strip
   * of 0 bytes is neither sent nor received (les_dd_halo_exchange moves the
   * x strips and the y strips in two calls; its strips are LES_DD_HALO nodes
   * deep and hold several fields, packed as the library unpacks them; every
   * rank passes the same sizes).  Called with the work enqueued on `stream`;
   * on return recv must hold the data for work later enqueued on that
   * stream.  Return 0 on success. */
  int (*exchange)(void *ctx, void *const *send, void *const *recv, const size_t *bytes, void *stream);
  /* Replace each of the n host doubles by its sum over all ranks; return 0
   * on success. */
  int (*allreduce)(void *ctx, double *values, int32_t n);
} les_dd_ops;
/* Device workspace of one sub-domain (its CG vectors with a one-node halo,
 * their face strips, the partial sums, and the strips of the decomposed
 * step's field halos: LES_DD_MAX_FIELDS fields, LES_DD_HALO deep).  LES_ERR_INVALID_ARG unless px divides
 * nx, py divides ny, nz >= 2 and the precision is 32 or 64. */
int les_dd_workspace_bytes(const les_config *cfg, int32_t px, int32_t py, size_t *bytes);
/* Sub-domain (rx, ry) of a px x py partition of *cfg's grid; the workspace
 * (>= 256-B aligned) is borrowed until les_dd_destroy; work runs on stream.
 * Only the compact operator (LES_OP_COMPACT) is decomposed. */
int les_dd_create(const les_config *cfg, int32_t px, int32_t py, int32_t rx, int32_t ry, void *workspace,
                  size_t workspace_bytes, void *stream, les_dd **out);
void les_dd_destroy(les_dd *d);
/* The local interior size and its global offset (any pointer may be NULL). */
int les_dd_local_shape(const les_dd *d, int32_t *nx, int32_t *ny, int32_t *nz, int32_t *x0, int32_t *y0);
/* Solve on this rank's part: d_rhs, d_x device arrays of the local interior
 * ((nx/px) x (ny/py) x nz, x fastest), d_x holds the rank's part of the
 * initial guess.  Every rank of the partition must call it with the same
 * rtol and maxit.  Synchronises the stream.  Returns LES_OK,
 * LES_ERR_NOT_CONVERGED, LES_ERR_NONFINITE (CG breakdown), LES_ERR_CUDA (a
 * CUDA call or a callback failed) or LES_ERR_INVALID_ARG. */
int les_dd_poisson_solve(les_dd *d, const les_dd_ops *ops, const void *d_rhs, void *d_x, double rtol,
                         int32_t maxit, int32_t *iters, double *rel_res);
const char *les_dd_last_error(const les_dd *d);

/* ---- the decomposed step ---------------------------------------------------
 * The whole step (Sec. 2.4: thermodynamics, the scalar and momentum
 * predictors, the Poisson solve and the correction) on one sub-domain of the
 * partition above, the paper's parallel LES (Sec. 2.5), with halo exchanges
 * before the stencil passes and the solver's sums reduced over all ranks.
 * The sub-domain's fields live in an ordinary handle (les_init with the
 * configuration from les_dd_step_config) whose grid is the sub-domain widened
 * by LES_DD_HALO = 2 nodes on each side in x and y, (nx/px + 4) x (ny/py + 4)
 * x nz: its node (i, j, k) is global node (x0 + i - 2, y0 + j - 2, k),
 * wrapped periodically.  The handle's stencil stages run on that grid as on a
 * periodic domain.  No stencil of the step reaches further than two nodes
 * along x or y (the upwind-biased QUICK face value, the Smagorinsky stress
 * with nu_t at the neighbouring nodes, the App. A term of the right side), so
 * with fresh halos the owned nodes get the values of the undivided domain,
 * bit for bit, and the halo nodes' values are discarded.  One step is
 *     exchange u v w p theta_l q_t;  BEGIN;
 *     for each sub-iteration k:  (k > 0: exchange u v w theta_l q_t);
 *         SCALAR;  MOMENTUM;  exchange u^ v^;  les_dd_stage_solve;
 *         exchange psi;  CORRECT;
 *     END
 * with BEGIN ... CORRECT, END by les_stage (the driver is
 * paper_2301_04698_gb300.decomp.decomposed_step).  The time step must be fixed
 * (cfg.dt > 0, or les_set_dt) and the same on every rank.  Diagnostics of
 * the widened handle (les_diagnostics) include its halo nodes. */
#define LES_DD_HALO 2
#define LES_DD_MAX_FIELDS 8
/* *out = the global configuration of d with nx, ny of the widened sub-domain. */
int les_dd_step_config(const les_dd *d, les_config *out);
/* Fill the LES_DD_HALO-deep x and y halos of nfields (1 .. LES_DD_MAX_FIELDS)
 * fields of the widened handle h (ids as les_get_state: LES_U, LES_THETA_L
 * (the current buffer), LES_UHAT, LES_PSI, ...) from the neighbours' owned
 * nodes: ops->exchange is called twice, first with the west and east strips
 * (the owned rows), then with the south and north strips over the whole
 * widened width, which carries the corner nodes.  Runs on h's stream.
 * LES_ERR_INVALID_ARG if h's grid is not d's widened sub-domain, a field id
 * is bad or repeated, or nfields is out of range; LES_ERR_CUDA if a launch or
 * the callback fails. */
int les_dd_halo_exchange(les_dd *d, les_handle *h, const les_dd_ops *ops, int32_t nfields, const int32_t *fields);
/* The SOLVE stage of the widened handle h (in les_stage's order, in place of
 * les_stage(h, LES_STAGE_SOLVE)), over the partition: the Poisson right side
 * (Eq. pressure_correction with App. A) is formed again from h's u^ (its halo
 * exchanged) and psi, the solve runs on the owned nodes by the decomposed CG
 * above from h's first guess (LES_WARM_ZERO or LES_WARM_PREV), and psi's owned
 * nodes receive the solution (its halo is stale until exchanged).  Every rank
 * calls it with the same configuration.  Returns as les_stage's solve stage
 * (LES_OK, LES_ERR_NOT_CONVERGED, ...); LES_ERR_STATE out of order;
 * LES_ERR_INVALID_ARG for a handle that is not d's widened sub-domain or asks
 * for the learned warm start or preconditioner. */
int les_dd_stage_solve(les_dd *d, les_handle *h, const les_dd_ops *ops, les_step_stats *stats);

/* ---- ensembles -----------------------------------------------------------------
 * Independent members -- different grids, seeds and forcings, as in ensembles
 * of LES runs that produce parameterisation training data -- stepped
 * together.  les_ensemble_step runs les_step(hs[i], nsteps, &stats[i]) for
 * the m distinct handles concurrently, one host thread per handle, each on its
 * own device and stream (give every handle its own stream, les_set_stream,
 * for the members' kernels to overlap).  The members' stencil kernels
 * overlap freely.  Their persistent CG solves share the device's SMs: a
 * member whose les_tuning.cg_max_blocks caps its solve at B blocks (B at
 * most the SM count) holds B SMs while the solve runs, an uncapped member
 * all of them; so members capped at a share of the SMs solve together, and
 * uncapped ones one at a time (the blocks of a persistent solve must all be
 * resident at once).  stats: optional array
 * of m; failed: optional, the index of the first member whose status is
 * returned (-1 if none).  Returns LES_OK, LES_ERR_NOT_CONVERGED (state valid)
 * or the first other error; LES_ERR_INVALID_ARG for m <= 0, m > 1024, a null
 * or repeated handle.  The paper runs one domain at a time and has no
 * counterpart. */
int les_ensemble_step(les_handle *const *hs, int32_t m, int32_t nsteps, les_step_stats *stats,
                      int32_t *failed);

/* ---- tuning of the persistent CG solve ---------------------------------------
 * The CG solve runs as one persistent cooperative launch when solver_path = 0
 * (compact operator).  For cg_variant 2 a thread block of
 * 32 x cg_tile_rows threads owns a tile of (32 * 16 B of cells) x
 * cg_tile_rows x cg_tile_planes nodes; every grid is capped by occupancy and
 * cg_max_blocks.  Each grid-barrier wait ends
 * after barrier_timeout_ms; the solve then returns LES_ERR_TIMEOUT and the
 * device stays usable.  fault_missing_arrivals is a failure-detection test
 * hook: the barrier then waits for that many blocks that never arrive, so
 * every wait runs out (in the register CG, every wait of its iterations; its
 * set-up sums wait for the launched blocks only); it must be 0 otherwise.  stencil_path selects the
 * stencil kernels (same results to rounding; both compute nu_t in place):
 * 0 (default) column marches where the grid allows them -- the correction
 * and the Poisson right side over 16-byte lanes (nx a multiple of 128 floats
 * / 64 doubles), the scalar and momentum predictors over two-node lanes (nx
 * a multiple of 64), ny a multiple of 8 -- and rolling z-marches elsewhere;
 * 1 rolling z-marches through shared-memory plane rings everywhere.  With
 * cg_resident = 0 or 2 the standard CG solve first tries a decomposition of
 * the grid into one brick per thread block (x extent 32, 64 or 128 dividing
 * nx, y and z extents dividing ny and nz, at most one block per SM, x, r and
 * p of a brick within the per-block shared memory; with cg_resident = 0 and
 * an FP32 grid 128 nodes wide, bricks of the whole x extent with at most six
 * planes per thread and p, r and q in registers); the blocks then exchange
 * only brick faces through global memory, and cg_tile_rows and
 * cg_tile_planes do not apply.  A zero field in a set call keeps the
 * current value (except fault_missing_arrivals, stencil_path, cg_variant and
 * cg_resident, which are always taken). */
typedef struct les_tuning {
  uint32_t struct_size;            /* sizeof(les_tuning)                   */
  int32_t  cg_tile_rows;           /* 1, 2, 4 or 8                          */
  int32_t  cg_tile_planes;         /* >= 1                                  */
  int32_t  cg_max_blocks;          /* >= 1                                  */
  double   barrier_timeout_ms;     /* > 0                                   */
  int32_t  fault_missing_arrivals; /* 0 in production                      */
  int32_t  stencil_path;           /* 0 columns (default), 1 rolling      */
  int32_t  cg_variant;             /* persistent CG: 0 (default) the
                                      standard CG iterates -- in shared
                                      memory when the grid fits there (see
                                      cg_resident), else variant 4 for
                                      FP32 grids of whole columns,
                                      else variant 2 on tile-aligned grids,
                                      else variant 3; 1 is not accepted;
                                      2 the
                                      two-phase streaming CG (two barriers
                                      per iteration); 3 one pass over memory
                                      and one grid reduction per iteration,
                                      any grid; 4 the same in 64 x 16 or
                                      32 x 32 columns with the z neighbours
                                      in registers (nx a multiple of 64 and
                                      ny of 16, or both of 32; else as 3).  2 needs nx a
                                      multiple of 128 (FP32) / 64 (FP64)
                                      and ny of cg_tile_rows, else the
                                      per-phase launches run               */
  int32_t  cg_resident;            /* 0 (default): standard CG keeps its
                                      vectors on chip when the grid fits
                                      there (FP32 grids with nx = 128: p, r
                                      and q in registers, x and a copy of p
                                      in shared memory; else all in shared
                                      memory); 1: always streams them
                                      through global memory; 2: on chip with
                                      every vector in shared memory        */
} les_tuning;
int les_get_tuning(les_handle *h, les_tuning *out);
int les_set_tuning(les_handle *h, const les_tuning *in);

/* ---- learned Poisson warm start (not in the paper) ---------------------------
 * A 3-level 3-D U-Net with periodic padding predicts the first guess psi_0 of
 * the pressure-correction solve from its right-hand side b (Sec. 2.4 defines
 * the solve; the network is this library's addition):
 *   x0 = b / s, s = rms(b); e1 = B(x0; 1->16); e2 = B(pool e1; 16->32);
 *   e3 = B(pool e2; 32->64); g2 = B([up e3, e2]; 96->32);
 *   g1 = B([up g2, e1]; 48->16); y = conv1x1(g1; 16->1); psi_0 = s (y - mean y)
 * B(.; a->c): two 3x3x3 convolutions, each followed by a leaky ReLU (0.1);
 * pool: 2x2x2 mean; up: nearest doubling; [.,.]: channel concatenation.
 * BF16 weights and activations, FP32 accumulation (tensor cores), FP32
 * master weights and Adam.  The grid is cubic, n a multiple of 4 (>= 8).
 * Weights are one flat FP32 vector of les_unet_param_count() values, layer by
 * layer (enc1a, enc1b, enc2a, enc2b, enc3a, enc3b, dec2a, dec2b, dec1a,
 * dec1b, head), each W[cout][cin][kz][ky][kx] followed by bias[cout].
 * The model borrows a caller-allocated device workspace like the solver.
 * b / psi arrays: device, batch * n^3 values of the given precision (32/64),
 * one sample after another, x fastest.  The output is scaled as
 * psi_0 = s * out_scale * (y - mean y) and the training target is
 * psi / (s * out_scale); out_scale (default 1) should be the typical ratio
 * rms(psi) / rms(b) of the data so that the network works at unit scale. */
typedef struct les_unet les_unet;
int64_t les_unet_param_count(void);
int les_unet_workspace_bytes(int32_t n, int32_t max_batch, size_t *bytes);
int les_unet_create(int32_t n, int32_t max_batch, void *workspace, size_t workspace_bytes, void *stream,
                    les_unet **out);
void les_unet_destroy(les_unet *u);
int les_unet_set_stream(les_unet *u, void *stream);
/* load / read the FP32 master weights (resets the Adam moments on load) */
int les_unet_set_weights(les_unet *u, const float *w, int32_t on_device);
int les_unet_get_weights(les_unet *u, float *w, int32_t on_device);
/* psi_0 for each of `batch` right-hand sides */
int les_unet_forward(les_unet *u, int32_t precision, const void *d_b, int32_t batch, void *d_psi0);
/* mean squared error of the network output against psi / s and its gradient
 * with respect to every weight (d_grad: device FP32, may be NULL); *loss on
 * the host (may be NULL; synchronises the stream when given) */
int les_unet_loss_grad(les_unet *u, int32_t precision, const void *d_b, const void *d_psi, int32_t batch,
                       double *loss, float *d_grad);
/* Training loss of les_unet_loss_grad / les_unet_train_step (default MSE):
 * LES_UNET_LOSS_MSE     mean of d^2,
 * LES_UNET_LOSS_ENERGY  sum of d (-Delta d) / count, -Delta the 7-point negative
 *                       Laplacian with unit spacing on the periodic grid: the
 *                       energy norm of the error, which weights each Fourier
 *                       mode by the operator's eigenvalue as a CG solve from
 *                       the guess does, and ignores the constant,
 * with d = y - psi / (s out_scale) per sample.  LES_ERR_INVALID_ARG for another
 * kind.  Not in the paper (the learned warm start is this library's). */
#define LES_UNET_LOSS_MSE     0
#define LES_UNET_LOSS_ENERGY  1
int les_unet_set_loss(les_unet *u, int32_t kind);
/* loss_grad followed by one Adam step (beta1 0.9, beta2 0.999, eps 1e-8) */
int les_unet_train_step(les_unet *u, int32_t precision, const void *d_b, const void *d_psi, int32_t batch,
                        float lr, double *loss);
int les_unet_set_output_scale(les_unet *u, double out_scale);
double les_unet_get_output_scale(const les_unet *u);
const char *les_unet_last_error(const les_unet *u);
/* Attach a model to a solver handle for LES_WARM_LEARNED (NULL detaches).
 * The model's grid must equal the handle's (nx = ny = nz = n); the handle
 * borrows the model until detached or destroyed.  The plain solver is the
 * fallback and the arbiter: if the model fails, or its guess leaves a larger
 * residual than a zero guess (||b - A psi_0|| > ||b||), the solve starts
 * from zero; every solve still iterates to the same relative residual. */
int les_set_warm_model(les_handle *h, les_unet *u);

/* ---- launch accounting and event profiling -------------------------------- */
#define LES_MAX_KERNELS 32
typedef struct les_kernel_stat {
  char    name[24];          /* kernel class, e.g. "cg_matvec"                     */
  int32_t fields_per_cell;   /* algorithmic fields read + written per launch/cell  */
  int32_t reserved0;
  int64_t launches;          /* launches since the last reset                      */
  int64_t timed;             /* launches bracketed by events (profiling enabled)   */
  double  total_ms;          /* summed event time of the timed launches            */
  double  bytes_per_launch;  /* fields_per_cell * nx*ny*nz * sizeof(element)       */
} les_kernel_stat;

/* Enable (1) / disable (0) CUDA-event timing of every kernel launch on the
 * handle's stream (adds two event records per launch).  Launches are always
 * counted. */
int les_profile_enable(les_handle *h, int32_t enable);
/* Copy up to max_entries kernel classes with at least one launch into out
 * (host array); *count receives the number written.  Synchronises on the
 * last recorded event. */
int les_profile_read(les_handle *h, les_kernel_stat *out, int32_t max_entries, int32_t *count);
/* Zero the launch counts and timings. */
int les_profile_reset(les_handle *h);
/* Total kernel launches issued by the handle since creation or reset. */
int64_t les_launch_count(const les_handle *h);

/* The step size (0 until fixed by the first step when cfg.dt == 0). */
double les_get_dt(const les_handle *h);
int    les_set_dt(les_handle *h, double dt);

/* Message of the last failed call on h (static string if h is NULL). */
const char *les_last_error(const les_handle *h);
const char *les_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* LES_H */
