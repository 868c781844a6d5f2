/*
 * rf.h -- C ABI of the GB300 (sm_103a) Richards-equation solver.
 *
 * The library solves the 3-D transient Richards equation in pressure-head
 * form (Orgogozo et al., arXiv:1809.10895, Eq. 1; z upward, h in m) with van
 * Genuchten / Mualem closures (Eq. 2-4) on a structured grid of equal cells,
 * by the scheme of Sec. 2.2: backward Euler in time, classical Picard
 * linearisation with a chord-slope capacity, implicit pressure Laplacian with
 * linearly interpolated face conductivity, explicit gravity lagged one Picard
 * iterate, a preconditioned conjugate-gradient linear solve, a global
 * max|dh| Picard exit test (Sec. 2.3) and EBATS adaptive time stepping.
 *
 * Conventions
 *   - SI units.  h: pressure head [m]; fluxes [m/s]; times [s].
 *   - Cells are indexed p = i + nx*(j + ny*k), x fastest, z slowest; cell
 *     (i,j,k) has its centre at z_bottom + (k + 1/2) dz.
 *   - Host arrays passed in are borrowed for the duration of the call and
 *     copied; device arrays ("d_" arguments) are CUDA device pointers on the
 *     context's device and must hold the stated number of elements.
 *   - Every call returns rf_status.  No exception crosses the ABI.  On an
 *     error the context state is unchanged (a step is all-or-nothing) and
 *     rf_last_error() returns a message for the calling thread.
 *   - There is no CPU fallback: without an sm_103 GPU, rf_mesh_create returns
 *     RF_ERR_NO_DEVICE.
 *   - A context is used by one host thread at a time; its work is ordered on
 *     the CUDA stream given at creation.
 */
#ifndef RF_H
#define RF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rf_ctx rf_ctx;

typedef enum rf_status {
    RF_OK = 0,
    RF_ERR_ARG = 1,            /* invalid argument                                  */
    RF_ERR_NO_DEVICE = 2,      /* no sm_103 GPU visible: there is no CPU fallback    */
    RF_ERR_CUDA = 3,           /* a CUDA runtime call failed                         */
    RF_ERR_NOMEM = 4,          /* device allocation failed                           */
    RF_ERR_STATE = 5,          /* call order (e.g. rf_step before rf_state_set)      */
    RF_ERR_PICARD = 6,         /* Picard did not converge (internal; EBATS reruns)   */
    RF_ERR_DT_MIN = 7,         /* EBATS shrank dt below dt_min without convergence   */
    RF_ERR_CG = 8,             /* CG non-finite / max_it where it is fatal            */
    RF_ERR_DEVICE_TIMEOUT = 9  /* a bounded device loop exhausted its budget          */
} rf_status;

/* Soil models: van Genuchten / Mualem (Eq. 2-4), Gardner (Eq. A6, a test
 * model) and Brooks-Corey (the alternative closure Sec. 1 names: air-entry
 * head -1/alpha, pore-size index n > 0, Se = (h_b/h)^n below h_b, K = Ks
 * Se^((2 + 3n)/n)). */
typedef enum rf_soil_model { RF_VG = 0, RF_GARDNER = 1, RF_BROOKS_COREY = 2 } rf_soil_model;

/* Boundary conditions.  RF_BC_FLUX: imposed total Darcy flux, m/s, positive
 * into the domain (the time-varying Neumann condition of Sec. 3.2).
 * RF_BC_FREE_DRAINAGE: unit hydraulic gradient (zero pressure gradient),
 * bottom face only.  RF_BC_SEEPAGE: Dirichlet h = 0 while the adjacent cell is
 * saturated at the start of the step, zero flux otherwise. */
typedef enum rf_bc_type {
    RF_BC_ZERO_FLUX = 0, RF_BC_DIRICHLET = 1, RF_BC_FLUX = 2,
    RF_BC_FREE_DRAINAGE = 3, RF_BC_SEEPAGE = 4
} rf_bc_type;

/* Face classes.  RF_ZMAX is the top face of the topmost active cell of each
 * column (the land surface of a masked grid); RF_ZMIN the bottom face of the
 * lowest active cell.  Lateral faces touching an inactive cell are zero-flux. */
typedef enum rf_face { RF_XMIN = 0, RF_XMAX, RF_YMIN, RF_YMAX, RF_ZMIN, RF_ZMAX } rf_face;

/* Arithmetic of the linear solve (Sec. 2.2's PCG).  FP64: the plain path,
 * an FP64 PCG on the FP64 operator.  MIXED: an FP32 inner PCG inside FP64
 * defect correction; the operator is assembled in FP64 and the outer
 * residual, the Picard test and the mass balance stay FP64.  The closures
 * follow closure_arith (below). */
typedef enum rf_precision {
    RF_PREC_FP64 = 0,
    RF_PREC_MIXED = 1
} rf_precision;

/* Arithmetic of the closures (Eq. 2-4).  AUTO: FP64 on the RF_PREC_FP64
 * path, double-float on the RF_PREC_MIXED path.  FP64: CUDA's FP64 log and
 * exp.  DOUBLE_FLOAT: pairs of FP32 values (about 48 significant bits: theta*
 * within 1.2e-14 relative, K and C within 2.4e-13), several times faster on
 * GB300, whose FP64 pipe is narrow.  Storage, the chord difference, the
 * operator, the Picard test and the balance are FP64 either way. */
typedef enum rf_closure_arith {
    RF_CLOSURE_AUTO = 0, RF_CLOSURE_FP64 = 1, RF_CLOSURE_DOUBLE_FLOAT = 2
} rf_closure_arith;

/* Interface conductivity of an interior face.  ARITHMETIC: (K_P + K_N)/2,
 * the linear interpolation of Sec. 2.2 (the default).  HARMONIC: 2 K_P K_N /
 * (K_P + K_N), the series conductance of two half cells (the interpolation
 * alternative of Sec. 2.2; RF_PREC_FP64 only).  The same Kbar enters the
 * Laplacian and the explicit gravity term. */
typedef enum rf_face_mean { RF_FACE_ARITHMETIC = 0, RF_FACE_HARMONIC = 1 } rf_face_mean;

/* Time discretisation (Sec. 2.2).  BACKWARD_EULER: the paper's scheme.  BDF2:
 * variable-step second-order backward differentiation in the mixed form,
 * V/dt [a0 theta^{n+1} - a1 theta^n + a2 theta^{n-1}] with w = dt/dt_prev,
 * a0 = (1+2w)/(1+w), a1 = 1+w, a2 = w^2/(1+w) (the multistep alternative
 * Sec. 2.2 names); needs picard_form MODIFIED and time_control EBATS; the
 * first step after a state is set is backward Euler. */
typedef enum rf_time_scheme { RF_TIME_BACKWARD_EULER = 0, RF_TIME_BDF2 = 1 } rf_time_scheme;

/* Step-size control (Sec. 2.2).  EBATS: the paper's controller (below).
 * RICHARDSON: step doubling, the alternative Sec. 2.2 names for prescribing
 * the temporal error: each step is taken once with dt and twice with dt/2
 * from the same state; the step is accepted, with the two-half-step result,
 * when max |h(2 x dt/2) - h(dt)| <= tol_time; either way the next dt is
 * dt 0.9 sqrt(tol_time / err) clamped to [0.2, 2] dt and to dt_max; a Picard
 * failure divides dt by f_shrink as in EBATS. */
typedef enum rf_time_control { RF_TIME_EBATS = 0, RF_TIME_RICHARDSON = 1 } rf_time_control;

/* Preconditioner of the inner PCG.  MG, DIC and ZLINE need RF_PREC_MIXED.
 * DIC is the diagonal incomplete Cholesky preconditioner Sec. 2.2 solves
 * with, the cells eliminated in red-black order (colour (i + j + k) mod 2) so
 * that its sweeps are data-parallel.  ZLINE (no counterpart in the paper;
 * ensemble only, rf_mesh_create and rf_set_params refuse it) is the operator
 * without its horizontal faces -- per column the tridiagonal matrix of the
 * storage term and the vertical faces -- solved exactly per column; it is
 * exact on residuals that are uniform across the columns, the vertical flow
 * of the ensemble's instances. */
typedef enum rf_precond {
    RF_PRECOND_JACOBI = 0,
    RF_PRECOND_MG = 1,
    RF_PRECOND_DIC = 2,
    RF_PRECOND_ZLINE = 3
} rf_precond;

/* Solver parameters (Sec. 2.2 leaves their values to the user).
 *   tol_picard  Picard exit test: max over active cells |h^{k+1} - h^k| <= tol [m]
 *   tol_cg      PCG stop: ||b - A x||_2 <= tol_cg ||b||_2
 *   cg_max_it   PCG iteration cap (hitting it rejects the step)
 *   dt0, dt_max, dt_min  EBATS initial / maximum / minimum step [s]
 *   f_grow, f_shrink     EBATS factors; n_inc consecutive accepted steps with
 *                        <= n_small Picard iterations grow dt; more than n_max
 *                        Picard iterations (or any failure) reject the step
 *   eps_chord   chord slope is replaced by dtheta/dh when |h^k - h^n| <= eps
 *   tol_inner, inner_max_it, outer_max_it   mixed precision inner FP32 PCG
 *               relative tolerance and caps                               */
/* Picard linearisation (Sec. 2.2).  CHORD: the classical Picard iteration
 * with the chord slope of theta* between h^n and h^k as capacity (the
 * paper's scheme).  MODIFIED: the mass-conservative modified Picard
 * iteration the paper also implements (the mixed form of Celia et al. 1990):
 * capacity C(h^k), storage V [theta*(h^k) + C(h^k)(h^{k+1} - h^k) -
 * theta*(h^n)] / dt.  Both converge to the same backward-Euler solution.
 * The batched ensemble supports CHORD only. */
typedef enum { RF_PICARD_CHORD = 0, RF_PICARD_MODIFIED = 1 } rf_picard_form;

typedef struct rf_solver_params {
    double tol_picard, tol_cg;
    int cg_max_it;
    int precond;      /* rf_precond   */
    int precision;    /* rf_precision */
    double dt0, dt_max, dt_min, f_grow, f_shrink;
    int n_inc, n_small, n_max;
    double eps_chord;
    double tol_inner;
    int inner_max_it, outer_max_it;
    int picard_form;    /* rf_picard_form   */
    int closure_arith;  /* rf_closure_arith */
    int face_mean;      /* rf_face_mean     */
    int time_scheme;    /* rf_time_scheme   */
    int time_control;   /* rf_time_control  */
    double tol_time;    /* Richardson control: bound on max |h(2 x dt/2) - h(dt)| per step [m] */
    double grav[3];     /* gradient of elevation along the grid's x, y, z axes: (0, 0, 1) for a
                           z-up grid; for a grid aligned with a tilted slab (Sec. 4.2), Eq. 1's
                           gravity term along each axis.  Gravity flux of a face = grad(elevation)
                           . n_out times Kbar A; free drainage follows it */
} rf_solver_params;

/* Fill *p with the defaults: tol_picard 1e-6, tol_cg 1e-10, cg_max_it 10000,
 * Jacobi, FP64, dt0 1, dt_max 600, dt_min 1e-3, f 1.3/1.3, n_inc 10, n_small 3,
 * n_max 8, eps_chord 1e-10, tol_inner 1e-4, inner_max_it 2000, outer_max_it 30,
 * classical (chord) Picard, AUTO closures, arithmetic face mean, backward
 * Euler under EBATS, tol_time 1e-3, grav (0, 0, 1). */
void rf_default_params(rf_solver_params *p);

/* Structured mesh of equal cells (the paper's solver requires a constant cell
 * volume, Restrictions paragraph).  active: nx*ny*nz bytes, nonzero = active,
 * NULL = all active. */
typedef struct rf_mesh_desc {
    int nx, ny, nz;
    double dx, dy, dz, z_bottom;
    const uint8_t *active;
} rf_mesh_desc;

/* Optional device-memory allocator.  When NULL the library uses cudaMalloc /
 * cudaFree.  alloc must return a device pointer aligned to 256 bytes or NULL. */
typedef struct rf_allocator {
    void *(*alloc)(size_t bytes, void *user);
    void (*free)(void *ptr, void *user);
    void *user;
} rf_allocator;

/* Create a context for a mesh on the current CUDA device; cuda_stream is a
 * cudaStream_t (NULL = the legacy default stream).  All device memory is
 * allocated here (through alloc when given) and released by rf_destroy.
 * The mesh and params are checked before the device is queried: a bad value
 * returns RF_ERR_ARG; no sm_103 device returns RF_ERR_NO_DEVICE (there is no
 * CPU fallback).  *out is NULL on every error. */
rf_status rf_mesh_create(const rf_mesh_desc *mesh, const rf_solver_params *params, void *cuda_stream,
                         const rf_allocator *alloc, rf_ctx **out);
void rf_destroy(rf_ctx *ctx);
rf_status rf_set_params(rf_ctx *ctx, const rf_solver_params *params);

/* Soil parameters per zone (Eq. 2-4 symbols; S is the storativity for h >= 0,
 * which the paper names but does not value).  zone_of_cell: N bytes or NULL
 * (all zone 0).  Ks_cell: N doubles overriding each cell's Ks, or NULL. */
typedef struct rf_soil {
    int model;   /* rf_soil_model */
    double theta_r, theta_s, alpha, n, Ks, S;
} rf_soil;
rf_status rf_soil_set(rf_ctx *ctx, const rf_soil *zones, int n_zones, const uint8_t *zone_of_cell,
                      const double *Ks_cell);

/* Boundary condition of a face class: a piecewise-constant series, v[i] on
 * [t[i], t[i+1]) (v[0] before t[0], v[n-1] after t[n-1]); t strictly
 * increasing; n = 1 for a constant; t may be NULL when n = 1.  Steps are
 * clipped to the series breakpoints so each step sees one value.  ZERO_FLUX,
 * FREE_DRAINAGE and SEEPAGE take no series (n = 0). */
rf_status rf_bc_set(rf_ctx *ctx, rf_face face, rf_bc_type type, const double *t, const double *v, int n);

/* Set the state h (N doubles, inactive entries are kept as given) at time t:
 * the pressure head of Eq. 1 at every cell centre.  Resets EBATS (dt = dt0,
 * Sec. 2.2), the BDF2 history and the mass balance (storage0 = sum of V
 * theta*(h) over active cells).  Non-finite heads on active cells return
 * RF_ERR_ARG; RF_ERR_STATE before rf_soil_set. */
rf_status rf_state_set(rf_ctx *ctx, const double *h, double t);
rf_status rf_state_set_device(rf_ctx *ctx, const double *d_h, double t);

typedef struct rf_state_meta {
    double t, dt_nom;
    int easy;          /* EBATS consecutive-easy-step counter */
    int n_active;
    long long steps;   /* accepted steps since rf_state_set   */
} rf_state_meta;
/* Read the state: h (host, N doubles, or NULL) and the time-stepping
 * counters (t, EBATS dt_nom and easy-step counter of Sec. 2.2, active cells,
 * accepted steps).  The device variant copies h into d_h (device, N). */
rf_status rf_state_get(rf_ctx *ctx, double *h, rf_state_meta *meta);
rf_status rf_state_get_device(rf_ctx *ctx, double *d_h);

/* Restore EBATS and mass-balance counters (checkpoint / resume): meta's t,
 * dt_nom, easy and steps; mass7 (NULL to keep them) holds the seven values of
 * rf_mass_balance_t in order, of which storage0, inflow_cum, outflow_cum,
 * closure_abs (as a signed sum) and nonlinear_defect_cum are restored.
 * RF_ERR_STATE before a state is set.  A run resumed this way is
 * bit-identical to an uninterrupted one. */
rf_status rf_state_meta_set(rf_ctx *ctx, const rf_state_meta *meta, const double *mass7);

typedef struct rf_step_info {
    double dt, t;          /* accepted step size and the time reached             */
    int picard_iters;      /* Picard iterations (linear solves) of the accepted try */
    int cg_iters;          /* CG iterations over all tries of this step            */
    int rejected;          /* EBATS reruns before acceptance                        */
    double max_dh;         /* last Picard update max|h^{k+1} - h^k|                 */
} rf_step_info;

/* One accepted time step of Sec. 2.2: Picard iterations from h^{n+1,0} = h^n
 * (closures of Eq. 2-4, chord-slope capacity, assembly, PCG solve, the
 * global max|dh| exit test of Sec. 2.3) until the test passes; a step that
 * needs more than n_max iterations, or whose solve fails, is rerun from h^n
 * with dt / f_shrink (EBATS, Sec. 2.2; or Richardson control, above).  The
 * step is clipped to the next boundary-series breakpoint.  out (may be NULL)
 * receives its record.  RF_ERR_DT_MIN when dt falls below dt_min; on any
 * error the state is unchanged. */
rf_status rf_step(rf_ctx *ctx, rf_step_info *out);

typedef struct rf_run_stats {
    long long steps, picard_iters, cg_iters, rejected;
} rf_run_stats;

/* Advance to t_end by repeated rf_step (Sec. 2.2), the last step clipped to
 * t_end.  stats (may be NULL): steps, Picard and CG iterations, reruns.
 * log: up to log_cap step records, or NULL.  Stops at the first failing
 * step, whose error it returns; the steps before it stay taken. */
rf_status rf_run(rf_ctx *ctx, double t_end, rf_run_stats *stats, rf_step_info *log, int log_cap);

/* Global water balance since rf_state_set (volumes, m^3).  The paper takes
 * the chord slope of Sec. 2.2 for its mass conservation but defines no
 * balance; this one is: storage = sum of V theta*(h) over active cells;
 * inflow_cum / outflow_cum sum dt times the boundary fluxes of each accepted
 * step's last linear system, split per face by sign.  closure_abs is
 * |sum over steps of [sum_P V C^k (h^{n+1}-h^n) - dt Q_boundary]| of each
 * accepted step's last linear system; closure_rel divides it by storage0 +
 * inflow_cum + outflow_cum.  nonlinear_defect_cum is sum of [storage change -
 * dt Q_boundary], bounded by the Picard tolerance. */
typedef struct rf_mass_balance_t {
    double storage0, storage, inflow_cum, outflow_cum, closure_abs, closure_rel, nonlinear_defect_cum;
} rf_mass_balance_t;
rf_status rf_mass_balance(rf_ctx *ctx, rf_mass_balance_t *out);

/* Message of the last failed call on this thread ("" if none). */
const char *rf_last_error(void);

/* ---- kernel-level entry points (device pointers, N doubles each) ------- */

/* Evaluate the closures at d_hk and assemble the Picard system at
 * (h^k = d_hk, h^n = d_hn, dt, t) into the context's operator; optionally
 * copy K(h^k), theta*(h^k), c = V C^k/dt, b and diag(A) out (NULL to skip).
 * Inactive entries are written as 0. */
rf_status rf_assemble(rf_ctx *ctx, const double *d_hk, const double *d_hn, double dt, double t,
                      double *d_K, double *d_theta, double *d_c, double *d_b, double *d_diag);

/* d_y = A d_x with the last assembled operator (FP64). */
rf_status rf_apply(rf_ctx *ctx, const double *d_x, double *d_y);

/* Solve the last assembled system with the context's precision and
 * preconditioner; d_x holds x0 on entry and the solution on return.
 * *iters: CG iterations (FP64) or inner FP32 iterations summed (mixed). */
rf_status rf_solve(rf_ctx *ctx, double *d_x, int *iters);

/* The stencil step of the FP32 inner PCG of the mixed path (Sec. 2.2's PCG
 * run in FP32, the kernel its iterations launch: TMA-staged planes when nx
 * is a multiple of 4, plain tiles otherwise) on the last assembled system.
 * With p = d_z + beta d_pold on active cells (beta == 0: p = d_z, d_pold
 * unread), it writes d_p = p and d_q = A32 p, where
 *     (A32 v)_P = cb_P v_P + sum_f w_f (K_P + K_N)/2 (v_P - v_N)
 * over interior faces to active neighbours, w_f = A_f/d_f, K = FP32 K(h^k),
 * cb = FP32 (c + Dirichlet half-cell terms); inactive entries are written 0.
 * d_z, d_pold, d_p, d_q: N floats on the device (d_p and d_q must not alias
 * the inputs).  *pq (may be NULL): p . q, FP32 sums within blocks, FP64
 * across them.  Overwrites the context's inner-solve scratch. */
rf_status rf_apply_inner(rf_ctx *ctx, const float *d_z, const float *d_pold, float beta, float *d_p, float *d_q,
                         double *pq);

/* Test hook for the bounded device waits (failure detection): polls that a
 * wait for staged data (the TMA planes of the FP32 stencil) makes before it
 * gives up; polls = 0 restores the default (about a second of suspending
 * polls); polls < 0 makes each such wait a single non-blocking test.  A wait
 * that gives up stops the solve, drains the copies still in flight with the
 * default limit, and the call in progress returns RF_ERR_DEVICE_TIMEOUT with
 * the state unchanged and the context usable. */
rf_status rf_set_wait_limit(rf_ctx *ctx, int polls);

/* Number of CUDA kernel launches this context has executed on the device,
 * counted by the kernels themselves (loop bodies replayed from CUDA graphs
 * included).  Synchronises the context's stream. */
unsigned long long rf_launch_count(rf_ctx *ctx);

/* Per-kind launch counters: out[2 k] = launches of kernel kind k, out[2 k + 1]
 * = those that did work (a finished loop's kernels return at once).  Kinds,
 * in order: closure, closure+Picard test, assembly, FP64 CG init, FP64 CG
 * stencil, FP64 CG update, FP64 operator apply, mixed start, FP64 outer
 * residual, FP32 CG stencil, FP32 CG update, correction add, water balance,
 * storage, accept.  Returns the number of values written (<= cap). */
int rf_launch_counts(rf_ctx *ctx, unsigned long long *out, int cap);

/* Kernels that rf_profile_kernel can time. */
typedef enum rf_kernel_kind {
    RF_K_CLOSURE = 0,      /* closures at h with max|h - h_prev|            */
    RF_K_ASSEMBLE = 1,     /* Picard-system assembly                        */
    RF_K_CG64_SPMV = 2,    /* FP64 p-update + stencil product + p.q         */
    RF_K_CG64_UPDATE = 3,  /* FP64 x, r, z update + r.r, r.z                */
    RF_K_RESID64 = 4,      /* FP64 outer residual of the mixed path         */
    RF_K_CG32_SPMV = 5,    /* FP32 inner p-update + stencil product + p.q   */
    RF_K_CG32_UPDATE = 6   /* FP32 inner x, r, z update + dots              */
} rf_kernel_kind;

/* Time `reps` launches of one kernel on the system assembled at the current
 * state (h, dt_nom), each bracketed by CUDA events on the context's stream.
 * Returns the mean device time per launch [ms] and the algorithmic bytes one
 * launch must move (per-active-cell bytes of that kernel times the active
 * cells, plus the flag bytes of all cells).  The state h is not modified;
 * the linear-solver scratch is. */
rf_status rf_profile_kernel(rf_ctx *ctx, int kind, int reps, double *avg_ms, double *bytes_per_launch);

/* ---- batched ensemble of independent problems ----------------------------
 *
 * Many independent instances of uneven size (soil columns and blocks), each
 * with its own grid, van Genuchten soil, uniform initial head, top and bottom
 * conditions (lateral faces zero-flux) and its own EBATS / Picard / PCG state,
 * advanced together by one persistent kernel launched from a CUDA graph.  A
 * work unit is a thread-block cluster of `cluster` CTAs that takes instances
 * from a device queue (largest first) and integrates each one in time; the
 * per-cell arithmetic is the single-domain solver's. */
typedef struct rf_ens rf_ens;

typedef struct rf_ens_instance {
    int nx, ny, nz;
    double dx, dy, dz;
    rf_soil soil;
    double h0;                            /* uniform initial head [m]                 */
    int top_type;                         /* RF_BC_DIRICHLET, RF_BC_FLUX, ZERO_FLUX   */
    double top_value;
    int bottom_type;                      /* RF_BC_FREE_DRAINAGE, DIRICHLET, ZERO_FLUX */
    double bottom_value;
} rf_ens_instance;

typedef struct rf_ens_stats {
    double t, dt_nom;
    long long steps, picard_iters, cg_iters, rejected;
    int status;                           /* RF_OK, RF_ERR_DT_MIN, RF_ERR_DEVICE_TIMEOUT */
    long long cells;
    double storage0, inflow_cum, outflow_cum, closure_abs, nonlinear_defect_cum;
    double busy_s;                        /* device wall time the instance held its CTAs (all runs) */
    int ctas;                             /* CTAs that ran it in the last run (cluster size or 1) */
} rf_ens_stats;

/* Create an ensemble (instances copied; params checked as for rf_mesh_create;
 * the precision selects FP64 PCG or FP32 inner PCG in FP64 defect
 * correction).  The ensemble runs the chord Picard form with Jacobi-PCG, or
 * with RF_PREC_MIXED and RF_PRECOND_ZLINE the vertical-line-preconditioned
 * inner PCG: another picard_form or precond returns RF_ERR_ARG.  Instances and params are
 * checked before the device is queried; *out is NULL on every error. */
rf_status rf_ens_create(const rf_ens_instance *inst, int n, const rf_solver_params *params, void *cuda_stream,
                        const rf_allocator *alloc, rf_ens **out);
void rf_ens_destroy(rf_ens *ens);
/* Tiling of the work units: cluster size 1, 2, 4 or 8 CTAs and CTA size
 * (threads) 128, 256 or 512 (smaller CTAs put more instances on an SM at
 * once).  Default: clusters of 1 CTA of 512 threads. */
rf_status rf_ens_set_tiling(rf_ens *ens, int cluster, int threads);
/* Schedule of the work queue: order[k] = the instance (user index) popped
 * k-th, a permutation of 0..n-1 (NULL: largest instances first, the
 * default); the first n_wide of them run on a whole cluster each, the rest on
 * one CTA each (n_wide < 0 or >= n: all on clusters, the default).  Applies
 * to later runs; the state is untouched. */
rf_status rf_ens_set_schedule(rf_ens *ens, const int *order, int n_wide);
/* Advance every instance to t_end (one graph launch; synchronises). */
rf_status rf_ens_run(rf_ens *ens, double t_end);
/* State of instance i (user order): h (host, its nx*ny*nz cells, or NULL). */
rf_status rf_ens_get(rf_ens *ens, int i, double *h, rf_ens_stats *stats);
/* Return every instance to its initial state. */
rf_status rf_ens_reset(rf_ens *ens);
/* Tuner: from the initial state to t_probe, time every tiling that fits
 * (cluster 1, 2, 4, 8 x 256 or 512 threads) with every instance on a whole
 * work unit, recording each instance's run time at each width; order the
 * queue heaviest first and predict each tiling's makespan with a
 * list-scheduling model of the persistent queue; time the three best
 * predictions; keep the fastest measured tiling and order, and reset to the
 * initial state.  Every instance stays on a whole unit (best_wide = n): a
 * short probe cannot tell which instances stay light for a whole window, so
 * split schedules are set explicitly with rf_ens_set_schedule.  Outputs may
 * be NULL. */
rf_status rf_ens_tune(rf_ens *ens, double t_probe, int *best_cluster, int *best_threads, int *best_wide,
                      double *best_ms);
/* The tuner's model of the persistent queue (host arithmetic only, no
 * device): `units` work units of `cluster` CTAs pop the n instances in
 * `order` (a permutation of 0..n-1); the first n_wide run on a whole unit
 * for wide_s[i] seconds; the first other pop splits its unit into `cluster`
 * single CTAs, which run instances for solo_s[i] seconds (solo_s may be NULL
 * when n_wide >= n).  *makespan: when the last instance ends. */
rf_status rf_ens_model_makespan(const double *wide_s, const double *solo_s, const int *order, int n, int n_wide,
                                int units, int cluster, double *makespan);

/* ---- a linear solve that allocates no device memory ----------------------
 *
 * No counterpart in the paper: this is a library facility.  Some callers
 * cannot call cudaMalloc: host applications that own the device's memory
 * through their own pool and forbid allocation once their time loop runs,
 * coupled-model frameworks that must not pay cudaMalloc/cudaFree's implicit
 * device synchronisation inside a step, and code held to a memory budget
 * fixed at start-up.  rf_pcg_solve_noalloc solves the 7-point system
 *     (A x)_P = diag_P x_P - sum_f T_f x_N = b_P
 * with Jacobi-preconditioned CG and allocates nothing: its work vectors live
 * in one file-scope device array sized for RF_NOALLOC_MAX_CELLS cells
 * (3 343 104 bytes, about 3.3 MB), which every GPU that loads the library
 * holds until the process exits.
 *
 *   nx, ny, nz   grid (cells indexed i + nx (j + ny k)); nx*ny*nz must not
 *                exceed RF_NOALLOC_MAX_CELLS, else RF_ERR_ARG
 *   d_diag       N doubles, diag(A); a cell with diag <= 0 is inactive (its
 *                row and column are ignored, its x is left as given)
 *   d_Tx/Ty/Tz   N doubles each: coefficient of the cell's +x / +y / +z face
 *                (0 at the grid edge and next to inactive cells), so the -x
 *                coefficient of cell p is d_Tx[p - 1], etc.
 *   d_b          N doubles, right-hand side
 *   d_x          N doubles: x0 on entry, the solution on return
 *   tol, max_it  stop when ||b - A x||_2 <= tol ||b||_2 (recursive
 *                residual); RF_ERR_CG when max_it iterations do not reach it
 *   cuda_stream  cudaStream_t the work is ordered on (NULL: legacy stream)
 *   iters        CG iterations done (may be NULL)
 * All pointers are device pointers on the current device, borrowed.
 * Errors: RF_ERR_ARG (bad size or pointer), RF_ERR_NO_DEVICE (the current
 * device is not sm_103), RF_ERR_CUDA (a launch or copy failed),
 * RF_ERR_CG (max_it reached or a non-finite solve).
 *
 * The first call on a device checks the device and looks up the array's
 * device address (a cudaGetSymbolAddress with that device current), then
 * caches both.  Every call reads its iteration count back to the host and
 * synchronises cuda_stream, so it must not be issued while that stream is
 * being captured into a CUDA graph.  Every call shares the one array: calls
 * that overlap on the GPU (other streams or host threads) race and must be
 * serialised by the caller.  Each call clears what has to start at zero
 * (solver scalars, reduction ticket, counters); nothing else of a previous
 * call's contents is read. */
#define RF_NOALLOC_MAX_CELLS 65536
rf_status rf_pcg_solve_noalloc(int nx, int ny, int nz, const double *d_diag, const double *d_Tx,
                               const double *d_Ty, const double *d_Tz, const double *d_b, double *d_x,
                               double tol, int max_it, void *cuda_stream, int *iters);

/* ---------------------------------------------------------------------
 * Learned warm start.  The paper starts each Picard sequence (Sec. 2.2) from
 * the previous time level h^n; this extension starts it from a network's
 * guess instead.  Picard still runs to tol_picard from that guess, so the
 * method judges the guess's error; when an attempt from a guess does not
 * converge, the step falls back to the plain method (restart from h^n with
 * dt / f_shrink, as for any rejected attempt).
 *
 * Network: a 3-D convolutional residual network in BF16 with FP32
 * accumulation -- input convolution 4 -> 32, four residual blocks of two
 * 32 -> 32 convolutions (ReLU after the first; the block input is added
 * before the second ReLU), output convolution 32 -> 1.  All convolutions
 * are 3x3x3, stride 1, zero padding 1, cross-correlation.  Volumes are
 * channels-last, voxel index x + W (y + H (z + D b)); a mesh is one volume
 * with D = nz, H = ny, W = nx, so voxel = cell index p.
 *
 * Parameters are exchanged as RF_NN_PARAMS floats, layer by layer (input,
 * block 1 conv 1, block 1 conv 2, ..., output): W[cout][3][3][3][cin] (the
 * first index of each 3 is the -1 offset along z, y, x) then b[cout].
 * --------------------------------------------------------------------- */
typedef struct rf_nn rf_nn;
#define RF_NN_PARAMS 225793

/* Feature and output scales.  Features of an active cell:
 *   0: h / h_scale                       1: (ln Ks - lnK_mean) / lnK_std
 *   2: q_top / q_scale on cells that carry the top (z max) boundary face, 0
 *      elsewhere; q_top is the top flux condition's value at the step's
 *      start time (0 if the top condition is not RF_BC_FLUX)
 *   3: ln(dt / t_scale)
 * and all zero on inactive cells.  The guess is h + y out_scale dt. */
typedef struct rf_ws_scales {
    double h_scale, lnK_mean, lnK_std, q_scale, t_scale, out_scale;
} rf_ws_scales;

/* Adam (Kingma & Ba 2015) settings of a training step. */
typedef struct rf_adam {
    float lr, beta1, beta2, eps;
} rf_adam;

/* Create a network on the current device, parameters zero, work ordered on
 * cuda_stream (a cudaStream_t, NULL = legacy stream).  Device memory
 * (parameters, optimizer moments, activations sized for the largest volume
 * seen) comes from alloc when given. */
rf_status rf_nn_create(void *cuda_stream, const rf_allocator *alloc, rf_nn **out);
void rf_nn_destroy(rf_nn *net);
/* Copy RF_NN_PARAMS host floats in / out (n must equal RF_NN_PARAMS).
 * Setting parameters also clears the Adam moments and step count. */
rf_status rf_nn_set_params(rf_nn *net, const float *params, long long n);
rf_status rf_nn_get_params(rf_nn *net, float *params, long long n);
/* Forward pass.  d_x: B*D*H*W*4 floats (features, channels-last, 16-byte
 * aligned); d_y: B*D*H*W floats (output).  Asynchronous on the network's
 * stream. */
rf_status rf_nn_forward(rf_nn *net, const float *d_x, int B, int D, int H, int W, float *d_y);
/* Loss L = (1/M) sum_v mask_v (y_v - target_v)^2 over the M = B*D*H*W
 * voxels (d_mask may be NULL: all ones), and its gradient.  grad: NULL or
 * RF_NN_PARAMS host floats (parameter order above).  Synchronises. */
rf_status rf_nn_loss_grad(rf_nn *net, const float *d_x, const float *d_target, const float *d_mask, int B, int D,
                          int H, int W, float *loss, float *grad);
/* One training step: loss, gradient, Adam update of the FP32 master
 * parameters.  loss: NULL (asynchronous) or where to write L (synchronises). */
rf_status rf_nn_train_step(rf_nn *net, const float *d_x, const float *d_target, const float *d_mask, int B, int D,
                           int H, int W, const rf_adam *opt, float *loss);
/* Kernel launches issued by this network so far (host count). */
long long rf_nn_launch_count(const rf_nn *net);

/* Trace of a gradient evaluation, for checking each layer's kernels element
 * by element: after rf_nn_set_trace(net, 1), every rf_nn_loss_grad /
 * rf_nn_train_step also keeps each layer's BF16 output gradient (the values
 * its weight-gradient and input-gradient contractions read), and
 * rf_nn_trace_get copies one stored tensor of the last evaluation into host
 * memory, channels-last over its M = B*D*H*W voxels:
 *   RF_NN_TRACE_INPUT     index 0: BF16 features, M x 8 (4 features, 4 zero)
 *   RF_NN_TRACE_BLOCK_OUT index 0..4: BF16 activation after the input
 *                         convolution (0) and after residual block i (i), M x 32
 *   RF_NN_TRACE_BLOCK_MID index 0..3: BF16 activation between the two
 *                         convolutions of residual block i + 1, M x 32
 *   RF_NN_TRACE_OUT_GRAD  index 0..9: BF16 gradient of the loss with respect
 *                         to layer index's output (after its ReLU mask),
 *                         M x 32 (layer 9: M x 8, channel 0 used)
 *   RF_NN_TRACE_OUTPUT    index 0: FP32 network output, M x 8 (channel 0 used)
 * BF16 values are copied as their 16-bit patterns.  count must equal the
 * tensor's element count (RF_ERR_ARG otherwise); RF_ERR_STATE when no traced
 * evaluation exists.  Synchronises the network's stream. */
enum { RF_NN_TRACE_INPUT = 0, RF_NN_TRACE_BLOCK_OUT = 1, RF_NN_TRACE_BLOCK_MID = 2, RF_NN_TRACE_OUT_GRAD = 3,
       RF_NN_TRACE_OUTPUT = 4 };
rf_status rf_nn_set_trace(rf_nn *net, int on);
rf_status rf_nn_trace_get(rf_nn *net, int what, int index, void *host, long long count);

/* Features of a state of the mesh for a step of size dt from time t (the
 * top flux feature takes the top condition's value at t): d_h is N doubles
 * on the device, or NULL for the context's current state; d_x receives N*4
 * floats (16-byte aligned).  Ordered on the context's stream.  The warm
 * start computes the same features from the current state and time. */
rf_status rf_ws_features(rf_ctx *ctx, const rf_ws_scales *sc, const double *d_h, double t, double dt, float *d_x);
/* Training target of the step just taken from d_h_old (N doubles, the state
 * before the step) with size dt: d_target[p] = (h[p] - h_old[p]) /
 * (out_scale dt) on active cells, else 0; d_mask (may be NULL) 1 / 0. */
rf_status rf_ws_target(rf_ctx *ctx, const rf_ws_scales *sc, const double *d_h_old, double dt, float *d_target,
                       float *d_mask);
/* Attach a network (borrowed; NULL detaches): every step's first attempt
 * starts Picard from the network's guess.  The network must live on the
 * context's device; its inference then runs on the context's stream. */
rf_status rf_ws_attach(rf_ctx *ctx, rf_nn *net, const rf_ws_scales *sc);
typedef struct rf_ws_stats {
    long long guesses;     /* attempts started from a guess                    */
    long long fallbacks;   /* of those, attempts that did not converge         */
} rf_ws_stats;
rf_status rf_ws_get_stats(rf_ctx *ctx, rf_ws_stats *out);


#ifdef __cplusplus
}
#endif
#endif /* RF_H */
