/*
 * richards_oracle.c -- plain, slow, FP64 CPU oracle for the Picard /
 * backward-Euler / finite-volume solve of the 3-D transient Richards equation
 * (Orgogozo et al., "RichardsFOAM", arXiv:1809.10895).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, calls or
 * includes this file; only the tests, the package entry's smoke check and the
 * benchmark's CPU-baseline leg load it.  It shares no code, header, table or
 * helper with the CUDA path.
 *
 * What it follows, step by step, in the paper's order:
 *   - Eq. 1 (pressure-head form, z upward) and Eq. 2-4 (van Genuchten / Mualem
 *     closures), written literally with pow();
 *   - Sec. 2.2: classical Picard linearisation, chord-slope capacity,
 *     backward Euler for the pressure term, explicit (lagged one Picard iterate)
 *     gravity with linearly interpolated face conductivity, PCG linear solve,
 *     EBATS adaptive time stepping;
 *   - Sec. 2.2 also names a modified Picard linearisation, kept for mass
 *     conservation: the mixed-form scheme (theta expanded about the current
 *     iterate, theta(h^{k+1}) ~ theta(h^k) + C(h^k) (h^{k+1} - h^k)), selected
 *     with the parameter picard_form = 1;
 *   - Sec. 2.3: the Picard exit test is a global max over the domain;
 *   - Appendix A: Gardner conductivity K = Ks exp(alpha h) (test model).
 * Options for alternatives the paper names: the DIC preconditioner of
 * Sec. 2.2 (natural and red-black order), Brooks-Corey closures (Sec. 1), a
 * harmonic interface mean, Richardson step-doubling and variable-step BDF2
 * time control (Sec. 2.2), and gravity along any grid axis for a grid
 * aligned with the tilted slab of Sec. 4.2.  Readings of passages the paper
 * leaves open (storage S for h >= 0, the form of boundary terms, the CG
 * stopping norm, EBATS details) are restated where they are used below.
 *
 * The linear system is stored explicitly in CSR over the active cells and
 * solved by a textbook Jacobi-PCG or DIC-PCG, or by a dense Cholesky
 * factorisation on tiny grids.  No blocking, fusion or reordering beyond
 * those definitions.
 *
 * Built plainly it runs on one thread.  Built with -fopenmp, the loops that
 * treat every cell on its own (closures, matrix rows, the Jacobi-PCG vector
 * operations, the water balance) and the sums and maxima over cells run on
 * all cores; a sum over cells is then added in another order, so results
 * differ by rounding only.  The pins use the one-thread build; the threaded
 * one serves the all-core CPU baseline.
 *
 * Pins (tests/test_oracle_*.py): closed forms of the closures, C = dtheta/dh
 * by finite differences, Mualem's integral for K, the hydrostatic fixed point,
 * the saturated linear (heat-equation) limit with exact discrete eigenmodes,
 * Appendix A's analytic Gardner profile, unit-gradient steady state, dense
 * Cholesky vs CG, global mass-balance closure, a scripted EBATS sequence,
 * exact linear steady states through seepage and Dirichlet faces, and for
 * each option a closed form or an invariant (exact DIC on a tridiagonal
 * column, axis-permutation invariance of gravity, the layered steady state
 * of the harmonic mean, the temporal orders of BDF2 and Richardson).
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { OR_VG = 0, OR_GARDNER = 1, OR_BROOKS_COREY = 2 };
enum { OR_ZERO_FLUX = 0, OR_DIRICHLET = 1, OR_FLUX = 2, OR_FREE_DRAINAGE = 3, OR_SEEPAGE = 4 };
enum { OR_XMIN = 0, OR_XMAX, OR_YMIN, OR_YMAX, OR_ZMIN, OR_ZMAX, OR_NFACES };
enum { OR_OK = 0, OR_ERR_ARG = 1, OR_ERR_PICARD = 6, OR_ERR_DT_MIN = 7, OR_ERR_CG = 8 };
/* linear solvers: Jacobi-PCG, dense Cholesky (tiny grids), and PCG with the
 * diagonal incomplete Cholesky (DIC) preconditioner the paper uses (Sec. 2.2),
 * eliminating cells in natural (cell index) order or red-black order */
enum { OR_SOLVER_PCG = 0, OR_SOLVER_DENSE = 1, OR_SOLVER_DIC = 2, OR_SOLVER_DIC_RB = 3 };

typedef struct {
    int model;
    double theta_r, theta_s, alpha, n, Ks, S;
} or_soil;

typedef struct {
    int type;
    int n;          /* number of breakpoints */
    double *t, *v;  /* piecewise-constant series: v[i] holds on [t[i], t[i+1]) */
} or_bc;

typedef struct or_problem {
    int nx, ny, nz, N;   /* N = nx*ny*nz cells, x fastest, z slowest */
    double dx, dy, dz, zb;
    unsigned char *active;
    int *idx;            /* cell -> compact active index or -1 */
    int *cell;           /* compact index -> cell */
    int na;              /* number of active cells */

    int nzones;
    or_soil *zones;
    unsigned char *zone; /* per cell */
    double *Ks;          /* per cell saturated conductivity */

    or_bc bc[OR_NFACES];

    /* parameters */
    double tol_picard, tol_cg, dt0, dt_max, dt_min, f_grow, f_shrink, eps_chord;
    int cg_max_it, n_inc, n_small, n_max, solver;
    int picard_form;     /* 0 classical Picard with chord capacity, 1 modified Picard */
    int face_mean;       /* interface K: 0 arithmetic (linear interpolation, Sec. 2.2), 1 harmonic */
    int time_control;    /* 0 EBATS (Sec. 2.2), 1 Richardson step doubling */
    int time_scheme;     /* 0 backward Euler (Sec. 2.2), 1 variable-step BDF2 (needs picard_form 1) */
    double *h_prev;      /* BDF2: h^{n-1} */
    double dt_prev;      /* BDF2: the previous step's dt (0: no history, the step is backward Euler) */
    double tol_time;     /* Richardson: bound on max |h(2 x dt/2) - h(dt)| per step [m] */
    double err_last, err_max;   /* Richardson estimate of the last and the largest accepted step */
    double grav[3];      /* gradient of elevation in grid axes (x, y, z); (0, 0, 1) for z up.
                          * Eq. 1's gravity term for a grid aligned with a tilted slab */

    int *row_ptr;        /* na + 1: CSR row starts, fixed by the active pattern */

    /* state */
    double *h;           /* N */
    double t, dt_nom;
    int easy;

    /* mass balance */
    double storage0, inflow_cum, outflow_cum, closure_cum, defect_cum;
} or_problem;

static int neighbour(const or_problem *P, int i, int j, int k, int f);

/* ------------------------------------------------------------------------ */
/* Closures, Eq. 2-4 (van Genuchten / Mualem) and Appendix A (Gardner).      */
/* theta* = theta(h) for h < 0 and theta_s + S*h for h >= 0: with that       */
/* reading d(theta*)/dh equals Eq. 3 on both branches, so the chord slope of    */
/* theta* is the mass-consistent capacity.  The tie h = 0 takes the          */
/* saturated branch.                                                         */
/* ------------------------------------------------------------------------ */
static void closure(const or_soil *s, double Ks, double h, double *theta, double *K, double *C)
{
    if (h >= 0.0) {
        *theta = s->theta_s + s->S * h;
        *K = Ks;
        *C = s->S;
        return;
    }
    if (s->model == OR_BROOKS_COREY) {
        /* Brooks and Corey, the alternative closure Sec. 1 names: air-entry
         * head h_b = -1/alpha, pore-size index lambda = n;
         * Se = (h_b / h)^lambda below h_b, 1 above;
         * theta = theta_r + (theta_s - theta_r) Se, C = d theta / dh,
         * K = Ks Se^((2 + 3 lambda) / lambda) (Brooks and Corey's own form). */
        double hb = -1.0 / s->alpha, lam = s->n;
        if (h >= hb) {
            *theta = s->theta_s;
            *K = Ks;
            *C = 0.0;
            return;
        }
        double se = pow(hb / h, lam);
        *theta = s->theta_r + (s->theta_s - s->theta_r) * se;
        *C = -lam * (s->theta_s - s->theta_r) * se / h;
        *K = Ks * pow(se, (2.0 + 3.0 * lam) / lam);
        return;
    }
    if (s->model == OR_GARDNER) {
        /* Appendix A, Eq. A6: K = Ks exp(alpha h).  The paper gives no
         * retention curve for this test model; theta = theta_r +
         * (theta_s - theta_r) exp(alpha h) is used, which only shapes the
         * transient path to the steady state. */
        double e = exp(s->alpha * h);
        *K = Ks * e;
        *theta = s->theta_r + (s->theta_s - s->theta_r) * e;
        *C = (s->theta_s - s->theta_r) * s->alpha * e;
        return;
    }
    double a = s->alpha, n = s->n;
    double m = 1.0 - 1.0 / n;
    double base = 1.0 + pow(-a * h, n);          /* 1 + (-alpha h)^n          */
    double se = pow(base, -(1.0 - 1.0 / n));     /* Eq. 2 bracket             */
    *theta = (s->theta_s - s->theta_r) * se + s->theta_r;                 /* Eq. 2 */
    *C = (s->theta_s - s->theta_r) * a * n * (1.0 - 1.0 / n) * pow(-a * h, n - 1.0)
         * pow(base, -(2.0 - 1.0 / n));                                   /* Eq. 3 */
    /* Eq. 4, with the garbled exponent "(n/n-1)" read as n/(n-1) = 1/m. */
    *K = Ks * pow(se, 0.5) * pow(1.0 - pow(1.0 - pow(se, n / (n - 1.0)), m), 2.0);
}

void or_closure_eval(int model, double theta_r, double theta_s, double alpha, double n,
                     double Ks, double S, double h, double *out3)
{
    or_soil s = { model, theta_r, theta_s, alpha, n, Ks, S };
    closure(&s, Ks, h, &out3[0], &out3[1], &out3[2]);
}

/* ------------------------------------------------------------------------ */
/* Problem set-up                                                            */
/* ------------------------------------------------------------------------ */
or_problem *or_create(int nx, int ny, int nz, double dx, double dy, double dz, double z_bottom,
                      const unsigned char *active)
{
    if (nx < 1 || ny < 1 || nz < 1 || !(dx > 0) || !(dy > 0) || !(dz > 0)) return NULL;
    or_problem *P = (or_problem *)calloc(1, sizeof(or_problem));
    P->nx = nx; P->ny = ny; P->nz = nz; P->N = nx * ny * nz;
    P->dx = dx; P->dy = dy; P->dz = dz; P->zb = z_bottom;
    P->active = (unsigned char *)malloc(P->N);
    P->idx = (int *)malloc(sizeof(int) * P->N);
    P->cell = (int *)malloc(sizeof(int) * P->N);
    P->na = 0;
    for (int p = 0; p < P->N; p++) {
        P->active[p] = active ? (active[p] != 0) : 1;
        if (P->active[p]) { P->idx[p] = P->na; P->cell[P->na] = p; P->na++; }
        else P->idx[p] = -1;
    }
    /* a matrix row holds the diagonal and one entry per active neighbour */
    P->row_ptr = (int *)malloc(sizeof(int) * (P->na + 1));
    P->row_ptr[0] = 0;
    for (int a = 0; a < P->na; a++) {
        int p = P->cell[a], i = p % nx, j = (p / nx) % ny, k = p / (nx * ny), nnz = 1;
        for (int f = 0; f < 6; f++) {
            int q = neighbour(P, i, j, k, f);
            if (q >= 0 && P->active[q]) nnz++;
        }
        P->row_ptr[a + 1] = P->row_ptr[a] + nnz;
    }
    P->zone = (unsigned char *)calloc(P->N, 1);
    P->Ks = (double *)calloc(P->N, sizeof(double));
    P->h = (double *)calloc(P->N, sizeof(double));
    P->h_prev = (double *)calloc(P->N, sizeof(double));
    for (int f = 0; f < OR_NFACES; f++) P->bc[f].type = OR_ZERO_FLUX;
    /* defaults (readings): Picard 1e-6 m, CG 1e-10 relative, EBATS 10/3/8, f 1.3 */
    P->tol_picard = 1e-6; P->tol_cg = 1e-10; P->cg_max_it = 10000;
    P->dt0 = 1.0; P->dt_max = 600.0; P->dt_min = 1e-3; P->f_grow = 1.3; P->f_shrink = 1.3;
    P->n_inc = 10; P->n_small = 3; P->n_max = 8; P->eps_chord = 1e-10;
    P->grav[0] = 0.0; P->grav[1] = 0.0; P->grav[2] = 1.0;
    P->tol_time = 1e-3;
    P->solver = OR_SOLVER_PCG;
    P->dt_nom = P->dt0;
    return P;
}

void or_destroy(or_problem *P)
{
    if (!P) return;
    for (int f = 0; f < OR_NFACES; f++) { free(P->bc[f].t); free(P->bc[f].v); }
    free(P->active); free(P->idx); free(P->cell); free(P->zones); free(P->zone);
    free(P->Ks); free(P->h); free(P->h_prev); free(P->row_ptr); free(P);
}

int or_num_active(const or_problem *P) { return P->na; }

/* threads the per-cell loops run on: 1 unless built with OpenMP */
int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

int or_set_soils(or_problem *P, int nzones, const int *model, const double *theta_r,
                 const double *theta_s, const double *alpha, const double *n, const double *Ks,
                 const double *S, const unsigned char *zone_of_cell, const double *Ks_cell)
{
    if (nzones < 1 || nzones > 256) return OR_ERR_ARG;
    free(P->zones);
    P->zones = (or_soil *)malloc(sizeof(or_soil) * nzones);
    P->nzones = nzones;
    for (int z = 0; z < nzones; z++) {
        or_soil s = { model[z], theta_r[z], theta_s[z], alpha[z], n[z], Ks[z], S[z] };
        if (s.model == OR_VG && !(s.n > 1.0)) return OR_ERR_ARG;
        if (s.model == OR_BROOKS_COREY && !(s.n > 0.0)) return OR_ERR_ARG;
        P->zones[z] = s;
    }
    for (int p = 0; p < P->N; p++) {
        int z = zone_of_cell ? zone_of_cell[p] : 0;
        if (z >= nzones) return OR_ERR_ARG;
        P->zone[p] = (unsigned char)z;
        P->Ks[p] = Ks_cell ? Ks_cell[p] : P->zones[z].Ks;
    }
    return OR_OK;
}

int or_set_bc(or_problem *P, int face, int type, const double *t, const double *v, int n)
{
    if (face < 0 || face >= OR_NFACES || type < 0 || type > OR_SEEPAGE) return OR_ERR_ARG;
    if (type == OR_FREE_DRAINAGE && face != OR_ZMIN) return OR_ERR_ARG;
    if ((type == OR_DIRICHLET || type == OR_FLUX) && (n < 1 || !v)) return OR_ERR_ARG;
    or_bc *b = &P->bc[face];
    free(b->t); free(b->v); b->t = NULL; b->v = NULL; b->n = 0;
    b->type = type;
    if (n > 0 && v) {
        b->n = n;
        b->t = (double *)malloc(sizeof(double) * n);
        b->v = (double *)malloc(sizeof(double) * n);
        for (int i = 0; i < n; i++) { b->t[i] = t ? t[i] : 0.0; b->v[i] = v[i]; }
        for (int i = 1; i < n; i++) if (!(b->t[i] > b->t[i - 1])) return OR_ERR_ARG;
    }
    return OR_OK;
}

int or_set_param(or_problem *P, const char *name, double value)
{
#define DP(nm) if (!strcmp(name, #nm)) { P->nm = value; return OR_OK; }
#define IP(nm) if (!strcmp(name, #nm)) { P->nm = (int)value; return OR_OK; }
    DP(tol_picard) DP(tol_cg) DP(dt0) DP(dt_max) DP(dt_min) DP(f_grow) DP(f_shrink) DP(eps_chord)
    if (!strcmp(name, "grav_x")) { P->grav[0] = value; return OR_OK; }
    if (!strcmp(name, "grav_y")) { P->grav[1] = value; return OR_OK; }
    if (!strcmp(name, "grav_z")) { P->grav[2] = value; return OR_OK; }
    IP(cg_max_it) IP(n_inc) IP(n_small) IP(n_max) IP(solver) IP(picard_form) IP(face_mean) IP(time_control)
    IP(time_scheme)
    DP(tol_time)
#undef DP
#undef IP
    return OR_ERR_ARG;
}

/* Time-tolerance used when comparing simulated times to breakpoints. */
static double t_tol(double t) { return 1e-9 * (fabs(t) > 1.0 ? fabs(t) : 1.0); }

/* value of a piecewise-constant series at the start time of a step */
static double series_at(const or_bc *b, double t)
{
    int i = 0;
    while (i + 1 < b->n && b->t[i + 1] <= t + t_tol(t)) i++;
    return b->v[i];
}

static double storage_of(const or_problem *P, const double *h)
{
    double V = P->dx * P->dy * P->dz, s = 0.0;
#pragma omp parallel for reduction(+ : s)
    for (int a = 0; a < P->na; a++) {
        int p = P->cell[a];
        double th, K, C;
        closure(&P->zones[P->zone[p]], P->Ks[p], h[p], &th, &K, &C);
        s += V * th;
    }
    return s;
}

int or_set_state(or_problem *P, const double *h, double t)
{
    if (!P->zones) return OR_ERR_ARG;
    memcpy(P->h, h, sizeof(double) * P->N);
    P->t = t;
    P->dt_nom = P->dt0 < P->dt_max ? P->dt0 : P->dt_max;
    P->easy = 0;
    P->storage0 = storage_of(P, P->h);
    P->inflow_cum = P->outflow_cum = P->closure_cum = P->defect_cum = 0.0;
    P->err_last = P->err_max = 0.0;
    P->dt_prev = 0.0;
    return OR_OK;
}

/* Resume bookkeeping: the time and the EBATS nominal step and easy-step
 * counter of a state saved elsewhere (the state itself via or_set_state). */
int or_set_clock(or_problem *P, double t, double dt_nom, int easy)
{
    if (!(dt_nom > 0.0) || easy < 0) return OR_ERR_ARG;
    P->t = t;
    P->dt_nom = dt_nom;
    P->easy = easy;
    return OR_OK;
}

void or_get_state(const or_problem *P, double *h, double *meta4)
{
    if (h) memcpy(h, P->h, sizeof(double) * P->N);
    if (meta4) { meta4[0] = P->t; meta4[1] = P->dt_nom; meta4[2] = P->easy; meta4[3] = P->na; }
}

/* ------------------------------------------------------------------------ */
/* Assembly of the Picard linear system (Sec. 2.2; Eq. 1 in FV form).        */
/*                                                                          */
/*   V C^k_P (h_P - h^n_P)/dt = sum_f T_f (h_N - h_P) + G_P + B_P            */
/*                                                                          */
/* T_f = Kbar_f A_f / d_f with Kbar_f = (K_P + K_N)/2 (linear interpolation  */
/* on a uniform grid), G_P = A_z (Kbar_top - Kbar_bottom) (explicit gravity, */
/* K at the previous Picard iterate), B_P the boundary terms.  C^k is the     */
/* chord slope (theta*(h^k) - theta*(h^n))/(h^k - h^n), or d(theta*)/dh at h^k */
/* when |h^k - h^n| <= eps_chord.                                            */
/* ------------------------------------------------------------------------ */
typedef struct {
    int *row_ptr, *col;
    double *val;
    double *b, *diag;      /* na */
    double *K, *theta, *c; /* na: K(h^k), theta*(h^k), V C^k / dt */
    double *s0;            /* na: storage part of b (c h^n, or c h^k - V (theta^k - theta^n) / dt) */
    /* boundary-face bookkeeping for the mass balance: per active cell and
     * face, the flux into the cell as an affine function of x_P:
     *   flux = fa + fb * x_P  */
    double *fa, *fb;       /* na * 6 */
    int nnz;
} or_system;

static void sys_alloc(or_system *S, int na)
{
    S->row_ptr = (int *)malloc(sizeof(int) * (na + 1));
    S->col = (int *)malloc(sizeof(int) * (7 * (size_t)na));
    S->val = (double *)malloc(sizeof(double) * (7 * (size_t)na));
    S->b = (double *)malloc(sizeof(double) * na);
    S->diag = (double *)malloc(sizeof(double) * na);
    S->K = (double *)malloc(sizeof(double) * na);
    S->theta = (double *)malloc(sizeof(double) * na);
    S->c = (double *)malloc(sizeof(double) * na);
    S->s0 = (double *)malloc(sizeof(double) * na);
    S->fa = (double *)malloc(sizeof(double) * 6 * (size_t)na);
    S->fb = (double *)malloc(sizeof(double) * 6 * (size_t)na);
}

static void sys_free(or_system *S)
{
    free(S->row_ptr); free(S->col); free(S->val); free(S->b); free(S->diag);
    free(S->K); free(S->theta); free(S->c); free(S->s0); free(S->fa); free(S->fb);
}

/* neighbour of cell (i,j,k) across face f, or -1 outside the domain */
static int neighbour(const or_problem *P, int i, int j, int k, int f)
{
    switch (f) {
    case OR_XMIN: return i > 0 ? (i - 1) + P->nx * (j + P->ny * k) : -1;
    case OR_XMAX: return i < P->nx - 1 ? (i + 1) + P->nx * (j + P->ny * k) : -1;
    case OR_YMIN: return j > 0 ? i + P->nx * ((j - 1) + P->ny * k) : -1;
    case OR_YMAX: return j < P->ny - 1 ? i + P->nx * ((j + 1) + P->ny * k) : -1;
    case OR_ZMIN: return k > 0 ? i + P->nx * (j + P->ny * (k - 1)) : -1;
    default:      return k < P->nz - 1 ? i + P->nx * (j + P->ny * (k + 1)) : -1;
    }
}

static void assemble(const or_problem *P, const double *hk, const double *hn, double dt, double t,
                     or_system *S)
{
    const double V = P->dx * P->dy * P->dz;
    const double A[6] = { P->dy * P->dz, P->dy * P->dz, P->dx * P->dz, P->dx * P->dz,
                          P->dx * P->dy, P->dx * P->dy };
    const double d[6] = { P->dx, P->dx, P->dy, P->dy, P->dz, P->dz };
    /* gravity flux factor of each face of a cell, grad(elevation) . n_out:
     * with z up, +1 for the top face (water enters from above), -1 for the
     * bottom face, 0 lateral; along a tilted frame every axis carries its
     * component of the elevation gradient */
    const double g[6] = { -P->grav[0], P->grav[0], -P->grav[1], P->grav[1], -P->grav[2], P->grav[2] };
    double bcv[6];
    for (int f = 0; f < 6; f++) bcv[f] = P->bc[f].n > 0 ? series_at(&P->bc[f], t) : 0.0;

    /* closures at h^k and the capacity term.  Classical Picard: the chord
     * slope C^k = (theta*(h^k) - theta*(h^n)) / (h^k - h^n), storage
     * c (h^{k+1} - h^n).  Modified Picard: C^k = C(h^k), storage
     * c (h^{k+1} - h^k) + V (theta*(h^k) - theta*(h^n)) / dt.  Both vanish
     * in the same way at a converged iterate, V (theta* - theta*^n) / dt. */
#pragma omp parallel for
    for (int a = 0; a < P->na; a++) {
        int p = P->cell[a];
        const or_soil *s = &P->zones[P->zone[p]];
        double thk, Kk, Ck, thn, Kn, Cn;
        closure(s, P->Ks[p], hk[p], &thk, &Kk, &Ck);
        closure(s, P->Ks[p], hn[p], &thn, &Kn, &Cn);
        S->K[a] = Kk;
        S->theta[a] = thk;
        if (P->picard_form == 1 && P->time_scheme == 1 && P->dt_prev > 0.0) {
            /* variable-step BDF2 (the multistep alternative Sec. 2.2 names),
             * mixed form: V/dt [a0 theta^{n+1} - a1 theta^n + a2 theta^{n-1}]
             * with w = dt / dt_prev, a0 = (1 + 2w)/(1 + w), a1 = 1 + w,
             * a2 = w^2 / (1 + w); theta^{n+1} linearised about h^k as in the
             * modified Picard form */
            const double w = dt / P->dt_prev;
            const double a0 = (1.0 + 2.0 * w) / (1.0 + w), a1 = 1.0 + w, a2 = w * w / (1.0 + w);
            double thp, Kp, Cp;
            closure(s, P->Ks[p], P->h_prev[p], &thp, &Kp, &Cp);
            S->c[a] = a0 * V * Ck / dt;
            S->s0[a] = S->c[a] * hk[p] - V * (a0 * thk - a1 * thn + a2 * thp) / dt;
        } else if (P->picard_form == 1) {
            S->c[a] = V * Ck / dt;
            S->s0[a] = S->c[a] * hk[p] - V * (thk - thn) / dt;
        } else {
            double Cch;
            if (fabs(hk[p] - hn[p]) > P->eps_chord) Cch = (thk - thn) / (hk[p] - hn[p]);
            else Cch = Ck;
            S->c[a] = V * Cch / dt;
            S->s0[a] = S->c[a] * hn[p];
        }
    }

#pragma omp parallel for
    for (int a = 0; a < P->na; a++) {
        int p = P->cell[a];
        int i = p % P->nx, j = (p / P->nx) % P->ny, k = p / (P->nx * P->ny);
        const or_soil *s = &P->zones[P->zone[p]];
        double diag = S->c[a];
        double rhs = S->s0[a];
        int nb_col[6];
        double nb_val[6];
        for (int f = 0; f < 6; f++) {
            S->fa[6 * a + f] = 0.0;
            S->fb[6 * a + f] = 0.0;
            nb_col[f] = -1;
            int q = neighbour(P, i, j, k, f);
            if (q >= 0 && P->active[q]) {
                int aq = P->idx[q];
                /* interface conductivity: the linear interpolation of Sec. 2.2
                 * (arithmetic mean), or the harmonic mean, the exact series
                 * conductance of two half cells in steady flow */
                double Kbar = P->face_mean == 1
                                  ? (S->K[a] + S->K[aq] > 0.0 ? 2.0 * S->K[a] * S->K[aq] / (S->K[a] + S->K[aq]) : 0.0)
                                  : 0.5 * (S->K[a] + S->K[aq]);
                double T = Kbar * A[f] / d[f];
                diag += T;
                nb_col[f] = aq;
                nb_val[f] = -T;
                rhs += g[f] * Kbar * A[f];
                continue;
            }
            /* a boundary face: the domain edge, or a z-face whose neighbour
             * is inactive (top / bottom of an active column).  x/y faces that
             * touch an inactive cell are zero-flux. */
            if (q >= 0 && (f == OR_XMIN || f == OR_XMAX || f == OR_YMIN || f == OR_YMAX)) continue;
            int type = P->bc[f].type;
            double hD = 0.0;
            if (type == OR_SEEPAGE) {
                /* seepage face: Dirichlet h = 0 while the cell is saturated at
                 * the start of the step, zero flux otherwise */
                if (hn[p] >= 0.0) { type = OR_DIRICHLET; hD = 0.0; }
                else type = OR_ZERO_FLUX;
            } else if (type == OR_DIRICHLET) {
                hD = bcv[f];
            }
            if (type == OR_DIRICHLET) {
                double thD, KD, CD;
                closure(s, P->Ks[p], hD, &thD, &KD, &CD);
                double T = KD * A[f] / (0.5 * d[f]);
                diag += T;
                rhs += T * hD + g[f] * KD * A[f];
                S->fa[6 * a + f] = T * hD + g[f] * KD * A[f];
                S->fb[6 * a + f] = -T;
            } else if (type == OR_FLUX) {
                rhs += bcv[f] * A[f];
                S->fa[6 * a + f] = bcv[f] * A[f];
            } else if (type == OR_FREE_DRAINAGE) {
                /* unit hydraulic gradient: pressure gradient zero, gravity
                 * drives an outflow K(h^k_P) A_z (times the elevation
                 * gradient across the face in a tilted frame) */
                rhs += g[f] * S->K[a] * A[f];
                S->fa[6 * a + f] = g[f] * S->K[a] * A[f];
            }
        }
        /* CSR row with columns in ascending cell order */
        int nnz = P->row_ptr[a];
        S->row_ptr[a] = nnz;
        const int order[7] = { OR_ZMIN, OR_YMIN, OR_XMIN, -1, OR_XMAX, OR_YMAX, OR_ZMAX };
        for (int o = 0; o < 7; o++) {
            int f = order[o];
            if (f < 0) { S->col[nnz] = a; S->val[nnz] = diag; nnz++; }
            else if (nb_col[f] >= 0) { S->col[nnz] = nb_col[f]; S->val[nnz] = nb_val[f]; nnz++; }
        }
        S->diag[a] = diag;
        S->b[a] = rhs;
    }
    S->row_ptr[P->na] = P->row_ptr[P->na];
    S->nnz = P->row_ptr[P->na];
}

/* ------------------------------------------------------------------------ */
/* Linear solvers                                                            */
/* ------------------------------------------------------------------------ */
static void csr_spmv(int n, const int *rp, const int *col, const double *val, const double *x, double *y)
{
#pragma omp parallel for
    for (int r = 0; r < n; r++) {
        double s = 0.0;
        for (int e = rp[r]; e < rp[r + 1]; e++) s += val[e] * x[col[e]];
        y[r] = s;
    }
}

static double dot(int n, const double *a, const double *b)
{
    double s = 0.0;
#pragma omp parallel for reduction(+ : s)
    for (int i = 0; i < n; i++) s += a[i] * b[i];
    return s;
}

/* Textbook Jacobi-preconditioned CG (Sec. 2.2 uses a PCG; the Jacobi
 * preconditioner M = diag(A) is the reading taken for this path).
 * Stops when ||b - A x||_2 (recursive residual) <= tol * ||b||_2.
 * Returns iterations, or -1 if max_it is reached, -2 on a non-finite value. */
static int pcg_jacobi(int n, const int *rp, const int *col, const double *val, const double *diag,
                      const double *b, double *x, double tol, int max_it, double *res_out)
{
    double *r = (double *)malloc(sizeof(double) * n), *z = (double *)malloc(sizeof(double) * n);
    double *p = (double *)malloc(sizeof(double) * n), *q = (double *)malloc(sizeof(double) * n);
    csr_spmv(n, rp, col, val, x, q);
#pragma omp parallel for
    for (int i = 0; i < n; i++) r[i] = b[i] - q[i];
    double bnorm = sqrt(dot(n, b, b));
    double rnorm = sqrt(dot(n, r, r));
    int it = 0, status = 0;
    if (!(rnorm <= tol * bnorm)) {
#pragma omp parallel for
        for (int i = 0; i < n; i++) { z[i] = r[i] / diag[i]; p[i] = z[i]; }
        double rz = dot(n, r, z);
        for (it = 1; it <= max_it; it++) {
            csr_spmv(n, rp, col, val, p, q);
            double pq = dot(n, p, q);
            double alpha = rz / pq;
#pragma omp parallel for
            for (int i = 0; i < n; i++) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
            rnorm = sqrt(dot(n, r, r));
            if (!isfinite(rnorm)) { status = -2; break; }
            if (rnorm <= tol * bnorm) break;
#pragma omp parallel for
            for (int i = 0; i < n; i++) z[i] = r[i] / diag[i];
            double rz_new = dot(n, r, z);
            double beta = rz_new / rz;
            rz = rz_new;
#pragma omp parallel for
            for (int i = 0; i < n; i++) p[i] = z[i] + beta * p[i];
        }
        if (status == 0 && it > max_it) status = -1;
    }
    if (res_out) *res_out = rnorm;
    free(r); free(z); free(p); free(q);
    return status ? status : it;
}

/* PCG with the diagonal incomplete Cholesky (DIC) preconditioner of Sec. 2.2:
 * with L the strictly lower part of A in the elimination order and D the
 * diagonal with d_a = a_aa - sum_{b before a} a_ab^2 / d_b, M = (D + L) D^{-1}
 * (D + L^T) has the diagonal of A and the couplings of A.  z = M^{-1} r by a
 * forward sweep (D + L) u = r and a backward sweep (D + L^T) z = D u.  order:
 * the compact cells in elimination order; rank: the inverse permutation.
 * The rest is the textbook PCG of pcg_jacobi. */
static int pcg_dic(int n, const int *rp, const int *col, const double *val, const double *b, double *x,
                   double tol, int max_it, const int *order, const int *rank, double *res_out)
{
    double *d = (double *)malloc(sizeof(double) * n), *u = (double *)malloc(sizeof(double) * n);
    double *r = (double *)malloc(sizeof(double) * n), *z = (double *)malloc(sizeof(double) * n);
    double *p = (double *)malloc(sizeof(double) * n), *q = (double *)malloc(sizeof(double) * n);
    int status = 0, it = 0;
    /* D: the pivots of the incomplete factorisation */
    for (int o = 0; o < n && !status; o++) {
        int a = order[o];
        double s = 0.0, aa = 0.0;
        for (int e = rp[a]; e < rp[a + 1]; e++) {
            int c = col[e];
            if (c == a) aa = val[e];
            else if (rank[c] < rank[a]) s += val[e] * val[e] / d[c];
        }
        d[a] = aa - s;
        if (!(d[a] > 0.0)) status = -2;
    }
    double rnorm = 0.0;
    if (!status) {
        csr_spmv(n, rp, col, val, x, q);
        for (int i = 0; i < n; i++) r[i] = b[i] - q[i];
        double bnorm = sqrt(dot(n, b, b));
        rnorm = sqrt(dot(n, r, r));
        double rz = 0.0;
        for (it = 0; it <= max_it; it++) {
            if (rnorm <= tol * bnorm) break;
            if (it == max_it) { status = -1; break; }
            /* z = M^{-1} r */
            for (int o = 0; o < n; o++) {
                int a = order[o];
                double s = r[a];
                for (int e = rp[a]; e < rp[a + 1]; e++)
                    if (col[e] != a && rank[col[e]] < rank[a]) s -= val[e] * u[col[e]];
                u[a] = s / d[a];
            }
            for (int o = n - 1; o >= 0; o--) {
                int a = order[o];
                double s = 0.0;
                for (int e = rp[a]; e < rp[a + 1]; e++)
                    if (col[e] != a && rank[col[e]] > rank[a]) s += val[e] * z[col[e]];
                z[a] = u[a] - s / d[a];
            }
            double rz_new = dot(n, r, z);
            if (it == 0) for (int i = 0; i < n; i++) p[i] = z[i];
            else {
                double beta = rz_new / rz;
                for (int i = 0; i < n; i++) p[i] = z[i] + beta * p[i];
            }
            rz = rz_new;
            csr_spmv(n, rp, col, val, p, q);
            double alpha = rz / dot(n, p, q);
            for (int i = 0; i < n; i++) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
            rnorm = sqrt(dot(n, r, r));
            if (!isfinite(rnorm)) { status = -2; break; }
        }
    }
    if (res_out) *res_out = rnorm;
    free(d); free(u); free(r); free(z); free(p); free(q);
    return status ? status : it;
}

/* Elimination order of the compact cells: natural (cell index), or red-black
 * (cells with i + j + k even first, each colour in cell index order). */
static void dic_order(const or_problem *P, int red_black, int *order, int *rank)
{
    int o = 0;
    for (int pass = 0; pass < (red_black ? 2 : 1); pass++)
        for (int a = 0; a < P->na; a++) {
            int c = P->cell[a];
            int i = c % P->nx, j = (c / P->nx) % P->ny, k = c / (P->nx * P->ny);
            if (!red_black || ((i + j + k) & 1) == pass) order[o++] = a;
        }
    for (int q = 0; q < P->na; q++) rank[order[q]] = q;
}

/* One linear solve of an assembled system with the problem's solver. */
static int solve_system(const or_problem *P, int method, const or_system *S, double *x, double *res_out);

/* Dense Cholesky solve of the same system (tiny grids only): A = L L^T. */
static int dense_cholesky(int n, const int *rp, const int *col, const double *val, const double *b, double *x)
{
    double *M = (double *)calloc((size_t)n * n, sizeof(double));
    for (int r = 0; r < n; r++)
        for (int e = rp[r]; e < rp[r + 1]; e++) M[(size_t)r * n + col[e]] = val[e];
    for (int j = 0; j < n; j++) {
        double s = M[(size_t)j * n + j];
        for (int k = 0; k < j; k++) s -= M[(size_t)j * n + k] * M[(size_t)j * n + k];
        if (!(s > 0.0)) { free(M); return -2; }
        double Ljj = sqrt(s);
        M[(size_t)j * n + j] = Ljj;
        for (int i = j + 1; i < n; i++) {
            double u = M[(size_t)i * n + j];
            for (int k = 0; k < j; k++) u -= M[(size_t)i * n + k] * M[(size_t)j * n + k];
            M[(size_t)i * n + j] = u / Ljj;
        }
    }
    for (int i = 0; i < n; i++) {            /* L y = b */
        double s = b[i];
        for (int k = 0; k < i; k++) s -= M[(size_t)i * n + k] * x[k];
        x[i] = s / M[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; i--) {       /* L^T x = y */
        double s = x[i];
        for (int k = i + 1; k < n; k++) s -= M[(size_t)k * n + i] * x[k];
        x[i] = s / M[(size_t)i * n + i];
    }
    free(M);
    return 1;
}

/* ------------------------------------------------------------------------ */
/* One Picard attempt at a given dt (Sec. 2.2, exit test of Sec. 2.3).       */
/* ------------------------------------------------------------------------ */
typedef struct {
    int converged, picard, cg, status;
    double max_dh;
    double lin_change, bnd_in, bnd_out, defect;   /* mass balance (m^3) */
} or_attempt;

static void attempt(const or_problem *P, double dt, double *hk_out, or_attempt *R)
{
    const int na = P->na;
    or_system S;
    sys_alloc(&S, na);
    double *hk = (double *)malloc(sizeof(double) * P->N);
    double *x = (double *)malloc(sizeof(double) * na);
    memcpy(hk, P->h, sizeof(double) * P->N);
    memset(R, 0, sizeof(*R));
    for (int it = 1; it <= P->n_max; it++) {
        assemble(P, hk, P->h, dt, P->t, &S);
#pragma omp parallel for
        for (int a = 0; a < na; a++) x[a] = hk[P->cell[a]];
        int cg;
        cg = solve_system(P, P->solver, &S, x, NULL);
        R->picard = it;
        if (cg < 0) { R->status = OR_ERR_CG; break; }
        R->cg += cg;
        double dh = 0.0;
        int finite = 1;
#pragma omp parallel for reduction(max : dh) reduction(min : finite)
        for (int a = 0; a < na; a++) {
            double e = fabs(x[a] - hk[P->cell[a]]);
            if (!isfinite(x[a])) finite = 0;
            if (e > dh) dh = e;
        }
#pragma omp parallel for
        for (int a = 0; a < na; a++) hk[P->cell[a]] = x[a];
        R->max_dh = dh;
        if (!finite) { R->status = OR_ERR_CG; break; }
        if (dh <= P->tol_picard) {
            R->converged = 1;
            /* mass balance of the last linear system (interior fluxes cancel) */
            const double V = P->dx * P->dy * P->dz;
            double lin = 0.0, bin = 0.0, bout = 0.0, ds = 0.0;
#pragma omp parallel for reduction(+ : lin, bin, bout, ds)
            for (int a = 0; a < na; a++) {
                int p = P->cell[a];
                /* storage of the solved system: c (x - h^n), or for modified
                 * Picard c (x - h^k) + V (theta*^k - theta*^n) / dt (= c x - s0) */
                if (P->picard_form == 1) lin += dt * (S.c[a] * x[a] - S.s0[a]);
                else lin += S.c[a] * dt * (x[a] - P->h[p]);
                for (int f = 0; f < 6; f++) {
                    double fl = S.fa[6 * a + f] + S.fb[6 * a + f] * x[a];
                    if (fl > 0) bin += dt * fl; else bout -= dt * fl;
                }
                double th1, th0, K_, C_;
                closure(&P->zones[P->zone[p]], P->Ks[p], x[a], &th1, &K_, &C_);
                closure(&P->zones[P->zone[p]], P->Ks[p], P->h[p], &th0, &K_, &C_);
                ds += V * (th1 - th0);
            }
            R->lin_change = lin;
            R->bnd_in = bin;
            R->bnd_out = bout;
            R->defect = ds - (bin - bout);
            break;
        }
    }
    if (!R->converged && R->status == 0) R->status = OR_ERR_PICARD;
    memcpy(hk_out, hk, sizeof(double) * P->N);
    free(hk); free(x);
    sys_free(&S);
}

/* next breakpoint of any boundary series strictly after t (or +inf) */
static double next_breakpoint(const or_problem *P, double t)
{
    double nb = INFINITY;
    for (int f = 0; f < OR_NFACES; f++)
        for (int i = 0; i < P->bc[f].n; i++)
            if (P->bc[f].t[i] > t + t_tol(t) && P->bc[f].t[i] < nb) nb = P->bc[f].t[i];
    return nb;
}

/* EBATS controller after an accepted step (Sec. 2.2): count consecutive
 * accepted steps with at most n_small Picard iterations; after n_inc of them
 * multiply the nominal dt by f_grow (capped at dt_max) and restart the count.
 * A rejection divides the attempted dt by f_shrink and resets the count. */
void or_ebats_accept(double *dt_nom, int *easy, int picard, int n_small, int n_inc,
                     double f_grow, double dt_max)
{
    if (picard <= n_small) (*easy)++;
    else *easy = 0;
    if (*easy >= n_inc) {
        *dt_nom = *dt_nom * f_grow;
        if (*dt_nom > dt_max) *dt_nom = dt_max;
        *easy = 0;
    }
}

void or_ebats_reject(double *dt_nom, int *easy, double dt_attempted, double f_shrink)
{
    *dt_nom = dt_attempted / f_shrink;
    *easy = 0;
}

/* One accepted step, with EBATS reruns; t_stop clips the step (INFINITY for
 * none).  info: dt, t, picard, cg, rejected, max_dh.  All-or-nothing: on an
 * error the state is left as it was. */
static int do_step(or_problem *P, double t_stop, double *info)
{
    double dt_nom0 = P->dt_nom;
    int easy0 = P->easy, rejected = 0, cg_total = 0;
    double *hk = (double *)malloc(sizeof(double) * P->N);
    for (;;) {
        double dt = P->dt_nom;
        double bp = next_breakpoint(P, P->t);
        if (bp - P->t < dt) dt = bp - P->t;
        if (t_stop - P->t < dt) dt = t_stop - P->t;
        or_attempt R;
        attempt(P, dt, hk, &R);
        cg_total += R.cg;
        if (R.converged) {
            if (P->time_scheme == 1) {
                memcpy(P->h_prev, P->h, sizeof(double) * P->N);
                P->dt_prev = dt;
            }
            memcpy(P->h, hk, sizeof(double) * P->N);
            double tn = P->t + dt;
            if (fabs(tn - bp) <= t_tol(tn)) tn = bp;
            if (fabs(tn - t_stop) <= t_tol(tn)) tn = t_stop;
            P->t = tn;
            P->inflow_cum += R.bnd_in;
            P->outflow_cum += R.bnd_out;
            P->closure_cum += R.lin_change - (R.bnd_in - R.bnd_out);
            P->defect_cum += R.defect;
            or_ebats_accept(&P->dt_nom, &P->easy, R.picard, P->n_small, P->n_inc, P->f_grow, P->dt_max);
            if (info) {
                info[0] = dt; info[1] = P->t; info[2] = R.picard; info[3] = cg_total;
                info[4] = rejected; info[5] = R.max_dh;
            }
            free(hk);
            return OR_OK;
        }
        rejected++;
        or_ebats_reject(&P->dt_nom, &P->easy, dt, P->f_shrink);
        if (P->dt_nom < P->dt_min) {
            P->dt_nom = dt_nom0;
            P->easy = easy0;
            free(hk);
            return OR_ERR_DT_MIN;
        }
    }
}

/* The Richardson alternative to EBATS that Sec. 2.2 names for prescribing
 * the temporal error: each step is taken once with dt and twice with dt/2
 * from the same state; the difference of the two results estimates the
 * local error of the dt step (backward Euler: O(dt^2)).  The step is
 * accepted, with the more accurate two-half-step result, when the estimate
 * is within tol_time; either way the next dt is dt * 0.9 sqrt(tol_time / err)
 * (clamped to [0.2, 2] and to dt_max).  A Picard failure in any of the three
 * solves divides dt by f_shrink as in EBATS. */
static int do_step_richardson(or_problem *P, double t_stop, double *info)
{
    const double dt_nom0 = P->dt_nom, t0 = P->t;
    const size_t nb = sizeof(double) * P->N;
    int rejected = 0, cg_total = 0, pic_total = 0;
    double *h0 = (double *)malloc(nb), *hf = (double *)malloc(nb), *hm = (double *)malloc(nb),
           *h2 = (double *)malloc(nb);
    memcpy(h0, P->h, nb);
    int status = OR_OK;
    for (;;) {
        double dt = P->dt_nom;
        const double bp = next_breakpoint(P, t0);
        if (bp - t0 < dt) dt = bp - t0;
        if (t_stop - t0 < dt) dt = t_stop - t0;
        or_attempt Rf, R1, R2;
        memset(&R1, 0, sizeof(R1));
        memset(&R2, 0, sizeof(R2));
        attempt(P, dt, hf, &Rf);
        cg_total += Rf.cg; pic_total += Rf.picard;
        int ok = Rf.converged;
        if (ok) {
            attempt(P, 0.5 * dt, hm, &R1);
            cg_total += R1.cg; pic_total += R1.picard;
            ok = R1.converged;
        }
        if (ok) {
            memcpy(P->h, hm, nb);
            P->t = t0 + 0.5 * dt;
            attempt(P, 0.5 * dt, h2, &R2);
            memcpy(P->h, h0, nb);
            P->t = t0;
            cg_total += R2.cg; pic_total += R2.picard;
            ok = R2.converged;
        }
        if (!ok) {
            rejected++;
            P->dt_nom = dt / P->f_shrink;
            if (P->dt_nom < P->dt_min) { P->dt_nom = dt_nom0; status = OR_ERR_DT_MIN; break; }
            continue;
        }
        double err = 0.0;
        for (int a = 0; a < P->na; a++) {
            const int c = P->cell[a];
            const double e = fabs(h2[c] - hf[c]);
            if (e > err) err = e;
        }
        double fac = err > 0.0 ? 0.9 * sqrt(P->tol_time / err) : 2.0;
        if (fac > 2.0) fac = 2.0;
        if (fac < 0.2) fac = 0.2;
        P->dt_nom = dt * fac < P->dt_max ? dt * fac : P->dt_max;
        P->err_last = err;
        if (err > P->tol_time) {
            rejected++;
            if (P->dt_nom < P->dt_min) { P->dt_nom = dt_nom0; status = OR_ERR_DT_MIN; break; }
            continue;
        }
        if (err > P->err_max) P->err_max = err;
        memcpy(P->h, h2, nb);
        double tn = t0 + dt;
        if (fabs(tn - bp) <= t_tol(tn)) tn = bp;
        if (fabs(tn - t_stop) <= t_tol(tn)) tn = t_stop;
        P->t = tn;
        P->inflow_cum += R1.bnd_in + R2.bnd_in;
        P->outflow_cum += R1.bnd_out + R2.bnd_out;
        P->closure_cum += (R1.lin_change - (R1.bnd_in - R1.bnd_out)) + (R2.lin_change - (R2.bnd_in - R2.bnd_out));
        P->defect_cum += R1.defect + R2.defect;
        if (info) {
            info[0] = dt; info[1] = P->t; info[2] = pic_total; info[3] = cg_total;
            info[4] = rejected; info[5] = R2.max_dh;
        }
        break;
    }
    free(h0); free(hf); free(hm); free(h2);
    return status;
}

double or_time_error(const or_problem *P, int which) { return which ? P->err_max : P->err_last; }

/* BDF2 runs in the mixed (modified Picard) form, under EBATS */
static int scheme_ok(const or_problem *P)
{
    return P->time_scheme == 0 || (P->time_scheme == 1 && P->picard_form == 1 && P->time_control == 0);
}

int or_step(or_problem *P, double *info)
{
    if (!scheme_ok(P)) return OR_ERR_ARG;
    return P->time_control == 1 ? do_step_richardson(P, INFINITY, info) : do_step(P, INFINITY, info);
}

/* Advance to t_end.  log: up to log_cap rows of the 6 step-info values. */
int or_run(or_problem *P, double t_end, double *log, int log_cap, int *n_steps)
{
    int ns = 0;
    if (!scheme_ok(P)) return OR_ERR_ARG;
    while (P->t < t_end - t_tol(t_end)) {
        double info[6];
        int st = P->time_control == 1 ? do_step_richardson(P, t_end, info) : do_step(P, t_end, info);
        if (st) { if (n_steps) *n_steps = ns; return st; }
        if (log && ns < log_cap) memcpy(&log[6 * ns], info, sizeof(info));
        ns++;
    }
    if (n_steps) *n_steps = ns;
    return OR_OK;
}

/* storage0, storage, inflow_cum, outflow_cum, closure_abs, closure_rel,
 * nonlinear_defect_cum (volumes in m^3) */
void or_mass_balance(const or_problem *P, double *out7)
{
    double st = storage_of(P, P->h);
    out7[0] = P->storage0;
    out7[1] = st;
    out7[2] = P->inflow_cum;
    out7[3] = P->outflow_cum;
    out7[4] = fabs(P->closure_cum);
    out7[5] = fabs(P->closure_cum) / (P->storage0 + P->inflow_cum + P->outflow_cum);
    out7[6] = P->defect_cum;
}

/* ------------------------------------------------------------------------ */
/* Kernel-level entry points used by the parity tests.                       */
/* ------------------------------------------------------------------------ */

/* Assemble at (h^k, h^n, dt, t) and return, per active cell, K(h^k),
 * theta*(h^k), c = V C^k/dt, b and diag; optionally the CSR matrix
 * (row_ptr: na+1, col/val: up to 7 na; nnz written to *nnz). */
int or_assemble(or_problem *P, const double *hk, const double *hn, double dt, double t,
                double *K, double *theta, double *c, double *b, double *diag,
                int *row_ptr, int *col, double *val, int *nnz)
{
    or_system S;
    sys_alloc(&S, P->na);
    assemble(P, hk, hn, dt, t, &S);
    int na = P->na;
    if (K) memcpy(K, S.K, sizeof(double) * na);
    if (theta) memcpy(theta, S.theta, sizeof(double) * na);
    if (c) memcpy(c, S.c, sizeof(double) * na);
    if (b) memcpy(b, S.b, sizeof(double) * na);
    if (diag) memcpy(diag, S.diag, sizeof(double) * na);
    if (row_ptr) memcpy(row_ptr, S.row_ptr, sizeof(int) * (na + 1));
    if (col) memcpy(col, S.col, sizeof(int) * S.nnz);
    if (val) memcpy(val, S.val, sizeof(double) * S.nnz);
    if (nnz) *nnz = S.nnz;
    sys_free(&S);
    return OR_OK;
}

static int solve_system(const or_problem *P, int method, const or_system *S, double *x, double *res_out)
{
    if (method == OR_SOLVER_DENSE) return dense_cholesky(P->na, S->row_ptr, S->col, S->val, S->b, x);
    if (method == OR_SOLVER_DIC || method == OR_SOLVER_DIC_RB) {
        int *order = (int *)malloc(sizeof(int) * (P->na ? P->na : 1));
        int *rank = (int *)malloc(sizeof(int) * (P->na ? P->na : 1));
        dic_order(P, method == OR_SOLVER_DIC_RB, order, rank);
        int r = pcg_dic(P->na, S->row_ptr, S->col, S->val, S->b, x, P->tol_cg, P->cg_max_it, order, rank,
                        res_out);
        free(order);
        free(rank);
        return r;
    }
    return pcg_jacobi(P->na, S->row_ptr, S->col, S->val, S->diag, S->b, x, P->tol_cg, P->cg_max_it, res_out);
}

/* Solve A x = b for the system assembled at (h^k, h^n, dt, t) with method
 * (an OR_SOLVER_* value); x holds x0 on entry (compact active order).
 * Returns iterations (PCG) or a negative code. */
int or_solve(or_problem *P, const double *hk, const double *hn, double dt, double t,
             double *x, int method, double *res_out)
{
    or_system S;
    sys_alloc(&S, P->na);
    assemble(P, hk, hn, dt, t, &S);
    int r = solve_system(P, method, &S, x, res_out);
    sys_free(&S);
    return r;
}

/* y = A x with A assembled at (h^k, h^n, dt, t). */
int or_spmv(or_problem *P, const double *hk, const double *hn, double dt, double t,
            const double *x, double *y)
{
    or_system S;
    sys_alloc(&S, P->na);
    assemble(P, hk, hn, dt, t, &S);
    csr_spmv(P->na, S.row_ptr, S.col, S.val, x, y);
    sys_free(&S);
    return OR_OK;
}

void or_active_cells(const or_problem *P, int *cells) { memcpy(cells, P->cell, sizeof(int) * P->na); }
