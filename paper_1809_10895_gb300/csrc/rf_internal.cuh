// rf_internal.cuh -- device data structures and launch helpers shared by the
// CUDA translation units of the solver (closures/assembly, PCG, host driver).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <nvtx3/nvToolsExt.h>

#include "ff.cuh"
#include "tma.cuh"

namespace rf {

// An NVTX range over a host scope (visible to profilers that record NVTX;
// NVTX 3 is header-only and costs next to nothing when no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Face order used everywhere: 0 -x, 1 +x, 2 -y, 3 +y, 4 -z (bottom), 5 +z (top).
enum { F_XMIN = 0, F_XMAX, F_YMIN, F_YMAX, F_ZMIN, F_ZMAX };
enum { BC_ZERO_FLUX = 0, BC_DIRICHLET = 1, BC_FLUX = 2, BC_FREE_DRAINAGE = 3, BC_SEEPAGE = 4 };
enum { M_VG = 0, M_GARDNER = 1, M_BROOKS_COREY = 2 };

// Per-cell flag byte: bit f (0..5) = face f is a boundary face on which the
// boundary condition of face class f applies; bit 7 = active cell.
constexpr uint8_t FLAG_ACTIVE = 0x80;

// Division of 0 <= n < 2^31 by an invariant d >= 1 with one multiply and a
// shift (Granlund & Montgomery, "Division by invariant integers using
// multiplication", PLDI 1994): q = (n * m) >> (32 + l) with l = ceil(log2 d)
// and m = ceil(2^(32+l) / d) < 2^33; exact because n * (m d - 2^(32+l)) <
// 2^31 * d <= 2^(32+l).
struct FastDiv {
    unsigned long long m;
    int shift;      // 32 + l
    int pad;
};

inline FastDiv make_fastdiv(unsigned int d)
{
    int l = 0;
    while ((1ULL << l) < d) l++;
    const unsigned long long num = 1ULL << (32 + l);
    FastDiv f;
    f.m = (num + d - 1) / d;
    f.shift = 32 + l;
    f.pad = 0;
    return f;
}

// Kernel kinds, for the per-kind launch counters (launched / did work).
enum KernelKind {
    KK_CLOSURE = 0, KK_CLOSURE_PICARD, KK_ASSEMBLE, KK_CG64_INIT, KK_CG64_SPMV, KK_CG64_UPDATE, KK_APPLY64,
    KK_MIXED_START, KK_RESID64, KK_CG32_SPMV, KK_CG32_UPDATE, KK_ADD_CORRECTION, KK_MASS_BALANCE, KK_STORAGE,
    KK_ACCEPT, KK_COUNT
};

struct DevSoil {
    int model;
    double theta_r, theta_s, alpha, n, m, S;
    float n_hi, n_lo, m_hi, m_lo;   // n and m as double-float pairs
    double cfac;                    // ((theta_s - theta_r) alpha) n m, the factor of C (Eq. 3)
};

struct Grid {
    int nx, ny, nz;
    long long N;      // nx*ny*nz
    long long sxy;    // nx*ny
    double V;         // cell volume
    double A[6];      // face areas
    double w[6];      // A/d for interior faces
    double wb[6];     // A/(d/2) for boundary (half-cell) faces
    double hw[6];     // A/(2 d): T_f = (K_P + K_N) hw_f
    double gf[6];     // gravity flux factor of each face, grad(elevation) . n_out: (-gx, gx, -gy, gy, -gz, gz)
    double hg[6];     // gf A / 2: explicit gravity of an interior face is (K_P + K_N) hg_f
    float w32[3];     // A/d per axis, FP32 (mixed-precision operator)
    FastDiv fx, fxy;  // division by nx and by nx*ny
    int cap;          // most blocks a tiled stencil kernel launches (partials hold 8 values per block)
    int closure64;    // 1: closures in FP64 (CUDA's FP64 log / exp); 0: double-float arithmetic
    int tilted;       // 1: the elevation gradient has x / y components (gravity on lateral faces)
    int harmonic;     // 1: harmonic interface conductivity; 0: arithmetic mean (linear interpolation)
    int wait_tries;   // polls of a bounded device wait before it gives up (set for tests; 0: default)
    const FFTables *tab;       // double-float exp/log tables (device)
    unsigned long long *ctr;   // per-kind counters: [2 kind] launches, [2 kind + 1] launches that did work
};

// Values that change per step attempt; lives in device memory so kernels can
// be replayed from a CUDA graph.
struct StepParams {
    double dt, t, eps_chord;
    int bc_type[6];
    double bc_val[6];
    int modified;   // 1: modified Picard (tangent capacity, mixed-form storage); 0: chord capacity
    int bdf2;       // 1: variable-step BDF2 storage (modified form) with the coefficients below
    double a0, a1, a2;   // BDF2: V/dt [a0 theta^{n+1} - a1 theta^n + a2 theta^{n-1}]
};

// Device-side scalars of one PCG solve.
struct CgScal {
    double rho;       // r.z
    double pq;        // p.q
    double alpha, beta;
    double rr;        // ||r||^2 (recursive)
    double stop2;     // converged when ||r|| <= stop2
    double bb;        // ||b||^2 (FP64) / ||r0||^2 (inner)
    double rz_part;   // r.z over the black cells (DIC, between its two sweeps)
    int iter;         // iterations of this solve
    int done;
    int status;       // CG_OK, CG_MAXIT, CG_NONFINITE
    int max_it;
    int total;        // iterations accumulated over inner solves (mixed)
    int pad;
};

enum { CG_OK = 0, CG_MAXIT = 1, CG_NONFINITE = 2 };

// Picard-loop control for a device-resident attempt (Sec. 2.2 / 2.3).
struct PicardCtl {
    double tol;        // Picard tolerance on max|dh|
    double max_dh;     // last update
    int n_max;         // iteration cap
    int it;            // iterations done (linear solves)
    int conv, fail, done;
    int cg_total;      // CG iterations over the attempt
    int mb_pending;    // (unused)
    int pad;
};

// A conditional-node handle a kernel may set (use = 0 outside graphs).
struct CondSet {
    unsigned long long h;
    int use;
};

// Start of the linear solve fused into the assembly kernel: x = h^k and the
// first residual b - A h^k from the freshly computed face coefficients.
enum { ASM_ONLY = 0, ASM_CG64 = 1, ASM_MIXED = 2 };
struct SolveStart {
    double *x;                 // x0 = h^k copied here
    double *r, *z;             // FP64 residual and D^-1 r (ASM_CG64)
    float *r32, *z32, *d32;    // FP32 inner seeds (ASM_MIXED)
    CgScal *sc;                // FP64 solve, or the outer defect-correction loop
    CgScal *inner;             // inner FP32 solve (ASM_MIXED)
    double tol, tol_inner;
    int max_it, inner_max_it, outer_max_it;
    int pad;
    CondSet cond, cond_inner;  // loop conditions raised for the solve
};

// Results of the per-step reductions, read back by the host.
struct StepResults {
    double max_dh;
    double lin_change;   // sum V C^k (x - h^n)  (= dt * sum c (x - h^n))
    double dstore;       // sum V (theta*(x) - theta*(h^n))
    double bnd_in, bnd_out;  // dt * boundary inflow / outflow
    double storage;      // sum V theta*(h)
    int nonfinite;
    int pad;
};

constexpr int RED_THREADS = 256;

#ifdef __CUDACC__
__device__ __forceinline__ void count_launch(const Grid &g, int kind)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&g.ctr[2 * kind], 1ULL);
}
__device__ __forceinline__ void count_work(const Grid &g, int kind)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&g.ctr[2 * kind + 1], 1ULL);
}
__device__ __forceinline__ unsigned int fdiv(unsigned int n, const FastDiv &f)
{
    return (unsigned int)(((unsigned long long)n * f.m) >> f.shift);
}
// (i, j, k) of cell p (p < 2^31)
__device__ __forceinline__ void cell_ijk(const Grid &g, long long p, int &i, int &j, int &k)
{
    const unsigned int u = (unsigned int)p;
    const unsigned int kk = fdiv(u, g.fxy);
    const unsigned int r = u - kk * (unsigned int)g.sxy;
    const unsigned int jj = fdiv(r, g.fx);
    i = (int)(r - jj * (unsigned int)g.nx);
    j = (int)jj;
    k = (int)kk;
}
// 1/a to about full double precision: single-precision estimate refined by
// two Newton-Raphson steps r <- r + r (1 - a r) (each doubles the correct
// bits: 23 -> 46 -> 92).  Falls back to IEEE division outside the range in
// which the single-precision estimate is normal.
__device__ __forceinline__ double rcp64(double a)
{
    const double m = fabs(a);
    if (!(m > 1e-30 && m < 1e30)) return 1.0 / a;
    float rf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"((float)a));
    double r = (double)rf;
    double e = fma(-a, r, 1.0);
    r = fma(r, e, r);
    e = fma(-a, r, 1.0);
    return fma(r, e, r);
}
__device__ __forceinline__ void set_cond(const CondSet &c, unsigned int v)
{
    if (c.use) cudaGraphSetConditional(c.h, v);
}

// FP64 PCG start from the reduced (r.z, r.r, b.b) of the initial residual.
__device__ __forceinline__ void cg64_start_scalars(CgScal *sc, const double (&v)[3], double tol, int max_it,
                                                   const CondSet &cond)
{
    sc->rho = v[0];
    sc->rr = v[1];
    sc->bb = v[2];
    sc->stop2 = tol * sqrt(v[2]);      // threshold on ||r||_2
    sc->alpha = 0.0;
    sc->beta = 0.0;
    sc->iter = 0;
    sc->total = 0;
    sc->max_it = max_it;
    const bool finite = isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]);
    sc->status = finite ? CG_OK : CG_NONFINITE;
    sc->done = (!finite || sqrt(v[1]) <= sc->stop2) ? 1 : 0;
    set_cond(cond, sc->done ? 0 : 1);
}

// Defect correction: test of an outer FP64 residual (r.r, b.b) and seeds of
// the inner FP32 solve (r32.r32, r32.z32); outer->iter already counts this
// residual, and the solve fails after outer_max_it residuals.
__device__ __forceinline__ void outer_residual_scalars(CgScal *outer, CgScal *inner, const double (&v)[4], double tol,
                                                       double tol_inner, int inner_max_it, int outer_max_it,
                                                       const CondSet &co, const CondSet &ci)
{
    const bool finite = isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]) && isfinite(v[3]);
    outer->rr = v[0];
    outer->bb = v[1];
    outer->stop2 = tol * sqrt(v[1]);
    if (!finite) {
        outer->status = CG_NONFINITE;
        outer->done = 1;
    } else if (sqrt(v[0]) <= outer->stop2) {
        outer->done = 1;
    } else if (outer->iter >= outer_max_it) {
        outer->status = CG_MAXIT;
        outer->done = 1;
    }
    inner->rho = v[3];
    inner->rr = v[2];
    inner->bb = v[2];
    inner->stop2 = tol_inner * sqrt(v[2]);
    inner->alpha = 0.0;
    inner->beta = 0.0;
    inner->iter = 0;
    inner->max_it = inner_max_it;
    inner->status = CG_OK;
    inner->done = (outer->done || !(v[2] > 0.0)) ? 1 : 0;
    set_cond(co, outer->done ? 0 : 1);
    set_cond(ci, inner->done ? 0 : 1);
}
#endif

// Message returned by rf_last_error() on the calling thread.
void set_last_error(const char *msg);

// ---- launch entry points implemented in the .cu files --------------------
void launch_closure(cudaStream_t s, int nblk, const Grid &g, const DevSoil *soils, const uint8_t *zone,
                    const double *Ks, const uint8_t *flags, const double *h, const double *hprev,
                    double *theta, double *K, double *Can, double *partials, unsigned int *ticket,
                    StepResults *res);

// Closures at the new Picard iterate x with the exit test against h^k; ends a
// Picard iteration (updates ctl, sets the Picard loop condition).
void launch_closure_picard(cudaStream_t s, int nblk, const Grid &g, const DevSoil *soils, const uint8_t *zone,
                           const double *Ks, const uint8_t *flags, const double *x, const double *hk,
                           double *theta, double *K, double *Can, double *partials, unsigned int *ticket,
                           PicardCtl *ctl, const CgScal *cg_status, const CgScal *cg_count, CondSet cond);

void launch_assemble(cudaStream_t s, int nblk, const Grid &g, const DevSoil *soils, const uint8_t *zone,
                     const double *Ks, const uint8_t *flags, const StepParams *sp, const double *hk,
                     const double *hn, const double *theta_k, const double *theta_n, const double *K,
                     const double *Can, double *c, double *b, double *Tx, double *Ty, double *Tz,
                     double *diag, double *dinv, float *K32, float *cb32, float *dinv32, const int *skip,
                     int mode = ASM_ONLY, const SolveStart *start = nullptr, double *partials = nullptr,
                     unsigned int *ticket = nullptr, double *s0 = nullptr, const double *theta_p = nullptr);

void launch_mass_balance(cudaStream_t s, int nblk, const Grid &g, const DevSoil *soils, const uint8_t *zone,
                         const double *Ks, const uint8_t *flags, const StepParams *sp, const double *x_odd,
                         const double *x_even, const double *hn, const double *c, const double *K_odd,
                         const double *K_even, const double *theta_x, const double *theta_n, double *partials,
                         unsigned int *ticket, StepResults *res, const PicardCtl *ctl, const double *s0 = nullptr);

void launch_storage(cudaStream_t s, int nblk, const Grid &g, const uint8_t *flags, const double *theta,
                    double *partials, unsigned int *ticket, StepResults *res);

// Uploaded state src checked on the device (res->nonfinite: a non-finite head
// on an active cell) and, only when valid, committed into dst (non-finite
// values on inactive cells become 0).
void launch_state_check_commit(cudaStream_t s, int nblk, const Grid &g, const uint8_t *flags, const double *src,
                               double *dst, double *partials, unsigned int *ticket, StepResults *res);

// Accept a converged attempt: h <- x_final, theta_n <- theta_k, K0 <- K1 (copyK).
void launch_accept(cudaStream_t s, int nblk, const Grid &g, const double *x_final, double *h,
                   const double *theta_k, double *theta_n, const double *K1, double *K0, int copyK);

// FP64 PCG (Jacobi), stored face coefficients.
void launch_cg64_init(cudaStream_t s, int nblk, const Grid &g, const uint8_t *flags, const double *x0,
                      double *x, const double *b, const double *Tx, const double *Ty, const double *Tz,
                      const double *diag, const double *dinv, double *r, double *z, double tol,
                      int max_it, double *partials, unsigned int *ticket, CgScal *sc, const int *skip,
                      CondSet cond);
void launch_cg64_spmv(cudaStream_t s, int nblk, const Grid &g, const uint8_t *flags, const double *z,
                      const double *p_in, double *p_out, double *q, const double *Tx, const double *Ty,
                      const double *Tz, const double *diag, double *partials, unsigned int *ticket, CgScal *sc);
void launch_cg64_update(cudaStream_t s, int nblk, const Grid &g, double *x, double *r, double *z,
                        const double *p, const double *q, const double *dinv, double *partials,
                        unsigned int *ticket, CgScal *sc, CondSet cond);
void launch_apply64(cudaStream_t s, int nblk, const Grid &g, const uint8_t *flags, const double *x, double *y,
                    const double *Tx, const double *Ty, const double *Tz, const double *diag);

// Mixed precision: FP64 outer residual + FP32 inner PCG (recomputed faces).
void launch_mixed_start(cudaStream_t s, int nblk, const Grid &g, const double *x0, double *x, CgScal *outer,
                        CgScal *inner, const int *skip, CondSet cond_outer);
void launch_resid64(cudaStream_t s, int nblk, const Grid &g, const uint8_t *flags, const double *x,
                    const double *b, const double *Tx, const double *Ty, const double *Tz,
                    const double *diag, const float *dinv32, float *r32, float *z32, float *d32,
                    double tol, double tol_inner, int inner_max_it, int outer_max_it, double *partials,
                    unsigned int *ticket, CgScal *outer, CgScal *inner, CondSet cond_outer, CondSet cond_inner);
void launch_cg32_spmv(cudaStream_t s, int nblk, const Grid &g, const float *z, const float *p_in, float *p_out,
                      float *q, const float *K32, const float *cb32, double *partials, unsigned int *ticket,
                      CgScal *sc, const TmaMaps32 *tma = nullptr, int *fault = nullptr);
void launch_cg32_update(cudaStream_t s, int nblk, const Grid &g, float *x, float *r, float *z, const float *p,
                        const float *q, const float *dinv, double *partials, unsigned int *ticket, CgScal *sc,
                        CondSet cond);
void launch_add_correction(cudaStream_t s, int nblk, const Grid &g, double *x, const float *d, CgScal *outer,
                           const CgScal *inner, CondSet cond_outer);

}  // namespace rf
