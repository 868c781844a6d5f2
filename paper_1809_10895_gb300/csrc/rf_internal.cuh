// rf_internal.cuh -- device data structures and launch helpers shared by the
// CUDA translation units of the solver (closures/assembly, PCG, host driver).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rf {

// Face order used everywhere: 0 -x, 1 +x, 2 -y, 3 +y, 4 -z (bottom), 5 +z (top).
enum { F_XMIN = 0, F_XMAX, F_YMIN, F_YMAX, F_ZMIN, F_ZMAX };
enum { BC_ZERO_FLUX = 0, BC_DIRICHLET = 1, BC_FLUX = 2, BC_FREE_DRAINAGE = 3, BC_SEEPAGE = 4 };
enum { M_VG = 0, M_GARDNER = 1 };

// Per-cell flag byte: bit f (0..5) = face f is a boundary face on which the
// boundary condition of face class f applies; bit 7 = active cell.
constexpr uint8_t FLAG_ACTIVE = 0x80;

struct DevSoil {
    int model;
    double theta_r, theta_s, alpha, n, m, S;
};

struct Grid {
    int nx, ny, nz;
    long long N;      // nx*ny*nz
    long long sxy;    // nx*ny
    double V;         // cell volume
    double A[6];      // face areas
    double w[6];      // A/d for interior faces
    double wb[6];     // A/(d/2) for boundary (half-cell) faces
    float w32[3];     // A/d per axis, FP32 (mixed-precision operator)
};

// Values that change per step attempt; lives in device memory so kernels can
// be replayed from a CUDA graph.
struct StepParams {
    double dt, t, eps_chord;
    int bc_type[6];
    double bc_val[6];
};

// Device-side scalars of one PCG solve.
struct CgScal {
    double rho;       // r.z
    double pq;        // p.q
    double alpha, beta;
    double rr;        // ||r||^2 (recursive)
    double stop2;     // converged when rr <= stop2
    double bb;        // ||b||^2 (FP64) / ||r0||^2 (inner)
    int iter;
    int done;
    int status;       // 0 ok/converged, 1 max_it, 2 non-finite/breakdown
    int max_it;
};

enum { CG_OK = 0, CG_MAXIT = 1, CG_NONFINITE = 2 };

// Reduction workspace: per-block partials, a ticket counter and results.
struct RedBuf {
    double *partials;     // nblocks * 8 doubles
    unsigned int *ticket; // one counter per reduction slot
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

// ---- launch entry points implemented in the .cu files --------------------
void launch_closure(cudaStream_t s, int nblk, const Grid &g, const DevSoil *soils, const uint8_t *zone,
                    const double *Ks, const uint8_t *flags, const double *h, const double *hprev,
                    double *theta, double *K, double *Can, double *partials, unsigned int *ticket,
                    StepResults *res);

void launch_assemble(cudaStream_t s, int nblk, const Grid &g, const DevSoil *soils, const uint8_t *zone,
                     const double *Ks, const uint8_t *flags, const StepParams *sp, const double *hk,
                     const double *hn, const double *theta_k, const double *theta_n, const double *K,
                     const double *Can, double *c, double *b, double *Tx, double *Ty, double *Tz,
                     double *diag, double *dinv, float *K32, float *cb32, float *dinv32);

void launch_mass_balance(cudaStream_t s, int nblk, const Grid &g, const DevSoil *soils, const uint8_t *zone,
                         const double *Ks, const uint8_t *flags, const StepParams *sp, const double *x,
                         const double *hn, const double *c, const double *Kold, const double *theta_x,
                         const double *theta_n, double *partials, unsigned int *ticket, StepResults *res);

void launch_storage(cudaStream_t s, int nblk, const Grid &g, const uint8_t *flags, const double *theta,
                    double *partials, unsigned int *ticket, StepResults *res);

// FP64 PCG (Jacobi), stored face coefficients.
void launch_cg64_init(cudaStream_t s, int nblk, const Grid &g, const uint8_t *flags, const double *x0,
                      double *x, const double *b, const double *Tx, const double *Ty, const double *Tz,
                      const double *diag, const double *dinv, double *r, double *z, double tol,
                      int max_it, double *partials, unsigned int *ticket, CgScal *sc);
void launch_cg64_spmv(cudaStream_t s, int nblk, const Grid &g, const uint8_t *flags, const double *z,
                      const double *p_in, double *p_out, double *q, const double *Tx, const double *Ty,
                      const double *Tz, const double *diag, double *partials, unsigned int *ticket, CgScal *sc);
void launch_cg64_update(cudaStream_t s, int nblk, const Grid &g, double *x, double *r, double *z,
                        const double *p, const double *q, const double *dinv, double *partials,
                        unsigned int *ticket, CgScal *sc);
void launch_apply64(cudaStream_t s, int nblk, const Grid &g, const uint8_t *flags, const double *x, double *y,
                    const double *Tx, const double *Ty, const double *Tz, const double *diag);

// Mixed precision: FP64 outer residual + FP32 inner PCG (recomputed faces).
void launch_resid64(cudaStream_t s, int nblk, const Grid &g, const uint8_t *flags, const double *x,
                    const double *b, const double *Tx, const double *Ty, const double *Tz,
                    const double *diag, const float *dinv32, float *r32, float *z32, float *d32,
                    double tol, double tol_inner, int inner_max_it, double *partials,
                    unsigned int *ticket, CgScal *outer, CgScal *inner);
void launch_cg32_spmv(cudaStream_t s, int nblk, const Grid &g, const float *z, const float *p_in, float *p_out,
                      float *q, const float *K32, const float *cb32, double *partials, unsigned int *ticket,
                      CgScal *sc);
void launch_cg32_update(cudaStream_t s, int nblk, const Grid &g, float *x, float *r, float *z, const float *p,
                        const float *q, const float *dinv, double *partials, unsigned int *ticket, CgScal *sc);
void launch_add_correction(cudaStream_t s, int nblk, const Grid &g, double *x, const float *d);

}  // namespace rf
