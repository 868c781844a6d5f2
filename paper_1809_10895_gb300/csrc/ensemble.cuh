// ensemble.cuh -- data structures of the batched ensemble (many independent
// instances of uneven size advanced by one persistent kernel).
#pragma once

#include "rf_internal.cuh"

namespace rf {

constexpr int ENS_THREADS = 512;   // default CTA size; 128 and 256 are the other tilings

enum { ENS_NEW = 0, ENS_RUNNING = 1, ENS_DT_MIN = 2, ENS_BUDGET = 3 };

// One instance: geometry, soil, boundary conditions, and its EBATS /
// water-balance state (kept on the device between runs).
struct EnsDesc {
    Grid g;
    DevSoil soil;
    StepParams sp;          // boundary types and values (dt, t set per attempt)
    long long off;          // first cell of the instance in the packed arrays
    double t, dt_nom;
    int easy, status;
    int hbuf, kbuf, tnbuf;  // buffers holding h, K(h), theta*(h)
    int ctas;               // CTAs that ran the instance in its last run
    long long steps, picard, cg, rejected;
    long long busy_ns;      // wall time the instance held its work unit
    double in_cum, out_cum, closure_cum, defect_cum, storage0;
};

// Packed per-cell arrays of all instances.
struct EnsBuffers {
    double *H[3], *TH[2], *K[2];
    double *Can, *c, *b, *Tx, *Ty, *Tz, *diag, *dinv;
    double *r, *z, *p[2], *q;
    float *K32, *cb32, *dinv32, *r32, *z32, *p32[2], *q32, *d32;
    float *lt_inv, *lt_c, *lt_P, *lt_Q;   // vertical-line factors (RF_PRECOND_ZLINE; null otherwise)
    float4 *lt_rs;                         // its reduced-system factors, at each segment's first cell
    uint8_t *flags, *zone;
    double *Ks;
};

struct EnsParams {
    double tol_picard, tol_cg, tol_inner, dt_max, dt_min, f_grow, f_shrink, eps_chord;
    int n_inc, n_small, n_max, cg_max_it, inner_max_it, outer_max_it;
    int zline;              // inner PCG preconditioned by the vertical-line solve
    long long step_budget;
};

// Schedule entry: descriptor index, plus ENS_SCHED_WIDE when the instance runs
// on a whole cluster (wide entries come first in a schedule).
constexpr int ENS_SCHED_WIDE = 1 << 30;
constexpr int ENS_SCHED_INDEX = ENS_SCHED_WIDE - 1;

cudaError_t launch_ensemble(cudaStream_t s, int cluster, int threads, int nclusters, int precision, EnsDesc *D,
                            int n_inst, const EnsBuffers &B, const EnsParams &P, const double *t_end,
                            unsigned int *queue, const int *sched);
// clusters of `cluster` CTAs of `threads` threads (128, 256 or 512) that fit
// on the device at once (0 when none fits)
int ensemble_max_clusters(int cluster, int threads, int precision);

}  // namespace rf
