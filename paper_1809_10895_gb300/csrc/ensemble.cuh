// ensemble.cuh -- data structures of the batched ensemble (many independent
// instances of uneven size advanced by one persistent kernel).
#pragma once

#include "rf_internal.cuh"

namespace rf {

constexpr int ENS_THREADS = 512;

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
    int pad;
    long long steps, picard, cg, rejected;
    double in_cum, out_cum, closure_cum, defect_cum, storage0;
};

// Packed per-cell arrays of all instances.
struct EnsBuffers {
    double *H[3], *TH[2], *K[2];
    double *Can, *c, *b, *Tx, *Ty, *Tz, *diag, *dinv;
    double *r, *z, *p[2], *q;
    float *K32, *cb32, *dinv32, *r32, *z32, *p32[2], *q32, *d32;
    uint8_t *flags, *zone;
    double *Ks;
};

struct EnsParams {
    double tol_picard, tol_cg, tol_inner, dt_max, dt_min, f_grow, f_shrink, eps_chord;
    int n_inc, n_small, n_max, cg_max_it, inner_max_it, outer_max_it;
    long long step_budget;
};

cudaError_t launch_ensemble(cudaStream_t s, int cluster, int nclusters, int precision, EnsDesc *D, int n_inst,
                            const EnsBuffers &B, const EnsParams &P, const double *t_end, unsigned int *queue);
// clusters of `cluster` CTAs that fit on the device at once
int ensemble_max_clusters(int cluster, int precision);

}  // namespace rf
