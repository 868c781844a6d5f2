// mg.cuh -- geometric multigrid hierarchy for the FP32 inner PCG.
#pragma once

#include "rf_internal.cuh"

namespace rf {

constexpr int MG_MAX_LEVELS = 16;
constexpr int MG_COARSE_SWEEPS = 40;
constexpr long long MG_COARSEST_CELLS = 512;

struct MgLevel {
    int level;
    int nx, ny, nz;
    int cx, cy, cz;          // coarsening factors to the next level (1 or 2)
    long long N, sxy;
    FastDiv fx, fxy;
    float w32[3];            // level 0: A/d per axis
    float *cb;               // capacity (+ Dirichlet) term (level 0: cb32)
    float *T[3];             // upper-face coefficients (levels >= 1)
    float *dinv;             // 1/diag (levels >= 1)
    const float *dinv0;      // level 0: the PCG's dinv32
    float *r;                // restricted residual (levels >= 1)
    float *e[2];             // correction and scratch
};

struct MgHierarchy {
    int nlev = 0;
    MgLevel lev[MG_MAX_LEVELS];
};

// Level dimensions: halve the axes whose spacing is within 2x of the finest.
struct MgShape {
    int nx, ny, nz;
    double dx, dy, dz;
};
int mg_plan(int nx, int ny, int nz, double dx, double dy, double dz, MgShape *out, int cap);

void launch_mg_build(cudaStream_t s, int nblk, const MgHierarchy &H, const float *K32, const int *skip);
void launch_mg_vcycle(cudaStream_t s, int nblk, const MgHierarchy &H, const float *K32, const float *r, float *z,
                      const int *done);
int mg_vcycle_launches(const MgHierarchy &H);

// FP32 inner PCG with the V-cycle preconditioner: the update kernel leaves z
// to the V-cycle, and a dot kernel finishes the iteration (r.z, beta, loop
// condition).
void launch_cg32_update_mg(cudaStream_t s, int nblk, const Grid &g, float *x, float *r, const float *p,
                           const float *q, const float *dinv, double *partials, unsigned int *ticket, CgScal *sc);
void launch_cg32_rz(cudaStream_t s, int nblk, const Grid &g, const float *r, const float *z, double *partials,
                    unsigned int *ticket, CgScal *sc, int start, CondSet cond);

}  // namespace rf
