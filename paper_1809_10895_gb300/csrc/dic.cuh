// dic.cuh -- diagonal incomplete Cholesky preconditioner of the FP32 inner
// PCG, cells eliminated in red-black order.
#pragma once

#include "rf_internal.cuh"

namespace rf {

// Pivots of the factorisation for the FP32 operator of this assembly (K32,
// cb32): diag32 <- diag(A), rd32 <- 1 / pivot (0 on inactive cells).
void launch_dic_setup(cudaStream_t s, int nblk, const Grid &g, const float *K32, const float *cb32, float *diag32,
                      float *rd32, const int *skip);

// z <- M^{-1} r finishing r.z into rho (start = 1) or beta and rho, and the
// inner loop condition (as launch_cg32_rz does after a V-cycle): the red
// pass (skipped when red_done: launch_cg32_update_dic did it), the black pass
// with the black cells' share of r.z, the red back-substitution with the rest.
void launch_dic_apply_rz(cudaStream_t s, int nblk, const Grid &g, const float *K32, const float *rd32, const float *r,
                         float *z, double *partials, unsigned int *ticket, CgScal *sc, int start, bool red_done,
                         CondSet cond);
// The inner PCG's update (as for multigrid) fused with DIC's red pass on the
// new residual.
void launch_cg32_update_dic(cudaStream_t s, int nblk, const Grid &g, float *x, float *r, float *z, const float *p,
                            const float *q, const float *dinv, const float *rd32, double *partials,
                            unsigned int *ticket, CgScal *sc);

}  // namespace rf
