// dic.cuh -- diagonal incomplete Cholesky preconditioner of the FP32 inner
// PCG, cells eliminated in red-black order.
#pragma once

#include "rf_internal.cuh"

namespace rf {

// Pivots of the factorisation for the FP32 operator of this assembly (K32,
// cb32): diag32 <- diag(A), rd32 <- 1 / pivot (0 on inactive cells).
void launch_dic_setup(cudaStream_t s, int nblk, const Grid &g, const float *K32, const float *cb32, float *diag32,
                      float *rd32, const int *skip);
// z <- M^{-1} r (three half-grid passes); nothing when *done.
void launch_dic_apply(cudaStream_t s, int nblk, const Grid &g, const float *K32, const float *rd32, const float *r,
                      float *z, const int *done);

}  // namespace rf
