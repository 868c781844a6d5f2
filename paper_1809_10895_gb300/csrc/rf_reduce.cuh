// rf_reduce.cuh -- deterministic block and grid reductions.
//
// Every reduction is two-level: each block reduces its threads' values with a
// fixed XOR-shuffle tree and writes one partial per value to
// partials[i * gridDim.x + blockIdx.x]; the last block to finish (found with
// an atomic ticket after a memory fence) folds the partials in a fixed order.
// With a fixed grid size the result is bit-reproducible run to run.
#pragma once

#include <cuda_runtime.h>

namespace rf {

struct OpSum {
    __device__ static double id() { return 0.0; }
    __device__ static double op(double a, double b) { return a + b; }
};
struct OpMax {
    __device__ static double id() { return 0.0; }   // values reduced with max are >= 0
    __device__ static double op(double a, double b) { return a > b ? a : b; }
};

template <class Op>
__device__ __forceinline__ double warp_reduce(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = Op::op(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Reduce NV values over the block; the totals are returned in warp 0 (all
// lanes).  sm must hold NV*32 doubles.  Contains __syncthreads().
template <class Op, int NV>
__device__ __forceinline__ void block_reduce(double (&v)[NV], double *sm)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; i++) v[i] = warp_reduce<Op>(v[i]);
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < NV; i++) sm[i * 32 + wid] = v[i];
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int i = 0; i < NV; i++) {
            double t = lane < nw ? sm[i * 32 + lane] : Op::id();
            v[i] = warp_reduce<Op>(t);
        }
    }
    __syncthreads();
}

// Grid-level reduction.  Every block calls this with its thread values; the
// function returns true in exactly one block (the last), whose warp 0 then
// holds the grid totals in v.  partials: NV * gridDim.x doubles.
template <class Op, int NV>
__device__ __forceinline__ bool grid_reduce(double (&v)[NV], double *partials, unsigned int *ticket)
{
    __shared__ double sm[NV * 32];
    __shared__ bool am_last;
    block_reduce<Op, NV>(v, sm);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < NV; i++) partials[i * gridDim.x + blockIdx.x] = v[i];
        __threadfence();
        unsigned int t = atomicInc(ticket, gridDim.x - 1);   // wraps to 0 for the next use
        am_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!am_last) return false;
    __threadfence();
#pragma unroll
    for (int i = 0; i < NV; i++) {
        double t = Op::id();
        for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) t = Op::op(t, __ldcg(&partials[i * gridDim.x + b]));
        v[i] = t;
    }
    block_reduce<Op, NV>(v, sm);
    return true;
}

// Grid-level sum of float thread values: warp and block levels in FP32 (no
// FP64 instructions per thread), the cross-block fold in FP64.  Same
// contract as grid_reduce.
template <int NV>
__device__ __forceinline__ bool grid_reduce_f32(float (&vf)[NV], double (&v)[NV], double *partials,
                                                unsigned int *ticket)
{
    __shared__ float smf[NV * 32];
    __shared__ double sm[NV * 32];
    __shared__ bool am_last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; i++) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) vf[i] += __shfl_xor_sync(0xffffffffu, vf[i], o);
    }
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < NV; i++) smf[i * 32 + wid] = vf[i];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < NV; i++) {
            float t = 0.0f;
            for (int w = 0; w < nw; w++) t += smf[i * 32 + w];
            partials[i * gridDim.x + blockIdx.x] = (double)t;
        }
        __threadfence();
        unsigned int t = atomicInc(ticket, gridDim.x - 1);
        am_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!am_last) return false;
    __threadfence();
#pragma unroll
    for (int i = 0; i < NV; i++) {
        double t = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) t += __ldcg(&partials[i * gridDim.x + b]);
        v[i] = t;
    }
    block_reduce<OpSum, NV>(v, sm);
    return true;
}

}  // namespace rf
