// dic.cu -- diagonal incomplete Cholesky (DIC) preconditioner for the FP32
// inner PCG.  Sec. 2.2 solves each Picard system with DIC-preconditioned CG;
// a sequential code eliminates the cells in index order, which serialises
// the triangular sweeps.  Here the cells are eliminated in red-black order
// (colour (i + j + k) mod 2, red = even first): every neighbour of a cell in
// the 7-point stencil has the other colour, so each sweep is two
// data-parallel half-grid passes.
//
// With L the strictly lower part of A in that order and D the pivots,
// M = (D + L) D^{-1} (D + L^T):
//   red pivots     d_r = a_rr                       (no earlier neighbour)
//   black pivots   d_b = a_bb - sum_j T_bj^2 / a_jj (all neighbours are red)
// and z = M^{-1} r by
//   red    u_r = r_r / d_r
//   black  z_b = (r_b + sum_j T_bj u_j) / d_b       (forward; the backward
//                                                    sweep leaves black as is)
//   red    z_r = u_r + sum_j T_rj z_j / d_r         (backward)
// with T the face coefficients of the FP32 operator, T_f = (w_f / 2)(K_P +
// K_N) over faces whose neighbour is active (K >= 0), and a_PP = cb_P +
// sum_f T_f.  A pivot that is not positive (possible only without any
// storage or boundary term in a whole neighbourhood) falls back to 1 / a_PP.
#include "dic.cuh"

namespace rf {

namespace {

__device__ __forceinline__ int colour_of(const Grid &g, long long p, int &i, int &j, int &k)
{
    cell_ijk(g, p, i, j, k);
    return (i + j + k) & 1;
}

// f(q, T) for every active neighbour q of active cell p (K_P = kP)
template <class F>
__device__ __forceinline__ void active_faces(const Grid &g, const float *__restrict__ K32, long long p, int i, int j,
                                             int k, float kP, F f)
{
    auto face = [&](bool inside, long long q, float w_half) {
        if (!inside) return;
        const float kN = K32[q];
        if (kN >= 0.0f) f(q, w_half * (kP + kN));
    };
    const float wx = 0.5f * g.w32[0], wy = 0.5f * g.w32[1], wz = 0.5f * g.w32[2];
    face(i > 0, p - 1, wx);
    face(i < g.nx - 1, p + 1, wx);
    face(j > 0, p - g.nx, wy);
    face(j < g.ny - 1, p + g.nx, wy);
    face(k > 0, p - g.sxy, wz);
    face(k < g.nz - 1, p + g.sxy, wz);
}

__global__ void __launch_bounds__(RED_THREADS)
k_dic_diag(Grid g, const float *__restrict__ K32, const float *__restrict__ cb32, float *__restrict__ diag32,
           const int *skip)
{
    if (skip && *skip) return;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < g.N; p += stride) {
        const float kP = K32[p];
        if (!(kP >= 0.0f)) {
            diag32[p] = 0.0f;
            continue;
        }
        int i, j, k;
        cell_ijk(g, p, i, j, k);
        float d = cb32[p];
        active_faces(g, K32, p, i, j, k, kP, [&](long long, float t) { d += t; });
        diag32[p] = d;
    }
}

__global__ void __launch_bounds__(RED_THREADS)
k_dic_pivots(Grid g, const float *__restrict__ K32, const float *__restrict__ diag32, float *__restrict__ rd32,
             const int *skip)
{
    if (skip && *skip) return;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < g.N; p += stride) {
        const float kP = K32[p];
        const float dP = diag32[p];
        if (!(kP >= 0.0f) || !(dP > 0.0f)) {
            rd32[p] = 0.0f;
            continue;
        }
        int i, j, k;
        if (colour_of(g, p, i, j, k) == 0) {
            rd32[p] = 1.0f / dP;
            continue;
        }
        float s = dP;
        active_faces(g, K32, p, i, j, k, kP, [&](long long q, float t) { s -= t * t / diag32[q]; });
        rd32[p] = (s > 0.0f && isfinite(s)) ? 1.0f / s : 1.0f / dP;
    }
}

// pass 0: red u = rd r;  pass 1: black z = rd (r + sum T u);  pass 2: red z = u + rd sum T z
template <int PASS>
__global__ void __launch_bounds__(RED_THREADS)
k_dic_sweep(Grid g, const float *__restrict__ K32, const float *__restrict__ rd32, const float *__restrict__ r,
            float *__restrict__ z, const int *done)
{
    if (done && *done) return;
    const int want = PASS == 1 ? 1 : 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < g.N; p += stride) {
        int i, j, k;
        if (colour_of(g, p, i, j, k) != want) continue;
        const float rd = rd32[p];
        if (rd == 0.0f) {                 // inactive
            if (PASS != 2) z[p] = 0.0f;
            continue;
        }
        if (PASS == 0) {
            z[p] = rd * r[p];
            continue;
        }
        float s = PASS == 1 ? r[p] : 0.0f;
        active_faces(g, K32, p, i, j, k, K32[p], [&](long long q, float t) { s = fmaf(t, z[q], s); });
        z[p] = PASS == 1 ? rd * s : fmaf(rd, s, z[p]);
    }
}

}  // namespace

void launch_dic_setup(cudaStream_t s, int nblk, const Grid &g, const float *K32, const float *cb32, float *diag32,
                      float *rd32, const int *skip)
{
    k_dic_diag<<<nblk, RED_THREADS, 0, s>>>(g, K32, cb32, diag32, skip);
    k_dic_pivots<<<nblk, RED_THREADS, 0, s>>>(g, K32, diag32, rd32, skip);
}

void launch_dic_apply(cudaStream_t s, int nblk, const Grid &g, const float *K32, const float *rd32, const float *r,
                      float *z, const int *done)
{
    k_dic_sweep<0><<<nblk, RED_THREADS, 0, s>>>(g, K32, rd32, r, z, done);
    k_dic_sweep<1><<<nblk, RED_THREADS, 0, s>>>(g, K32, rd32, r, z, done);
    k_dic_sweep<2><<<nblk, RED_THREADS, 0, s>>>(g, K32, rd32, r, z, done);
}

}  // namespace rf
