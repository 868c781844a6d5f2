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
#include "rf_reduce.cuh"

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

// The inner PCG's update (x += alpha p, r -= alpha q, ||r||^2 and the stop
// test, as for the multigrid path) with DIC's first pass on the new residual
// fused in: u = r / d on the red cells.  Inactive cells keep x, r and z = 0.
__global__ void __launch_bounds__(RED_THREADS)
k_cg32_update_dic(Grid g, float *__restrict__ x, float *__restrict__ r, float *__restrict__ z,
                  const float *__restrict__ pd, const float *__restrict__ q, const float *__restrict__ dinv,
                  const float *__restrict__ rd32, double *partials, unsigned int *ticket, CgScal *sc)
{
    count_launch(g, KK_CG32_UPDATE);
    if (sc->done) return;
    count_work(g, KK_CG32_UPDATE);
    const float alpha = (float)sc->alpha;
    float a0 = 0.0f;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < g.N;
         p += (long long)gridDim.x * blockDim.x) {
        if (dinv[p] == 0.0f) continue;
        x[p] = fmaf(alpha, pd[p], x[p]);
        const float rp = fmaf(-alpha, q[p], r[p]);
        r[p] = rp;
        a0 = fmaf(rp, rp, a0);
        int i, j, k;
        if (colour_of(g, p, i, j, k) == 0) z[p] = rd32[p] * rp;
    }
    float vf[1] = {a0};
    double v[1];
    if (grid_reduce_f32<1>(vf, v, partials, ticket) && threadIdx.x == 0) {
        sc->iter += 1;
        sc->total += 1;
        sc->rr = v[0];
        if (!isfinite(v[0])) {
            sc->status = CG_NONFINITE;
            sc->done = 1;
        } else if (sqrt(v[0]) <= sc->stop2) {
            sc->done = 1;
        } else if (sc->iter >= sc->max_it) {
            sc->status = CG_MAXIT;
            sc->done = 1;
        }
    }
}

// DIC's black pass, z_b = (r_b + sum T u) / d_b, with the black cells' share
// of r.z (into sc->rz_part).
__global__ void __launch_bounds__(RED_THREADS)
k_dic_black(Grid g, const float *__restrict__ K32, const float *__restrict__ rd32, const float *__restrict__ r,
            float *__restrict__ z, double *partials, unsigned int *ticket, CgScal *sc)
{
    if (sc->done) return;
    float a0 = 0.0f;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < g.N; p += stride) {
        int i, j, k;
        if (colour_of(g, p, i, j, k) != 1) continue;
        const float rd = rd32[p];
        if (rd == 0.0f) {                 // inactive
            z[p] = 0.0f;
            continue;
        }
        const float rp = r[p];
        float s = rp;
        active_faces(g, K32, p, i, j, k, K32[p], [&](long long q, float t) { s = fmaf(t, z[q], s); });
        const float zp = rd * s;
        z[p] = zp;
        a0 = fmaf(rp, zp, a0);
    }
    float vf[1] = {a0};
    double v[1];
    if (grid_reduce_f32<1>(vf, v, partials, ticket) && threadIdx.x == 0) sc->rz_part = v[0];
}

// DIC's red back-substitution, z_r = u_r + sum T z_b / d_r, finishing r.z:
// start = 1 sets rho (first preconditioned residual of an inner solve),
// otherwise beta = r.z / rho; always sets the inner loop condition.
__global__ void __launch_bounds__(RED_THREADS)
k_dic_red(Grid g, const float *__restrict__ K32, const float *__restrict__ rd32, const float *__restrict__ r,
          float *__restrict__ z, double *partials, unsigned int *ticket, CgScal *sc, int start, CondSet cond)
{
    if (sc->done) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_cond(cond, 0);
        return;
    }
    float a0 = 0.0f;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < g.N; p += stride) {
        int i, j, k;
        if (colour_of(g, p, i, j, k) != 0) continue;
        const float rd = rd32[p];
        if (rd == 0.0f) continue;         // inactive: z stays 0
        float s = 0.0f;
        active_faces(g, K32, p, i, j, k, K32[p], [&](long long q, float t) { s = fmaf(t, z[q], s); });
        const float zp = fmaf(rd, s, z[p]);
        z[p] = zp;
        a0 = fmaf(r[p], zp, a0);
    }
    float vf[1] = {a0};
    double v[1];
    if (grid_reduce_f32<1>(vf, v, partials, ticket) && threadIdx.x == 0) {
        const double rz = v[0] + sc->rz_part;
        if (!isfinite(rz) || !(rz > 0.0)) {
            // a zero or non-finite r.z with a non-zero residual: breakdown
            sc->status = CG_NONFINITE;
            sc->done = 1;
        } else if (start) {
            sc->rho = rz;
            sc->beta = 0.0;
        } else {
            sc->beta = rz / sc->rho;
            sc->rho = rz;
        }
        set_cond(cond, sc->done ? 0 : 1);
    }
}

}  // namespace

void launch_cg32_update_dic(cudaStream_t s, int nblk, const Grid &g, float *x, float *r, float *z, const float *p,
                            const float *q, const float *dinv, const float *rd32, double *partials,
                            unsigned int *ticket, CgScal *sc)
{
    k_cg32_update_dic<<<nblk, RED_THREADS, 0, s>>>(g, x, r, z, p, q, dinv, rd32, partials, ticket, sc);
}

void launch_dic_apply_rz(cudaStream_t s, int nblk, const Grid &g, const float *K32, const float *rd32, const float *r,
                         float *z, double *partials, unsigned int *ticket, CgScal *sc, int start, bool red_done,
                         CondSet cond)
{
    if (!red_done) k_dic_sweep<0><<<nblk, RED_THREADS, 0, s>>>(g, K32, rd32, r, z, &sc->done);
    k_dic_black<<<nblk, RED_THREADS, 0, s>>>(g, K32, rd32, r, z, partials, ticket, sc);
    k_dic_red<<<nblk, RED_THREADS, 0, s>>>(g, K32, rd32, r, z, partials, ticket, sc, start, cond);
}

void launch_dic_setup(cudaStream_t s, int nblk, const Grid &g, const float *K32, const float *cb32, float *diag32,
                      float *rd32, const int *skip)
{
    k_dic_diag<<<nblk, RED_THREADS, 0, s>>>(g, K32, cb32, diag32, skip);
    k_dic_pivots<<<nblk, RED_THREADS, 0, s>>>(g, K32, diag32, rd32, skip);
}

}  // namespace rf
