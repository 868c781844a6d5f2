// pcg.cu -- matrix-free 7-point stencil operator and Jacobi-preconditioned
// conjugate gradient for the Picard system (Sec. 2.2: PCG on the symmetric
// M-matrix of the backward-Euler / Picard linearisation).
//
// FP64 path: the operator is stored as diag(A) and the three upper-face
// coefficients Tx, Ty, Tz per cell (GB300's FP64 rate is low, so the face
// coefficients are read, not recomputed).
//   (A v)_P = diag_P v_P - sum_f T_f v_N
// FP32 inner path (mixed precision): faces are recomputed from K in FP32,
//   (A v)_P = cb_P v_P + sum_f w_f (K_P + K_N)/2 (v_P - v_N)
// where cb = c + Dirichlet half-cell terms; inactive neighbours carry K < 0.
//
// One PCG iteration is two kernels:
//   spmv   : p = z + beta p_old (recomputed for the stencil neighbours, so p
//            ping-pongs between two buffers), q = A p, partial p.q;
//   update : x += alpha p, r -= alpha q, z = D^-1 r, partial r.r and r.z.
// The scalars (alpha, beta, rho, convergence) live on the device and are
// produced by the last block of each grid reduction, so a solve needs no host
// round trip per iteration; kernels of a finished solve return at once.
#include <math.h>

#include "cell_ops.cuh"
#include "rf_internal.cuh"
#include "rf_reduce.cuh"

namespace rf {

#define GRID_STRIDE_LOOP(p)                                                                 \
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < g.N;           \
         p += (long long)gridDim.x * blockDim.x)

// ---------------------------------------------------------------- FP64 PCG
__global__ void __launch_bounds__(RED_THREADS)
k_cg64_init(Grid g, const uint8_t *__restrict__ flags, const double *__restrict__ x0, double *__restrict__ x,
            const double *__restrict__ b, const double *__restrict__ Tx, const double *__restrict__ Ty,
            const double *__restrict__ Tz, const double *__restrict__ diag, const double *__restrict__ dinv,
            double *__restrict__ r, double *__restrict__ z, double tol, int max_it, double *partials,
            unsigned int *ticket, CgScal *sc, const int *skip, CondSet cond)
{
    count_launch(g, KK_CG64_INIT);
    if (skip && *skip) {        // Picard attempt already finished: no solve, empty CG loop
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            sc->done = 1;
            set_cond(cond, 0);
        }
        return;
    }
    count_work(g, KK_CG64_INIT);
    double v[3] = {0.0, 0.0, 0.0};   // r.z, r.r, b.b
    GRID_STRIDE_LOOP(p)
    {
        const double xp = x0[p];
        x[p] = xp;
        if (!(flags[p] & FLAG_ACTIVE)) {
            r[p] = 0.0;
            z[p] = 0.0;
            continue;
        }
        const double bp = b[p];
        const double rp = bp - apply64(g, p, Tx, Ty, Tz, diag, [&](long long q) { return x0[q]; });
        const double zp = dinv[p] * rp;
        r[p] = rp;
        z[p] = zp;
        v[0] += rp * zp;
        v[1] += rp * rp;
        v[2] += bp * bp;
    }
    if (grid_reduce<OpSum, 3>(v, partials, ticket) && threadIdx.x == 0)
        cg64_start_scalars(sc, v, tol, max_it, cond);
}

__global__ void __launch_bounds__(RED_THREADS)
k_cg64_spmv(Grid g, const uint8_t *__restrict__ flags, const double *__restrict__ z, const double *__restrict__ p_in,
            double *__restrict__ p_out, double *__restrict__ q, const double *__restrict__ Tx,
            const double *__restrict__ Ty, const double *__restrict__ Tz, const double *__restrict__ diag,
            double *partials, unsigned int *ticket, CgScal *sc)
{
    count_launch(g, KK_CG64_SPMV);
    if (sc->done) return;
    count_work(g, KK_CG64_SPMV);
    const double beta = sc->beta;
    const bool first = sc->iter == 0;
    auto get = [&](long long qq) { return first ? z[qq] : fma(beta, p_in[qq], z[qq]); };
    double v[1] = {0.0};
    GRID_STRIDE_LOOP(p)
    {
        if (!(flags[p] & FLAG_ACTIVE)) {
            p_out[p] = 0.0;
            q[p] = 0.0;
            continue;
        }
        const double pp = get(p);
        const double qp = apply64(g, p, Tx, Ty, Tz, diag, get);
        p_out[p] = pp;
        q[p] = qp;
        v[0] += pp * qp;
    }
    if (grid_reduce<OpSum, 1>(v, partials, ticket) && threadIdx.x == 0) {
        sc->pq = v[0];
        const double a = sc->rho / v[0];
        if (!(v[0] > 0.0) || !isfinite(a)) {
            sc->status = CG_NONFINITE;
            sc->done = 1;
        }
        sc->alpha = a;
    }
}

__global__ void __launch_bounds__(RED_THREADS)
k_cg64_update(Grid g, double *__restrict__ x, double *__restrict__ r, double *__restrict__ z,
              const double *__restrict__ pd, const double *__restrict__ q, const double *__restrict__ dinv,
              double *partials, unsigned int *ticket, CgScal *sc, CondSet cond)
{
    count_launch(g, KK_CG64_UPDATE);
    if (sc->done) {             // every launch sets the loop condition
        if (blockIdx.x == 0 && threadIdx.x == 0) set_cond(cond, 0);
        return;
    }
    count_work(g, KK_CG64_UPDATE);
    const double alpha = sc->alpha;
    double v[2] = {0.0, 0.0};   // r.r, r.z
    GRID_STRIDE_LOOP(p)
    {
        const double di = dinv[p];
        if (di == 0.0) continue;                  // inactive
        x[p] = fma(alpha, pd[p], x[p]);
        const double rp = fma(-alpha, q[p], r[p]);
        const double zp = di * rp;
        r[p] = rp;
        z[p] = zp;
        v[0] += rp * rp;
        v[1] += rp * zp;
    }
    if (grid_reduce<OpSum, 2>(v, partials, ticket) && threadIdx.x == 0) {
        sc->iter += 1;
        sc->total += 1;
        sc->rr = v[0];
        if (!isfinite(v[0]) || !isfinite(v[1])) {
            sc->status = CG_NONFINITE;
            sc->done = 1;
        } else if (sqrt(v[0]) <= sc->stop2) {
            sc->done = 1;
        } else if (sc->iter >= sc->max_it) {
            sc->status = CG_MAXIT;
            sc->done = 1;
        } else {
            sc->beta = v[1] / sc->rho;
            sc->rho = v[1];
        }
        set_cond(cond, sc->done ? 0 : 1);
    }
}

__global__ void __launch_bounds__(RED_THREADS)
k_apply64(Grid g, const uint8_t *__restrict__ flags, const double *__restrict__ x, double *__restrict__ y,
          const double *__restrict__ Tx, const double *__restrict__ Ty, const double *__restrict__ Tz,
          const double *__restrict__ diag)
{
    count_launch(g, KK_APPLY64);
    count_work(g, KK_APPLY64);
    GRID_STRIDE_LOOP(p)
    {
        y[p] = (flags[p] & FLAG_ACTIVE) ? apply64(g, p, Tx, Ty, Tz, diag, [&](long long q) { return x[q]; }) : 0.0;
    }
}

// ------------------------------------------------------ mixed precision
// Start of a defect-correction solve: x = x0, counters reset, outer loop
// condition raised (or, when the Picard attempt is over, an empty loop).
__global__ void __launch_bounds__(RED_THREADS)
k_mixed_start(Grid g, const double *__restrict__ x0, double *__restrict__ x, CgScal *outer, CgScal *inner,
              const int *skip, CondSet cond_outer)
{
    count_launch(g, KK_MIXED_START);
    const bool skipped = skip && *skip;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        outer->iter = 0;
        outer->done = skipped ? 1 : 0;
        outer->status = CG_OK;
        inner->total = 0;
        inner->status = CG_OK;
        set_cond(cond_outer, skipped ? 0 : 1);
    }
    if (skipped) return;
    count_work(g, KK_MIXED_START);
    GRID_STRIDE_LOOP(p) { x[p] = x0[p]; }
}

// Outer FP64 residual r = b - A x; seeds the inner FP32 solve A d = r with
// d0 = 0 (so r32 = r, z32 = D^-1 r32).  Counts outer iterations and fails the
// solve after outer_max_it residuals without convergence.
__global__ void __launch_bounds__(RED_THREADS)
k_resid64(Grid g, const uint8_t *__restrict__ flags, const double *__restrict__ x, const double *__restrict__ b,
          const double *__restrict__ Tx, const double *__restrict__ Ty, const double *__restrict__ Tz,
          const double *__restrict__ diag, const float *__restrict__ dinv32, float *__restrict__ r32,
          float *__restrict__ z32, float *__restrict__ d32, double tol, double tol_inner, int inner_max_it,
          int outer_max_it, double *partials, unsigned int *ticket, CgScal *outer, CgScal *inner,
          CondSet cond_outer, CondSet cond_inner)
{
    count_launch(g, KK_RESID64);
    if (outer->done) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            inner->done = 1;
            set_cond(cond_outer, 0);
            set_cond(cond_inner, 0);
        }
        return;
    }
    count_work(g, KK_RESID64);
    double v[4] = {0.0, 0.0, 0.0, 0.0};   // r.r, b.b (FP64); r32.r32, r32.z32
    GRID_STRIDE_LOOP(p)
    {
        d32[p] = 0.0f;
        if (!(flags[p] & FLAG_ACTIVE)) {
            r32[p] = 0.0f;
            z32[p] = 0.0f;
            continue;
        }
        const double bp = b[p];
        const double rp = bp - apply64(g, p, Tx, Ty, Tz, diag, [&](long long q) { return x[q]; });
        const float rf = (float)rp;
        const float zf = dinv32[p] * rf;
        r32[p] = rf;
        z32[p] = zf;
        v[0] += rp * rp;
        v[1] += bp * bp;
        v[2] += (double)(rf * rf);
        v[3] += (double)(rf * zf);
    }
    if (grid_reduce<OpSum, 4>(v, partials, ticket) && threadIdx.x == 0) {
        outer->iter += 1;
        outer_residual_scalars(outer, inner, v, tol, tol_inner, inner_max_it, outer_max_it, cond_outer, cond_inner);
    }
}

__global__ void __launch_bounds__(RED_THREADS)
k_cg32_spmv(Grid g, const float *__restrict__ z, const float *__restrict__ p_in, float *__restrict__ p_out,
            float *__restrict__ q, const float *__restrict__ K32, const float *__restrict__ cb32, double *partials,
            unsigned int *ticket, CgScal *sc)
{
    count_launch(g, KK_CG32_SPMV);
    if (sc->done) return;
    count_work(g, KK_CG32_SPMV);
    const float beta = (float)sc->beta;
    const bool first = sc->iter == 0;
    auto get = [&](long long qq) { return first ? z[qq] : fmaf(beta, p_in[qq], z[qq]); };
    float acc = 0.0f;
    GRID_STRIDE_LOOP(p)
    {
        if (K32[p] < 0.0f) {
            p_out[p] = 0.0f;
            q[p] = 0.0f;
            continue;
        }
        const float pp = get(p);
        const float qp = apply32(g, p, K32, cb32, get);
        p_out[p] = pp;
        q[p] = qp;
        acc = fmaf(pp, qp, acc);
    }
    float vf[1] = {acc};
    double v[1];
    if (grid_reduce_f32<1>(vf, v, partials, ticket) && threadIdx.x == 0) {
        sc->pq = v[0];
        const double a = sc->rho / v[0];
        if (!(v[0] > 0.0) || !isfinite(a)) {
            sc->status = CG_NONFINITE;
            sc->done = 1;
        }
        sc->alpha = a;
    }
}

__global__ void __launch_bounds__(RED_THREADS)
k_cg32_update(Grid g, float *__restrict__ x, float *__restrict__ r, float *__restrict__ z,
              const float *__restrict__ pd, const float *__restrict__ q, const float *__restrict__ dinv,
              double *partials, unsigned int *ticket, CgScal *sc, CondSet cond)
{
    count_launch(g, KK_CG32_UPDATE);
    if (sc->done) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_cond(cond, 0);
        return;
    }
    count_work(g, KK_CG32_UPDATE);
    const float alpha = (float)sc->alpha;
    float a0 = 0.0f, a1 = 0.0f;
    GRID_STRIDE_LOOP(p)
    {
        const float di = dinv[p];
        if (di == 0.0f) continue;
        x[p] = fmaf(alpha, pd[p], x[p]);
        const float rp = fmaf(-alpha, q[p], r[p]);
        const float zp = di * rp;
        r[p] = rp;
        z[p] = zp;
        a0 = fmaf(rp, rp, a0);
        a1 = fmaf(rp, zp, a1);
    }
    float vf[2] = {a0, a1};
    double v[2];
    if (grid_reduce_f32<2>(vf, v, partials, ticket) && threadIdx.x == 0) {
        sc->iter += 1;
        sc->total += 1;
        sc->rr = v[0];
        if (!isfinite(v[0]) || !isfinite(v[1])) {
            sc->status = CG_NONFINITE;
            sc->done = 1;
        } else if (sqrt(v[0]) <= sc->stop2) {
            sc->done = 1;
        } else if (sc->iter >= sc->max_it) {
            sc->status = CG_MAXIT;
            sc->done = 1;
        } else {
            sc->beta = v[1] / sc->rho;
            sc->rho = v[1];
        }
        set_cond(cond, sc->done ? 0 : 1);
    }
}

// x += d after an inner solve; a non-finite inner solve fails the outer loop
// (an inner solve that only reached its iteration cap is still applied).
__global__ void __launch_bounds__(RED_THREADS)
k_add_correction(Grid g, double *__restrict__ x, const float *__restrict__ d, CgScal *outer, const CgScal *inner,
                 CondSet cond_outer)
{
    count_launch(g, KK_ADD_CORRECTION);
    if (outer->done) return;
    if (inner->status == CG_NONFINITE) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            outer->status = CG_NONFINITE;
            outer->done = 1;
            set_cond(cond_outer, 0);
        }
        return;
    }
    count_work(g, KK_ADD_CORRECTION);
    GRID_STRIDE_LOOP(p) { x[p] += (double)d[p]; }
}

// ------------------------------------------------------------ launchers
void launch_cg64_init(cudaStream_t s, int nblk, const Grid &g, const uint8_t *flags, const double *x0, double *x,
                      const double *b, const double *Tx, const double *Ty, const double *Tz, const double *diag,
                      const double *dinv, double *r, double *z, double tol, int max_it, double *partials,
                      unsigned int *ticket, CgScal *sc, const int *skip, CondSet cond)
{
    k_cg64_init<<<nblk, RED_THREADS, 0, s>>>(g, flags, x0, x, b, Tx, Ty, Tz, diag, dinv, r, z, tol, max_it, partials,
                                             ticket, sc, skip, cond);
}

void launch_cg64_spmv(cudaStream_t s, int nblk, const Grid &g, const uint8_t *flags, const double *z,
                      const double *p_in, double *p_out, double *q, const double *Tx, const double *Ty,
                      const double *Tz, const double *diag, double *partials, unsigned int *ticket, CgScal *sc)
{
    k_cg64_spmv<<<nblk, RED_THREADS, 0, s>>>(g, flags, z, p_in, p_out, q, Tx, Ty, Tz, diag, partials, ticket, sc);
}

void launch_cg64_update(cudaStream_t s, int nblk, const Grid &g, double *x, double *r, double *z, const double *p,
                        const double *q, const double *dinv, double *partials, unsigned int *ticket, CgScal *sc,
                        CondSet cond)
{
    k_cg64_update<<<nblk, RED_THREADS, 0, s>>>(g, x, r, z, p, q, dinv, partials, ticket, sc, cond);
}

void launch_apply64(cudaStream_t s, int nblk, const Grid &g, const uint8_t *flags, const double *x, double *y,
                    const double *Tx, const double *Ty, const double *Tz, const double *diag)
{
    k_apply64<<<nblk, RED_THREADS, 0, s>>>(g, flags, x, y, Tx, Ty, Tz, diag);
}

void launch_mixed_start(cudaStream_t s, int nblk, const Grid &g, const double *x0, double *x, CgScal *outer,
                        CgScal *inner, const int *skip, CondSet cond_outer)
{
    k_mixed_start<<<nblk, RED_THREADS, 0, s>>>(g, x0, x, outer, inner, skip, cond_outer);
}

void launch_resid64(cudaStream_t s, int nblk, const Grid &g, const uint8_t *flags, const double *x, const double *b,
                    const double *Tx, const double *Ty, const double *Tz, const double *diag, const float *dinv32,
                    float *r32, float *z32, float *d32, double tol, double tol_inner, int inner_max_it,
                    int outer_max_it, double *partials, unsigned int *ticket, CgScal *outer, CgScal *inner,
                    CondSet cond_outer, CondSet cond_inner)
{
    k_resid64<<<nblk, RED_THREADS, 0, s>>>(g, flags, x, b, Tx, Ty, Tz, diag, dinv32, r32, z32, d32, tol, tol_inner,
                                           inner_max_it, outer_max_it, partials, ticket, outer, inner, cond_outer,
                                           cond_inner);
}

void launch_cg32_spmv(cudaStream_t s, int nblk, const Grid &g, const float *z, const float *p_in, float *p_out,
                      float *q, const float *K32, const float *cb32, double *partials, unsigned int *ticket,
                      CgScal *sc)
{
    k_cg32_spmv<<<nblk, RED_THREADS, 0, s>>>(g, z, p_in, p_out, q, K32, cb32, partials, ticket, sc);
}

void launch_cg32_update(cudaStream_t s, int nblk, const Grid &g, float *x, float *r, float *z, const float *p,
                        const float *q, const float *dinv, double *partials, unsigned int *ticket, CgScal *sc,
                        CondSet cond)
{
    k_cg32_update<<<nblk, RED_THREADS, 0, s>>>(g, x, r, z, p, q, dinv, partials, ticket, sc, cond);
}

void launch_add_correction(cudaStream_t s, int nblk, const Grid &g, double *x, const float *d, CgScal *outer,
                           const CgScal *inner, CondSet cond_outer)
{
    k_add_correction<<<nblk, RED_THREADS, 0, s>>>(g, x, d, outer, inner, cond_outer);
}

}  // namespace rf
