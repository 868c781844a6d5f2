// closure_assemble.cu -- per-cell closures (Eq. 2-4, Eq. A6), Picard-system
// assembly (Sec. 2.2), water-balance reductions.
//
// Layout: structure-of-arrays over all nx*ny*nz cells, x fastest.  Inactive
// cells carry K = -1 (a sentinel the stencil kernels test instead of reading
// the flag array) and zeros elsewhere.
#include <math.h>

#include "cell_ops.cuh"
#include "rf_internal.cuh"
#include "rf_reduce.cuh"

namespace rf {

// Closures of every cell at h; with hprev, also max|h - hprev| and a
// non-finite flag in v[0], v[1].
__device__ __forceinline__ void closure_cells(const Grid &g, const DevSoil *__restrict__ soils,
                                              const uint8_t *__restrict__ zone, const double *__restrict__ Ks,
                                              const uint8_t *__restrict__ flags, const double *__restrict__ h,
                                              const double *__restrict__ hprev, double *__restrict__ theta,
                                              double *__restrict__ K, double *__restrict__ Can, double (&v)[2])
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < g.N; p += stride) {
        if (!(flags[p] & FLAG_ACTIVE)) {
            theta[p] = 0.0;
            K[p] = -1.0;
            Can[p] = 0.0;
            continue;
        }
        const double hp = h[p];
        if (hprev) {
            const double d = fabs(hp - hprev[p]);
            if (d <= 1e300) v[0] = fmax(v[0], d);
            else v[1] = 1.0;           // NaN or inf
        }
        const DevSoil s = soils[zone[p]];
        double th, k, c;
        closure(s, Ks[p], hp, g.tab, g.closure64, th, k, c);
        theta[p] = th;
        K[p] = k;
        Can[p] = c;
    }
}

__global__ void __launch_bounds__(RED_THREADS)
k_closure(Grid g, const DevSoil *__restrict__ soils, const uint8_t *__restrict__ zone,
          const double *__restrict__ Ks, const uint8_t *__restrict__ flags, const double *__restrict__ h,
          const double *__restrict__ hprev, double *__restrict__ theta, double *__restrict__ K,
          double *__restrict__ Can, double *partials, unsigned int *ticket, StepResults *res)
{
    count_launch(g, KK_CLOSURE);
    count_work(g, KK_CLOSURE);
    double v[2] = {0.0, 0.0};   // max |h - hprev|, non-finite flag
    closure_cells(g, soils, zone, Ks, flags, h, hprev, theta, K, Can, v);
    if (hprev) {
        if (grid_reduce<OpMax, 2>(v, partials, ticket) && threadIdx.x == 0) {
            res->max_dh = v[0];
            res->nonfinite = v[1] > 0.0;
        }
    }
}

// End of a Picard iteration on the device: closures at the new iterate x
// (which also serve the next assembly, or the next step once accepted), the
// exit test max|x - h^k| <= tol over all active cells (global, Sec. 2.3),
// and the loop control.  A failed linear solve or a non-finite update fails
// the attempt.  The last block sets the Picard loop condition; every launch
// sets it, so the loop always terminates (at the latest after n_max).
__global__ void __launch_bounds__(RED_THREADS)
k_closure_picard(Grid g, const DevSoil *__restrict__ soils, const uint8_t *__restrict__ zone,
                 const double *__restrict__ Ks, const uint8_t *__restrict__ flags, const double *__restrict__ x,
                 const double *__restrict__ hk, double *__restrict__ theta, double *__restrict__ K,
                 double *__restrict__ Can, double *partials, unsigned int *ticket, PicardCtl *ctl,
                 const CgScal *cg_status, const CgScal *cg_count, CondSet cond)
{
    count_launch(g, KK_CLOSURE_PICARD);
    if (ctl->done) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_cond(cond, 0);
        return;
    }
    count_work(g, KK_CLOSURE_PICARD);
    double v[2] = {0.0, 0.0};
    closure_cells(g, soils, zone, Ks, flags, x, hk, theta, K, Can, v);
    if (grid_reduce<OpMax, 2>(v, partials, ticket) && threadIdx.x == 0) {
        const int it = ++ctl->it;
        if (cg_status->status != CG_OK) {
            ctl->fail = 1;
        } else {
            ctl->cg_total += cg_count->total;
            ctl->max_dh = v[0];
            if (v[1] > 0.0) ctl->fail = 1;
            else if (v[0] <= ctl->tol) {
                ctl->conv = 1;
                ctl->mb_pending = 1;
            }
        }
        ctl->done = (ctl->conv || ctl->fail || it >= ctl->n_max) ? 1 : 0;
        set_cond(cond, ctl->done ? 0 : 1);
    }
}

// Assembly of V C^k (h - h^n)/dt = sum_f T_f (h_N - h) + G + B (Sec. 2.2):
//   c = V C^k / dt, C^k the chord slope of theta* (or C(h^k) when
//   |h^k - h^n| <= eps); T_f = Kbar_f A_f/d_f, Kbar_f = (K_P + K_N)/2;
//   explicit gravity A_z (Kbar_top - Kbar_bottom) with K at h^k;
//   boundary terms per face class (Dirichlet at the half cell with K(h_D),
//   imposed flux, free drainage -K(h^k) A_z, seepage as Dirichlet 0 while the
//   cell is saturated at the step start).
// Outputs: c, b, upper-face coefficients Tx/Ty/Tz (0 where the face is not an
// interior face), diag(A), 1/diag; FP32 copies of K (NaN on inactive cells,
// so that max(w (K_P + K_N), 0) closes their faces without a test) and of c
// plus the Dirichlet diagonal terms for the mixed-precision operator.
template <int MODE>
__global__ void __launch_bounds__(RED_THREADS)
k_assemble(Grid g, const DevSoil *__restrict__ soils, const uint8_t *__restrict__ zone,
           const double *__restrict__ Ks, const uint8_t *__restrict__ flags, const StepParams *__restrict__ spp,
           const double *__restrict__ hk, const double *__restrict__ hn, const double *__restrict__ thk,
           const double *__restrict__ thn, const double *__restrict__ K, const double *__restrict__ Can,
           double *__restrict__ c_out, double *__restrict__ b, double *__restrict__ Tx, double *__restrict__ Ty,
           double *__restrict__ Tz, double *__restrict__ diag_out, double *__restrict__ dinv,
           float *__restrict__ K32, float *__restrict__ cb32, float *__restrict__ dinv32, const int *skip,
           SolveStart st, double *partials, unsigned int *ticket, double *__restrict__ s0_out,
           const double *__restrict__ thp)
{
    count_launch(g, KK_ASSEMBLE);
    if (skip && *skip) {
        if (MODE != ASM_ONLY && blockIdx.x == 0 && threadIdx.x == 0) {
            // the Picard attempt is over: the linear-solve loops that follow are empty
            st.sc->done = 1;
            set_cond(st.cond, 0);
            if (MODE == ASM_MIXED) {
                st.inner->done = 1;
                set_cond(st.cond_inner, 0);
            }
        }
        return;
    }
    count_work(g, KK_ASSEMBLE);
    const double eps = spp->eps_chord;
    const double V_dt = g.V / spp->dt;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    float a_rr = 0.0f, a_bb = 0.0f, a_rz = 0.0f;   // mixed start: norms of the FP32 seeds, summed in FP32
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < g.N; p += stride) {
        const uint8_t fl = flags[p];
        if (!(fl & FLAG_ACTIVE)) {
            c_out[p] = 0.0; b[p] = 0.0; Tx[p] = 0.0; Ty[p] = 0.0; Tz[p] = 0.0;
            diag_out[p] = 0.0; dinv[p] = 0.0;
            K32[p] = __int_as_float(0x7fc00000); cb32[p] = 0.0f; dinv32[p] = 0.0f;   // NaN: fails every K >= 0 test
            if (MODE != ASM_ONLY) st.x[p] = hk[p];
            if (MODE == ASM_CG64) { st.r[p] = 0.0; st.z[p] = 0.0; }
            if (MODE == ASM_MIXED) { st.r32[p] = 0.0f; st.z32[p] = 0.0f; st.d32[p] = 0.0f; }
            continue;
        }
        int i, j, k;
        cell_ijk(g, p, i, j, k);
        const double hkP = hk[p];
        CellSystem cs;
        assemble_cell<MODE != ASM_ONLY>(g, soils, zone, Ks, fl, *spp, p, i, j, k, hk, hn, thk, thn, K, Can, thp, eps,
                                        V_dt, cs);
        const double c = cs.c, rhs = cs.rhs, diag = cs.diag, cb = cs.cb, sT = cs.sT, KP = cs.KP;
        const double *Tup = cs.Tup;
        c_out[p] = c;
        b[p] = rhs;
        if (s0_out) s0_out[p] = cs.s0;   // modified Picard: the water balance needs the storage part
        Tx[p] = Tup[0];
        Ty[p] = Tup[1];
        Tz[p] = Tup[2];
        // 1/diag: in FP64 for the FP64 PCG; the mixed path's Jacobi scaling
        // is FP32 only (its FP64 copy is not read), so it skips the FP64
        // reciprocal, a dozen instructions on the narrow FP64 pipe
        double di = 0.0;
        float di32;
        if (MODE == ASM_MIXED) {
            di32 = __frcp_rn((float)diag);
        } else {
            di = rcp64(diag);
            dinv[p] = di;
            di32 = (float)di;
        }
        diag_out[p] = diag;
        K32[p] = (float)KP;
        cb32[p] = (float)cb;
        dinv32[p] = di32;
        if (MODE != ASM_ONLY) {
            // first residual of the linear solve from x0 = h^k
            const double rp = rhs - (diag * hkP - sT);
            st.x[p] = hkP;
            if (MODE == ASM_CG64) {
                const double zp = di * rp;
                st.r[p] = rp;
                st.z[p] = zp;
                v[0] += rp * zp;
                v[1] += rp * rp;
                v[2] += rhs * rhs;
            } else {
                const float rf = (float)rp;
                const float zf = di32 * rf;
                const float bf = (float)rhs;
                st.r32[p] = rf;
                st.z32[p] = zf;
                st.d32[p] = 0.0f;
                a_rr = fmaf(rf, rf, a_rr);
                a_bb = fmaf(bf, bf, a_bb);
                a_rz = fmaf(rf, zf, a_rz);
            }
        }
    }
    if (MODE == ASM_CG64) {
        double w3[3] = {v[0], v[1], v[2]};
        if (grid_reduce<OpSum, 3>(w3, partials, ticket) && threadIdx.x == 0)
            cg64_start_scalars(st.sc, w3, st.tol, st.max_it, st.cond);
    } else if (MODE == ASM_MIXED) {
        // the residual is formed in FP64; its norms (a stopping test and CG
        // seeds) are summed in FP32 within a block, in FP64 across blocks
        float vf[3] = {a_rr, a_bb, a_rz};
        double w[3];
        if (grid_reduce_f32<3>(vf, w, partials, ticket) && threadIdx.x == 0) {
            v[0] = w[0];
            v[1] = w[1];
            v[2] = w[0];
            v[3] = w[2];
            st.sc->iter = 1;
            st.sc->done = 0;
            st.sc->status = CG_OK;
            st.inner->total = 0;
            outer_residual_scalars(st.sc, st.inner, v, st.tol, st.tol_inner, st.inner_max_it, st.outer_max_it,
                                   st.cond, st.cond_inner);
        }
    }
}

// Water balance of the accepted step's last linear system (x = h^{n+1}):
// sum c dt (x - h^n), sum V (theta*(x) - theta*(h^n)), and dt times the
// boundary inflow / outflow of that system, split per face by sign.
// After a Picard attempt (ctl given): only when it converged; the final
// iterate and the K of its last system sit in the buffers of the last
// iteration's half: x_odd / K_odd after an odd number of iterations, x_even /
// K_even after an even number.
__global__ void __launch_bounds__(RED_THREADS)
k_mass_balance(Grid g, const DevSoil *__restrict__ soils, const uint8_t *__restrict__ zone,
               const double *__restrict__ Ks, const uint8_t *__restrict__ flags,
               const StepParams *__restrict__ spp, const double *__restrict__ x_odd,
               const double *__restrict__ x_even, const double *__restrict__ hn, const double *__restrict__ c,
               const double *__restrict__ K_odd, const double *__restrict__ K_even, const double *__restrict__ thx,
               const double *__restrict__ thn, double *partials, unsigned int *ticket, StepResults *res,
               const PicardCtl *ctl, const double *__restrict__ s0)
{
    count_launch(g, KK_MASS_BALANCE);
    if (ctl && !ctl->conv) return;
    count_work(g, KK_MASS_BALANCE);
    const bool odd = !ctl || (ctl->it & 1);
    const double *__restrict__ x = odd ? x_odd : x_even;
    const double *__restrict__ Kold = odd ? K_odd : K_even;
    const double dt = spp->dt;
    double v[4] = {0.0, 0.0, 0.0, 0.0};   // lin, dS, in, out
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < g.N; p += stride) {
        const uint8_t fl = flags[p];
        if (!(fl & FLAG_ACTIVE)) continue;
        const double xp = x[p], hnP = hn[p];
        // storage of the solved system: c (x - h^n), or with modified Picard
        // c x - s0 = c (x - h^k) + V (theta*^k - theta*^n) / dt (times dt)
        v[0] += s0 ? dt * (c[p] * xp - s0[p]) : c[p] * dt * (xp - hnP);
        v[1] += g.V * (thx[p] - thn[p]);
        if (!(fl & 0x3f)) continue;
        double fin, fout;
        boundary_fluxes(g, soils[zone[p]], Ks[p], fl, *spp, xp, hnP, Kold[p], fin, fout);
        v[2] += dt * fin;
        v[3] += dt * fout;
    }
    if (grid_reduce<OpSum, 4>(v, partials, ticket) && threadIdx.x == 0) {
        res->lin_change = v[0];
        res->dstore = v[1];
        res->bnd_in = v[2];
        res->bnd_out = v[3];
    }
}

__global__ void __launch_bounds__(RED_THREADS)
k_storage(Grid g, const uint8_t *__restrict__ flags, const double *__restrict__ theta, double *partials,
          unsigned int *ticket, StepResults *res)
{
    count_launch(g, KK_STORAGE);
    count_work(g, KK_STORAGE);
    double v[1] = {0.0};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < g.N; p += stride)
        if (flags[p] & FLAG_ACTIVE) v[0] += g.V * theta[p];
    if (grid_reduce<OpSum, 1>(v, partials, ticket) && threadIdx.x == 0) res->storage = v[0];
}

__global__ void __launch_bounds__(RED_THREADS)
k_accept(Grid g, const double *__restrict__ xf, double *__restrict__ h, const double *__restrict__ thk,
         double *__restrict__ thn, const double *__restrict__ K1, double *__restrict__ K0, int copyK)
{
    count_launch(g, KK_ACCEPT);
    count_work(g, KK_ACCEPT);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < g.N; p += stride) {
        h[p] = xf[p];
        thn[p] = thk[p];
        if (copyK) K0[p] = K1[p];
    }
}

// Check of a state uploaded into src: the number of active cells whose head
// is not finite (res->nonfinite); then, only when there is none, the commit
// dst = src with non-finite values on inactive cells replaced by 0.
__global__ void __launch_bounds__(RED_THREADS)
k_state_check(Grid g, const uint8_t *__restrict__ flags, const double *__restrict__ src, double *partials,
              unsigned int *ticket, StepResults *res)
{
    double v[1] = {0.0};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < g.N; p += stride)
        if ((flags[p] & FLAG_ACTIVE) && !isfinite(src[p])) v[0] += 1.0;
    if (grid_reduce<OpSum, 1>(v, partials, ticket) && threadIdx.x == 0) res->nonfinite = v[0] > 0.0;
}

__global__ void __launch_bounds__(RED_THREADS)
k_state_commit(Grid g, const double *__restrict__ src, double *__restrict__ dst, const StepResults *res)
{
    if (res->nonfinite) return;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < g.N; p += stride) {
        const double v = src[p];
        dst[p] = isfinite(v) ? v : 0.0;
    }
}

void launch_state_check_commit(cudaStream_t s, int nblk, const Grid &g, const uint8_t *flags, const double *src,
                               double *dst, double *partials, unsigned int *ticket, StepResults *res)
{
    k_state_check<<<nblk, RED_THREADS, 0, s>>>(g, flags, src, partials, ticket, res);
    k_state_commit<<<nblk, RED_THREADS, 0, s>>>(g, src, dst, res);
}

// Both precisions' tables: the double-float ones from double arithmetic,
// the FP64 ones from long double (extended or quadruple precision on the
// hosts this builds for), each rounded once.
void make_ff_tables(FFTables *t)
{
    for (int j = 0; j < F64_TAB; j++) {
        const long double e = exp2l((long double)j / (long double)F64_TAB);
        const double hi = (double)e;
        t->e2[j] = make_double2(hi, (double)(e - (long double)hi));
    }
    for (int j = 0; j <= F64_TAB; j++) {
        const long double F = 1.0L + (long double)j / (long double)F64_TAB;
        const long double lf = logl(F);
        const double hi = (double)(rintl(lf * 4398046511104.0L) / 4398046511104.0L);   // 2^42 grid
        t->lF[j] = make_double2(hi, (double)(lf - (long double)hi));
        t->invF[j] = (double)(1.0L / F);
    }
    for (int j = 0; j < 64; j++) {
        const double e = exp2((double)j / 64.0);
        const double c = 1.0 + ((double)j + 0.5) / 64.0;
        const double lc = log(c), ic = 1.0 / c;
        const float eh = (float)e, lh = (float)lc, ih = (float)ic;
        t->exp2j[j] = make_float2(eh, (float)(e - (double)eh));
        t->logc[j] = make_float2(lh, (float)(lc - (double)lh));
        t->invc[j] = make_float2(ih, (float)(ic - (double)ih));
    }
}

void launch_closure(cudaStream_t s, int nblk, const Grid &g, const DevSoil *soils, const uint8_t *zone,
                    const double *Ks, const uint8_t *flags, const double *h, const double *hprev,
                    double *theta, double *K, double *Can, double *partials, unsigned int *ticket,
                    StepResults *res)
{
    k_closure<<<nblk, RED_THREADS, 0, s>>>(g, soils, zone, Ks, flags, h, hprev, theta, K, Can, partials, ticket, res);
}

void launch_closure_picard(cudaStream_t s, int nblk, const Grid &g, const DevSoil *soils, const uint8_t *zone,
                           const double *Ks, const uint8_t *flags, const double *x, const double *hk,
                           double *theta, double *K, double *Can, double *partials, unsigned int *ticket,
                           PicardCtl *ctl, const CgScal *cg_status, const CgScal *cg_count, CondSet cond)
{
    k_closure_picard<<<nblk, RED_THREADS, 0, s>>>(g, soils, zone, Ks, flags, x, hk, theta, K, Can, partials, ticket,
                                                  ctl, cg_status, cg_count, cond);
}

void launch_assemble(cudaStream_t s, int nblk, const Grid &g, const DevSoil *soils, const uint8_t *zone,
                     const double *Ks, const uint8_t *flags, const StepParams *sp, const double *hk,
                     const double *hn, const double *theta_k, const double *theta_n, const double *K,
                     const double *Can, double *c, double *b, double *Tx, double *Ty, double *Tz,
                     double *diag, double *dinv, float *K32, float *cb32, float *dinv32, const int *skip,
                     int mode, const SolveStart *start, double *partials, unsigned int *ticket, double *s0,
                     const double *theta_p)
{
    SolveStart st{};
    if (start) st = *start;
    if (mode == ASM_CG64)
        k_assemble<ASM_CG64><<<nblk, RED_THREADS, 0, s>>>(g, soils, zone, Ks, flags, sp, hk, hn, theta_k, theta_n, K,
                                                          Can, c, b, Tx, Ty, Tz, diag, dinv, K32, cb32, dinv32, skip,
                                                          st, partials, ticket, s0, theta_p);
    else if (mode == ASM_MIXED)
        k_assemble<ASM_MIXED><<<nblk, RED_THREADS, 0, s>>>(g, soils, zone, Ks, flags, sp, hk, hn, theta_k, theta_n,
                                                           K, Can, c, b, Tx, Ty, Tz, diag, dinv, K32, cb32, dinv32,
                                                           skip, st, partials, ticket, s0, theta_p);
    else
        k_assemble<ASM_ONLY><<<nblk, RED_THREADS, 0, s>>>(g, soils, zone, Ks, flags, sp, hk, hn, theta_k, theta_n, K,
                                                          Can, c, b, Tx, Ty, Tz, diag, dinv, K32, cb32, dinv32, skip,
                                                          st, partials, ticket, s0, theta_p);
}

void launch_accept(cudaStream_t s, int nblk, const Grid &g, const double *x_final, double *h,
                   const double *theta_k, double *theta_n, const double *K1, double *K0, int copyK)
{
    k_accept<<<nblk, RED_THREADS, 0, s>>>(g, x_final, h, theta_k, theta_n, K1, K0, copyK);
}

void launch_mass_balance(cudaStream_t s, int nblk, const Grid &g, const DevSoil *soils, const uint8_t *zone,
                         const double *Ks, const uint8_t *flags, const StepParams *sp, const double *x_odd,
                         const double *x_even, const double *hn, const double *c, const double *K_odd,
                         const double *K_even, const double *theta_x, const double *theta_n, double *partials,
                         unsigned int *ticket, StepResults *res, const PicardCtl *ctl, const double *s0)
{
    k_mass_balance<<<nblk, RED_THREADS, 0, s>>>(g, soils, zone, Ks, flags, sp, x_odd, x_even, hn, c, K_odd, K_even,
                                                theta_x, theta_n, partials, ticket, res, ctl, s0);
}

void launch_storage(cudaStream_t s, int nblk, const Grid &g, const uint8_t *flags, const double *theta,
                    double *partials, unsigned int *ticket, StepResults *res)
{
    k_storage<<<nblk, RED_THREADS, 0, s>>>(g, flags, theta, partials, ticket, res);
}

}  // namespace rf
