// ensemble.cu -- many independent Richards problems of uneven size in one
// persistent kernel launch (captured in a CUDA graph).
//
// Work unit: a thread-block cluster of CL CTAs (CL chosen by the tuner).  A
// cluster pops an instance from a device queue (instances are ordered largest
// first), splits its cells across its CTAs, and runs that instance's whole
// time integration -- EBATS steps, Picard iterations, PCG -- with the same
// per-cell arithmetic as the single-domain kernels (cell_ops.cuh).  Global
// reductions of the single-domain path become cluster reductions: each CTA
// reduces in shared memory, the cluster barrier publishes the partials, and
// every CTA folds them in rank order through distributed shared memory, so all
// CTAs hold bit-identical scalars and take identical control decisions.
// Every loop is bounded: PCG by max_it, defect correction by outer_max_it,
// Picard by n_max, EBATS by dt_min, and each instance by a step budget.
#include <cooperative_groups.h>

#include "cell_ops.cuh"
#include "ensemble.cuh"
#include "rf_reduce.cuh"

namespace cg = cooperative_groups;

namespace rf {

namespace {

constexpr int RB_SLOTS = 8;

struct ClusterCtx {
    cg::cluster_group cl;
    int rank, ncta;
    double (*red)[RB_SLOTS];   // shared [2][RB_SLOTS]
    int rb;                    // reduction double-buffer index (same in every CTA)
};

// Sum (or max) NV values over all threads of the cluster; every thread gets
// the totals.  Contains a cluster barrier.
template <class Op, int NV>
__device__ __forceinline__ void cl_reduce(ClusterCtx &C, double (&v)[NV])
{
    __shared__ double sm[RB_SLOTS * 32];
    block_reduce<Op, NV>(v, sm);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < NV; i++) C.red[C.rb][i] = v[i];
    }
    C.cl.sync();
#pragma unroll
    for (int i = 0; i < NV; i++) {
        double t = Op::id();
        for (int r = 0; r < C.ncta; r++) t = Op::op(t, C.cl.map_shared_rank(&C.red[C.rb][0], r)[i]);
        v[i] = t;
    }
    C.rb ^= 1;
}

__device__ __forceinline__ double t_tol_d(double t) { return 1e-9 * (fabs(t) > 1.0 ? fabs(t) : 1.0); }

}  // namespace

template <int PREC>
__global__ void __launch_bounds__(ENS_THREADS, 1)
k_ensemble(EnsDesc *__restrict__ D, int n_inst, EnsBuffers B, EnsParams P, const double *t_end_p, unsigned int *queue)
{
    const double t_end = *t_end_p;
    __shared__ double red[2][RB_SLOTS];
    __shared__ int s_inst;
    ClusterCtx C{cg::this_cluster(), 0, 1, red, 0};
    C.rank = (int)C.cl.block_rank();
    C.ncta = (int)C.cl.num_blocks();

    for (;;) {
        if (C.rank == 0 && threadIdx.x == 0) s_inst = (int)atomicAdd(queue, 1u);
        C.cl.sync();
        const int inst = *C.cl.map_shared_rank(&s_inst, 0);
        C.cl.sync();
        if (inst >= n_inst) break;

        EnsDesc &d = D[inst];
        const Grid &g = d.g;
        const long long N = g.N, off = d.off;
        const long long chunk = (N + C.ncta - 1) / C.ncta;
        const long long lo = C.rank * chunk, hi = (lo + chunk < N) ? lo + chunk : N;
        // instance views of the packed arrays
        double *H[3] = {B.H[0] + off, B.H[1] + off, B.H[2] + off};
        double *TH[2] = {B.TH[0] + off, B.TH[1] + off};
        double *KB[2] = {B.K[0] + off, B.K[1] + off};
        double *Can = B.Can + off, *cc = B.c + off, *bb = B.b + off;
        double *Tx = B.Tx + off, *Ty = B.Ty + off, *Tz = B.Tz + off, *dg = B.diag + off, *dinv = B.dinv + off;
        double *r64 = B.r + off, *z64 = B.z + off, *P64[2] = {B.p[0] + off, B.p[1] + off}, *q64 = B.q + off;
        float *K32 = B.K32 + off, *cb32 = B.cb32 + off, *di32 = B.dinv32 + off;
        float *r32 = B.r32 + off, *z32 = B.z32 + off, *P32[2] = {B.p32[0] + off, B.p32[1] + off};
        float *q32 = B.q32 + off, *d32 = B.d32 + off;
        const uint8_t *fl = B.flags + off, *zn = B.zone + off;
        const double *Ks = B.Ks + off;
        const DevSoil *soil = &d.soil;
        StepParams sp = d.sp;

        double t = d.t, dt_nom = d.dt_nom;
        int easy = d.easy, hb = d.hbuf, kb = d.kbuf, tn = d.tnbuf, status = d.status;
        long long steps = d.steps, picard_tot = d.picard, cg_tot = d.cg, rej_tot = d.rejected;
        double in_cum = d.in_cum, out_cum = d.out_cum, clo_cum = d.closure_cum, def_cum = d.defect_cum;
        long long budget = P.step_budget;

        // closures at the current state h (K, theta*_n, C)
        auto closure_at = [&](const double *hx, const double *hprev, double *thx, double *Kx, double (&v)[2]) {
            for (long long p = lo + threadIdx.x; p < hi; p += blockDim.x) {
                const double hp = hx[p];
                if (hprev) {
                    const double dd = fabs(hp - hprev[p]);
                    if (dd <= 1e300) v[0] = fmax(v[0], dd);
                    else v[1] = 1.0;
                }
                double th, k, c;
                closure(*soil, Ks[p], hp, g.tab, th, k, c);
                thx[p] = th;
                Kx[p] = k;
                Can[p] = c;
            }
        };
        if (status == ENS_NEW) {
            double v2[2] = {0.0, 0.0};
            closure_at(H[hb], nullptr, TH[tn], KB[kb], v2);
            double s1[1] = {0.0};
            for (long long p = lo + threadIdx.x; p < hi; p += blockDim.x) s1[0] += g.V * TH[tn][p];
            cl_reduce<OpSum, 1>(C, s1);   // also publishes the closures
            if (C.rank == 0 && threadIdx.x == 0) d.storage0 = s1[0];
            status = ENS_RUNNING;
        }
        bool closure_valid = true;

        while (status == ENS_RUNNING && t < t_end - t_tol_d(t_end)) {
            if (--budget < 0) { status = ENS_BUDGET; break; }
            const double dt_nom0 = dt_nom;
            const int easy0 = easy;
            int rejected = 0, cg_step = 0;
            bool accepted = false;
            for (;;) {                                   // EBATS attempts of one step
                double dt = dt_nom;
                if (t_end - t < dt) dt = t_end - t;
                sp.dt = dt;
                sp.t = t;
                const double V_dt = g.V / dt;
                int hkb = (hb + 1) % 3, xb = (hb + 2) % 3;
                for (long long p = lo + threadIdx.x; p < hi; p += blockDim.x) H[hkb][p] = H[hb][p];
                if (!closure_valid) {
                    double v2[2] = {0.0, 0.0};
                    closure_at(H[hkb], nullptr, TH[tn ^ 1], KB[kb], v2);
                    closure_valid = true;
                }
                C.cl.sync();
                int kin = kb, it = 0, cg_att = 0;
                bool conv = false, fail = false;
                for (it = 1; it <= P.n_max; it++) {
                    const double *hk = H[hkb], *hn = H[hb];
                    double *x = H[xb];
                    // ---- assembly + first residual (Sec. 2.2)
                    double v[4] = {0.0, 0.0, 0.0, 0.0};
                    for (long long p = lo + threadIdx.x; p < hi; p += blockDim.x) {
                        int i, j, k;
                        cell_ijk(g, p, i, j, k);
                        CellSystem cs;
                        assemble_cell<true>(g, soil, zn, Ks, fl[p], sp, p, i, j, k, hk, hn, TH[tn ^ 1], TH[tn],
                                            KB[kin], Can, P.eps_chord, V_dt, cs);
                        const double di = rcp64(cs.diag);
                        cc[p] = cs.c;
                        bb[p] = cs.rhs;
                        Tx[p] = cs.Tup[0];
                        Ty[p] = cs.Tup[1];
                        Tz[p] = cs.Tup[2];
                        dg[p] = cs.diag;
                        dinv[p] = di;
                        K32[p] = (float)cs.KP;
                        cb32[p] = (float)cs.cb;
                        const float d32v = (float)di;
                        di32[p] = d32v;
                        const double hkP = hk[p];
                        const double rp = cs.rhs - (cs.diag * hkP - cs.sT);
                        x[p] = hkP;
                        if (PREC == 0) {
                            const double zp = di * rp;
                            r64[p] = rp;
                            z64[p] = zp;
                            v[0] += rp * zp;
                            v[1] += rp * rp;
                            v[2] += cs.rhs * cs.rhs;
                        } else {
                            const float rf = (float)rp;
                            const float zf = d32v * rf;
                            r32[p] = rf;
                            z32[p] = zf;
                            d32[p] = 0.0f;
                            v[0] += rp * rp;
                            v[1] += cs.rhs * cs.rhs;
                            v[2] += (double)(rf * rf);
                            v[3] += (double)(rf * zf);
                        }
                    }
                    cl_reduce<OpSum, 4>(C, v);
                    int cg_it = 0;
                    bool lin_ok = true;
                    if (PREC == 0) {
                        // ---- FP64 Jacobi-PCG
                        double rho = v[0];
                        const double stop = P.tol_cg * sqrt(v[2]);
                        bool done = !(isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]));
                        if (done) lin_ok = false;
                        else done = sqrt(v[1]) <= stop;
                        double beta = 0.0;
                        int pi = 0;
                        while (!done) {
                            double *pin = P64[pi], *pout = P64[pi ^ 1];
                            const bool first = cg_it == 0;
                            auto get = [&](long long qq) { return first ? z64[qq] : fma(beta, pin[qq], z64[qq]); };
                            double w1[1] = {0.0};
                            for (long long p = lo + threadIdx.x; p < hi; p += blockDim.x) {
                                const double pp = get(p);
                                const double qp = apply64(g, p, Tx, Ty, Tz, dg, get);
                                pout[p] = pp;
                                q64[p] = qp;
                                w1[0] += pp * qp;
                            }
                            cl_reduce<OpSum, 1>(C, w1);
                            const double alpha = rho / w1[0];
                            if (!(w1[0] > 0.0) || !isfinite(alpha)) { lin_ok = false; break; }
                            double w2[2] = {0.0, 0.0};
                            for (long long p = lo + threadIdx.x; p < hi; p += blockDim.x) {
                                x[p] = fma(alpha, pout[p], x[p]);
                                const double rp2 = fma(-alpha, q64[p], r64[p]);
                                const double zp2 = dinv[p] * rp2;
                                r64[p] = rp2;
                                z64[p] = zp2;
                                w2[0] += rp2 * rp2;
                                w2[1] += rp2 * zp2;
                            }
                            cl_reduce<OpSum, 2>(C, w2);
                            cg_it++;
                            pi ^= 1;
                            if (!isfinite(w2[0]) || !isfinite(w2[1])) { lin_ok = false; break; }
                            if (sqrt(w2[0]) <= stop) break;
                            if (cg_it >= P.cg_max_it) { lin_ok = false; break; }
                            beta = w2[1] / rho;
                            rho = w2[1];
                        }
                    } else {
                        // ---- FP32 inner PCG inside FP64 defect correction
                        int outer = 1;
                        for (;;) {
                            const bool finite = isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]) && isfinite(v[3]);
                            if (!finite) { lin_ok = false; break; }
                            if (sqrt(v[0]) <= P.tol_cg * sqrt(v[1])) break;
                            if (outer >= P.outer_max_it) { lin_ok = false; break; }
                            // inner solve A d = r32 from d = 0
                            double rho = v[3];
                            const double stop = P.tol_inner * sqrt(v[2]);
                            bool done = !(v[2] > 0.0);
                            float beta = 0.0f;
                            int pi = 0, inner_it = 0;
                            while (!done) {
                                float *pin = P32[pi], *pout = P32[pi ^ 1];
                                const bool first = inner_it == 0;
                                auto get = [&](long long qq) { return first ? z32[qq] : fmaf(beta, pin[qq], z32[qq]); };
                                float a0 = 0.0f;
                                for (long long p = lo + threadIdx.x; p < hi; p += blockDim.x) {
                                    const float pp = get(p);
                                    const float qp = apply32(g, p, K32, cb32, get);
                                    pout[p] = pp;
                                    q32[p] = qp;
                                    a0 = fmaf(pp, qp, a0);
                                }
                                double w1[1] = {(double)a0};
                                cl_reduce<OpSum, 1>(C, w1);
                                const double alpha = rho / w1[0];
                                if (!(w1[0] > 0.0) || !isfinite(alpha)) { lin_ok = false; break; }
                                const float af = (float)alpha;
                                float b0 = 0.0f, b1 = 0.0f;
                                for (long long p = lo + threadIdx.x; p < hi; p += blockDim.x) {
                                    d32[p] = fmaf(af, pout[p], d32[p]);
                                    const float rp2 = fmaf(-af, q32[p], r32[p]);
                                    const float zp2 = di32[p] * rp2;
                                    r32[p] = rp2;
                                    z32[p] = zp2;
                                    b0 = fmaf(rp2, rp2, b0);
                                    b1 = fmaf(rp2, zp2, b1);
                                }
                                double w2[2] = {(double)b0, (double)b1};
                                cl_reduce<OpSum, 2>(C, w2);
                                inner_it++;
                                pi ^= 1;
                                if (!isfinite(w2[0]) || !isfinite(w2[1])) { lin_ok = false; break; }
                                if (sqrt(w2[0]) <= stop || inner_it >= P.inner_max_it) break;
                                beta = (float)(w2[1] / rho);
                                rho = w2[1];
                            }
                            cg_it += inner_it;
                            if (!lin_ok) break;
                            for (long long p = lo + threadIdx.x; p < hi; p += blockDim.x) x[p] += (double)d32[p];
                            C.cl.sync();
                            // FP64 outer residual and new inner seeds
                            v[0] = v[1] = v[2] = v[3] = 0.0;
                            for (long long p = lo + threadIdx.x; p < hi; p += blockDim.x) {
                                const double bp = bb[p];
                                const double rp = bp - apply64(g, p, Tx, Ty, Tz, dg, [&](long long qq) { return x[qq]; });
                                const float rf = (float)rp;
                                const float zf = di32[p] * rf;
                                r32[p] = rf;
                                z32[p] = zf;
                                d32[p] = 0.0f;
                                v[0] += rp * rp;
                                v[1] += bp * bp;
                                v[2] += (double)(rf * rf);
                                v[3] += (double)(rf * zf);
                            }
                            cl_reduce<OpSum, 4>(C, v);
                            outer++;
                        }
                    }
                    if (!lin_ok) { fail = true; break; }
                    cg_att += cg_it;
                    // ---- closures at the new iterate and the global Picard test (Sec. 2.3)
                    double w[2] = {0.0, 0.0};
                    closure_at(x, hk, TH[tn ^ 1], KB[kin ^ 1], w);
                    cl_reduce<OpMax, 2>(C, w);
                    const int kold = kin;
                    kin ^= 1;
                    { const int tmp = hkb; hkb = xb; xb = tmp; }
                    if (w[1] > 0.0) { fail = true; break; }
                    if (w[0] <= P.tol_picard) {
                        conv = true;
                        // water balance of this last linear system (x = H[hkb])
                        double m4[4] = {0.0, 0.0, 0.0, 0.0};
                        const double *xf = H[hkb];
                        for (long long p = lo + threadIdx.x; p < hi; p += blockDim.x) {
                            const double xp = xf[p], hnP = hn[p];
                            m4[0] += cc[p] * dt * (xp - hnP);
                            m4[1] += g.V * (TH[tn ^ 1][p] - TH[tn][p]);
                            if (fl[p] & 0x3f) {
                                double fin, fout;
                                boundary_fluxes(g, *soil, Ks[p], fl[p], sp, xp, hnP, KB[kold][p], fin, fout);
                                m4[2] += dt * fin;
                                m4[3] += dt * fout;
                            }
                        }
                        cl_reduce<OpSum, 4>(C, m4);
                        const double net = m4[2] - m4[3];
                        in_cum += m4[2];
                        out_cum += m4[3];
                        clo_cum += m4[0] - net;
                        def_cum += m4[1] - net;
                        break;
                    }
                }
                if (it > P.n_max) it = P.n_max;
                cg_step += cg_att;
                if (conv) {
                    // accept: the converged iterate becomes h, its closures stay
                    hb = hkb;
                    tn ^= 1;
                    kb = kin;
                    double tn1 = t + dt;
                    if (fabs(tn1 - t_end) <= t_tol_d(tn1)) tn1 = t_end;
                    t = tn1;
                    steps++;
                    picard_tot += it;
                    cg_tot += cg_step;
                    rej_tot += rejected;
                    if (it <= P.n_small) easy++;
                    else easy = 0;
                    if (easy >= P.n_inc) {
                        dt_nom = fmin(dt_nom * P.f_grow, P.dt_max);
                        easy = 0;
                    }
                    accepted = true;
                    break;
                }
                (void)fail;
                rejected++;
                dt_nom = dt / P.f_shrink;
                easy = 0;
                closure_valid = false;
                if (dt_nom < P.dt_min) {
                    dt_nom = dt_nom0;
                    easy = easy0;
                    status = ENS_DT_MIN;
                    break;
                }
                C.cl.sync();
            }
            if (!accepted) break;
        }
        C.cl.sync();
        if (C.rank == 0 && threadIdx.x == 0) {
            d.t = t;
            d.dt_nom = dt_nom;
            d.easy = easy;
            d.hbuf = hb;
            d.kbuf = kb;
            d.tnbuf = tn;
            d.status = status;
            d.steps = steps;
            d.picard = picard_tot;
            d.cg = cg_tot;
            d.rejected = rej_tot;
            d.in_cum = in_cum;
            d.out_cum = out_cum;
            d.closure_cum = clo_cum;
            d.defect_cum = def_cum;
        }
        C.cl.sync();
    }
}

cudaError_t launch_ensemble(cudaStream_t s, int cluster, int nclusters, int precision, EnsDesc *D, int n_inst,
                            const EnsBuffers &B, const EnsParams &P, const double *t_end, unsigned int *queue)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(cluster * nclusters), 1, 1);
    cfg.blockDim = dim3(ENS_THREADS, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (precision == 0) return cudaLaunchKernelEx(&cfg, k_ensemble<0>, D, n_inst, B, P, t_end, queue);
    return cudaLaunchKernelEx(&cfg, k_ensemble<1>, D, n_inst, B, P, t_end, queue);
}

int ensemble_max_clusters(int cluster, int precision)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)cluster, 1, 1);
    cfg.blockDim = dim3(ENS_THREADS, 1, 1);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    const cudaError_t e = precision == 0
                              ? cudaOccupancyMaxActiveClusters(&n, (void *)k_ensemble<0>, &cfg)
                              : cudaOccupancyMaxActiveClusters(&n, (void *)k_ensemble<1>, &cfg);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

}  // namespace rf
