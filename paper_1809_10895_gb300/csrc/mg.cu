// mg.cu -- geometric multigrid V-cycle used as the preconditioner of the FP32
// inner PCG (the paper names multigrid as the more efficient alternative to
// its DIC-PCG for moderate core counts, Sec. 2.2; on one GPU its load-balance
// objection does not apply).
//
// Hierarchy: each level halves the axes whose spacing is within a factor 2 of
// the level's finest spacing (semi-coarsening, so the strongly coupled
// direction of an anisotropic grid is coarsened first), down to a few hundred
// cells.  A coarse cell is active if any child is.  Coarse operators are
// rebuilt after every assembly by face aggregation:
//   T_C,f = (sum of the fine coefficients across the coarse face) * d_fine/d_coarse
//   cb_C  = sum of the children's capacity (+ Dirichlet) terms,
// and every level applies (A e)_P = cb_P e_P + sum_f T_f (e_P - e_N), which is
// an M-matrix.  Smoother: weighted Jacobi (omega = 0.8), two sweeps before and
// two after the coarse correction; transfer: piecewise-constant prolongation
// and its transpose (sum of children).  With equal pre/post sweeps the cycle
// is a symmetric positive-definite preconditioner, as CG requires.  The
// coarsest level is smoothed by one CTA with many sweeps.
#include <math.h>

#include "mg.cuh"
#include "rf_reduce.cuh"

namespace rf {

namespace {

constexpr float OMEGA = 0.8f;

__device__ __forceinline__ void ijk(const MgLevel &L, long long p, int &i, int &j, int &k)
{
    const unsigned int u = (unsigned int)p;
    const unsigned int kk = fdiv(u, L.fxy);
    const unsigned int r = u - kk * (unsigned int)L.sxy;
    const unsigned int jj = fdiv(r, L.fx);
    i = (int)(r - jj * (unsigned int)L.nx);
    j = (int)jj;
    k = (int)kk;
}

// Face coefficient of cell p at level l across face f (0 when no active
// neighbour).  Level 0 recomputes it from the FP32 conductivities.
__device__ __forceinline__ float face_T(const MgLevel &L, const float *__restrict__ K32, long long p, int i, int j,
                                        int k, int f, long long &q)
{
    bool in;
    switch (f) {
    case 0: q = p - 1; in = i > 0; break;
    case 1: q = p + 1; in = i < L.nx - 1; break;
    case 2: q = p - L.nx; in = j > 0; break;
    case 3: q = p + L.nx; in = j < L.ny - 1; break;
    case 4: q = p - L.sxy; in = k > 0; break;
    default: q = p + L.sxy; in = k < L.nz - 1; break;
    }
    if (!in) return 0.0f;
    if (L.level == 0) {
        const float KP = K32[p], KN = K32[q];
        if (!(KP >= 0.0f) || !(KN >= 0.0f)) return 0.0f;   // inactive cells carry K = NaN
        return L.w32[f >> 1] * 0.5f * (KP + KN);
    }
    const float *T = L.T[f >> 1];
    return (f & 1) ? T[p] : T[q];
}

__device__ __forceinline__ bool level_active(const MgLevel &L, const float *__restrict__ K32, long long p)
{
    return L.level == 0 ? K32[p] >= 0.0f : L.dinv[p] > 0.0f;
}

// (A e)_P at level L for an e supplied by get(q)
template <class Get>
__device__ __forceinline__ float apply_level(const MgLevel &L, const float *__restrict__ K32, long long p, Get get)
{
    int i, j, k;
    ijk(L, p, i, j, k);
    const float eP = get(p);
    float acc = L.cb[p] * eP;
#pragma unroll
    for (int f = 0; f < 6; f++) {
        long long q;
        const float T = face_T(L, K32, p, i, j, k, f, q);
        if (T != 0.0f) acc = fmaf(T, eP - get(q), acc);
    }
    return acc;
}

#define LEVEL_LOOP(L, p)                                                                    \
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < (L).N;       \
         p += (long long)gridDim.x * blockDim.x)

// Coarse operator of level c from level f = c - 1.
__global__ void k_mg_build(MgLevel F, MgLevel Cl, const float *__restrict__ K32, const int *skip)
{
    if (skip && *skip) return;
    LEVEL_LOOP(Cl, pc)
    {
        int I, J, Kc;
        ijk(Cl, pc, I, J, Kc);
        const int i0 = I * F.cx, j0 = J * F.cy, k0 = Kc * F.cz;
        float cb = 0.0f, Tsum[6] = {0, 0, 0, 0, 0, 0};
        bool act = false;
        for (int dk = 0; dk < F.cz; dk++)
            for (int dj = 0; dj < F.cy; dj++)
                for (int di = 0; di < F.cx; di++) {
                    const int i = i0 + di, j = j0 + dj, k = k0 + dk;
                    if (i >= F.nx || j >= F.ny || k >= F.nz) continue;
                    const long long p = i + (long long)F.nx * (j + (long long)F.ny * k);
                    if (!level_active(F, K32, p)) continue;
                    act = true;
                    cb += F.cb[p];
                    // faces of this child that lie on the coarse cell's boundary
                    const bool onb[6] = {di == 0, di == F.cx - 1, dj == 0, dj == F.cy - 1, dk == 0, dk == F.cz - 1};
#pragma unroll
                    for (int f = 0; f < 6; f++) {
                        if (!onb[f]) continue;
                        long long q;
                        Tsum[f] += face_T(F, K32, p, i, j, k, f, q);
                    }
                }
        const float sc[3] = {1.0f / (float)F.cx, 1.0f / (float)F.cy, 1.0f / (float)F.cz};
        float diag = cb;
#pragma unroll
        for (int f = 0; f < 6; f++) diag += Tsum[f] * sc[f >> 1];
        Cl.cb[pc] = act ? cb : 0.0f;
        Cl.T[0][pc] = act ? Tsum[1] * sc[0] : 0.0f;
        Cl.T[1][pc] = act ? Tsum[3] * sc[1] : 0.0f;
        Cl.T[2][pc] = act ? Tsum[5] * sc[2] : 0.0f;
        Cl.dinv[pc] = (act && diag > 0.0f) ? 1.0f / diag : 0.0f;
    }
}

// e_out = (first ? 0 : e_in) + omega D^-1 (r - A e_in)
__global__ void k_mg_smooth(MgLevel L, const float *__restrict__ K32, const float *__restrict__ r,
                            const float *__restrict__ e_in, float *__restrict__ e_out, int first, const int *done)
{
    if (done && *done) return;
    LEVEL_LOOP(L, p)
    {
        const float di = L.level == 0 ? L.dinv0[p] : L.dinv[p];
        if (di == 0.0f) { e_out[p] = 0.0f; continue; }
        if (first) {
            e_out[p] = OMEGA * di * r[p];
        } else {
            const float Ae = apply_level(L, K32, p, [&](long long q) { return e_in[q]; });
            e_out[p] = fmaf(OMEGA * di, r[p] - Ae, e_in[p]);
        }
    }
}

// r_c = restriction (sum over children) of r - A e
__global__ void k_mg_restrict(MgLevel F, MgLevel Cl, const float *__restrict__ K32, const float *__restrict__ r,
                              const float *__restrict__ e, float *__restrict__ rc, const int *done)
{
    if (done && *done) return;
    LEVEL_LOOP(Cl, pc)
    {
        int I, J, Kc;
        ijk(Cl, pc, I, J, Kc);
        float s = 0.0f;
        for (int dk = 0; dk < F.cz; dk++)
            for (int dj = 0; dj < F.cy; dj++)
                for (int di = 0; di < F.cx; di++) {
                    const int i = I * F.cx + di, j = J * F.cy + dj, k = Kc * F.cz + dk;
                    if (i >= F.nx || j >= F.ny || k >= F.nz) continue;
                    const long long p = i + (long long)F.nx * (j + (long long)F.ny * k);
                    const float dv = F.level == 0 ? F.dinv0[p] : F.dinv[p];
                    if (dv == 0.0f) continue;
                    s += r[p] - apply_level(F, K32, p, [&](long long q) { return e[q]; });
                }
        rc[pc] = s;
    }
}

__device__ __forceinline__ long long parent(const MgLevel &F, const MgLevel &Cl, long long p)
{
    int i, j, k;
    ijk(F, p, i, j, k);
    return (i / F.cx) + (long long)Cl.nx * ((j / F.cy) + (long long)Cl.ny * (k / F.cz));
}

// e_out = e1 + omega D^-1 (r - A e1) with e1 = e_in + P e_c
__global__ void k_mg_prolong_smooth(MgLevel F, MgLevel Cl, const float *__restrict__ K32,
                                    const float *__restrict__ r, const float *__restrict__ e_in,
                                    const float *__restrict__ ec, float *__restrict__ e_out, const int *done)
{
    if (done && *done) return;
    auto e1 = [&](long long q) { return e_in[q] + ec[parent(F, Cl, q)]; };
    LEVEL_LOOP(F, p)
    {
        const float di = F.level == 0 ? F.dinv0[p] : F.dinv[p];
        if (di == 0.0f) { e_out[p] = 0.0f; continue; }
        const float Ae = apply_level(F, K32, p, e1);
        e_out[p] = fmaf(OMEGA * di, r[p] - Ae, e1(p));
    }
}

// Coarsest level: `sweeps` weighted-Jacobi sweeps from zero, one CTA.
__global__ void k_mg_coarsest(MgLevel L, const float *__restrict__ K32, const float *__restrict__ r,
                              float *__restrict__ ea, float *__restrict__ eb, int sweeps, const int *done)
{
    if (done && *done) return;
    for (long long p = threadIdx.x; p < L.N; p += blockDim.x) ea[p] = OMEGA * L.dinv[p] * r[p];
    __syncthreads();
    float *a = ea, *b = eb;
    for (int s = 1; s < sweeps; s++) {
        for (long long p = threadIdx.x; p < L.N; p += blockDim.x) {
            const float di = L.dinv[p];
            if (di == 0.0f) { b[p] = 0.0f; continue; }
            const float Ae = apply_level(L, K32, p, [&](long long q) { return a[q]; });
            b[p] = fmaf(OMEGA * di, r[p] - Ae, a[p]);
        }
        __syncthreads();
        float *t = a; a = b; b = t;
    }
    if (a != ea)
        for (long long p = threadIdx.x; p < L.N; p += blockDim.x) ea[p] = a[p];
}

}  // namespace

void launch_mg_build(cudaStream_t s, int nblk, const MgHierarchy &H, const float *K32, const int *skip)
{
    for (int l = 0; l + 1 < H.nlev; l++)
        k_mg_build<<<nblk, RED_THREADS, 0, s>>>(H.lev[l], H.lev[l + 1], K32, skip);
}

// z = V-cycle(r) on level 0 (r and z are the inner PCG's FP32 vectors).
void launch_mg_vcycle(cudaStream_t s, int nblk, const MgHierarchy &H, const float *K32, const float *r, float *z,
                      const int *done)
{
    // level 0 arrays: r given, e = z (result) with scratch H.lev[0].e[1]
    const int L = H.nlev;
    const float *rl[MG_MAX_LEVELS];
    float *el[MG_MAX_LEVELS];
    rl[0] = r;
    el[0] = z;
    for (int l = 1; l < L; l++) {
        rl[l] = H.lev[l].r;
        el[l] = H.lev[l].e[0];
    }
    for (int l = 0; l + 1 < L; l++) {
        const MgLevel &F = H.lev[l];
        float *scratch = F.e[1];
        // two pre-smoothing sweeps from zero: el -> scratch -> el
        k_mg_smooth<<<nblk, RED_THREADS, 0, s>>>(F, K32, rl[l], el[l], scratch, 1, done);
        k_mg_smooth<<<nblk, RED_THREADS, 0, s>>>(F, K32, rl[l], scratch, el[l], 0, done);
        k_mg_restrict<<<nblk, RED_THREADS, 0, s>>>(F, H.lev[l + 1], K32, rl[l], el[l], const_cast<float *>(rl[l + 1]),
                                                   done);
    }
    const MgLevel &Cst = H.lev[L - 1];
    k_mg_coarsest<<<1, 1024, 0, s>>>(Cst, K32, rl[L - 1], el[L - 1], Cst.e[1], MG_COARSE_SWEEPS, done);
    for (int l = L - 2; l >= 0; l--) {
        const MgLevel &F = H.lev[l];
        float *scratch = F.e[1];
        // prolongation + first post-smoothing sweep, then the second sweep
        k_mg_prolong_smooth<<<nblk, RED_THREADS, 0, s>>>(F, H.lev[l + 1], K32, rl[l], el[l], el[l + 1], scratch,
                                                         done);
        k_mg_smooth<<<nblk, RED_THREADS, 0, s>>>(F, K32, rl[l], scratch, el[l], 0, done);
    }
}

int mg_vcycle_launches(const MgHierarchy &H) { return 5 * (H.nlev - 1) + 1; }

int mg_plan(int nx, int ny, int nz, double dx, double dy, double dz, MgShape *out, int cap)
{
    int n = 0;
    MgShape s{nx, ny, nz, dx, dy, dz};
    out[n++] = s;
    while (n < cap) {
        const long long cells = (long long)s.nx * s.ny * s.nz;
        if (cells <= MG_COARSEST_CELLS) break;
        double dmin = 1e300;
        if (s.nx > 1) dmin = fmin(dmin, s.dx);
        if (s.ny > 1) dmin = fmin(dmin, s.dy);
        if (s.nz > 1) dmin = fmin(dmin, s.dz);
        if (dmin >= 1e300) break;
        MgShape c = s;
        if (s.nx > 1 && s.dx <= 2.0 * dmin) { c.nx = (s.nx + 1) / 2; c.dx = 2.0 * s.dx; }
        if (s.ny > 1 && s.dy <= 2.0 * dmin) { c.ny = (s.ny + 1) / 2; c.dy = 2.0 * s.dy; }
        if (s.nz > 1 && s.dz <= 2.0 * dmin) { c.nz = (s.nz + 1) / 2; c.dz = 2.0 * s.dz; }
        out[n++] = c;
        s = c;
    }
    return n;
}

// ---------------------------------------------------- PCG kernels for MG
__global__ void __launch_bounds__(RED_THREADS)
k_cg32_update_mg(Grid g, float *__restrict__ x, float *__restrict__ r, const float *__restrict__ pd,
                 const float *__restrict__ q, const float *__restrict__ dinv, double *partials, unsigned int *ticket,
                 CgScal *sc)
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

// rho = r.z after the V-cycle.  start = 1: first preconditioned residual of
// an inner solve (sets rho); otherwise beta = r.z / rho.  Always sets the
// inner loop condition.
__global__ void __launch_bounds__(RED_THREADS)
k_cg32_rz(Grid g, const float *__restrict__ r, const float *__restrict__ z, double *partials, unsigned int *ticket,
          CgScal *sc, int start, CondSet cond)
{
    if (sc->done) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_cond(cond, 0);
        return;
    }
    float a0 = 0.0f;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < g.N;
         p += (long long)gridDim.x * blockDim.x)
        a0 = fmaf(r[p], z[p], a0);
    float vf[1] = {a0};
    double v[1];
    if (grid_reduce_f32<1>(vf, v, partials, ticket) && threadIdx.x == 0) {
        if (!isfinite(v[0]) || !(v[0] > 0.0)) {
            // a zero or non-finite r.z with a non-zero residual: breakdown
            sc->status = CG_NONFINITE;
            sc->done = 1;
        } else if (start) {
            sc->rho = v[0];
            sc->beta = 0.0;
        } else {
            sc->beta = v[0] / sc->rho;
            sc->rho = v[0];
        }
        set_cond(cond, sc->done ? 0 : 1);
    }
}

void launch_cg32_update_mg(cudaStream_t s, int nblk, const Grid &g, float *x, float *r, const float *p,
                           const float *q, const float *dinv, double *partials, unsigned int *ticket, CgScal *sc)
{
    k_cg32_update_mg<<<nblk, RED_THREADS, 0, s>>>(g, x, r, p, q, dinv, partials, ticket, sc);
}

void launch_cg32_rz(cudaStream_t s, int nblk, const Grid &g, const float *r, const float *z, double *partials,
                    unsigned int *ticket, CgScal *sc, int start, CondSet cond)
{
    k_cg32_rz<<<nblk, RED_THREADS, 0, s>>>(g, r, z, partials, ticket, sc, start, cond);
}

}  // namespace rf
