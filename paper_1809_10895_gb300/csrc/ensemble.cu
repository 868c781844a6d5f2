// ensemble.cu -- many independent Richards problems of uneven size in one
// persistent kernel launch (captured in a CUDA graph).
//
// Work unit: a thread-block cluster of CL CTAs (CL chosen by the tuner) for
// the heavy instances, a single CTA for the others.  The work queue is a
// schedule: a list of instances, the "wide" ones first (by default every
// instance, largest first; the tuner orders it by measured work).  While the
// queue yields wide instances, a cluster pops one, splits its cells across
// its CTAs, and runs that instance's whole time integration -- EBATS steps,
// Picard iterations, PCG -- with the same per-cell arithmetic as the
// single-domain kernels (cell_ops.cuh).  Global reductions of the
// single-domain path become cluster reductions: each CTA reduces in shared
// memory, the cluster barrier publishes the partials, and every CTA folds
// them in the same order through distributed shared memory, so all CTAs hold
// bit-identical scalars and take identical control decisions.  Once the
// queue reaches the other instances the cluster's CTAs go solo: each pops and
// runs instances on its own, with block barriers and block reductions in
// place of the cluster ones.
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
constexpr int RB_WARPS = 16;   // warps of the largest CTA (512 threads)

struct ClusterCtx {
    cg::cluster_group cl;
    int rank, ncta;                        // rank 0, ncta 1 when solo
    bool solo;                             // this CTA runs its instance alone
    double (*red)[RB_SLOTS][RB_WARPS];     // shared [2][RB_SLOTS][RB_WARPS]: per-warp FP64 partials
    double (*bc)[RB_SLOTS];                // shared [2][RB_SLOTS]: FP64 totals for the whole CTA
    float (*redf)[RB_SLOTS][RB_WARPS];     // shared [2][RB_SLOTS][RB_WARPS]: per-warp FP32 partials
    double *part;                          // shared [RB_PART][blockDim]: per-thread FP64 partials
    int rb;                                // reduction double-buffer index (same in every CTA)
};

constexpr int RB_PART = 4;   // FP64 values a single-CTA reduction stages per thread

// Finisher of a reduction that derives nothing.
struct NoFin {
    template <int NV>
    __device__ void operator()(const double (&)[NV], double *) const {}
};

// Barrier over the threads that share the current instance.
__device__ __forceinline__ void unit_sync(ClusterCtx &C)
{
    if (C.solo) __syncthreads();
    else C.cl.sync();
}

struct FSum {
    __device__ static float id() { return 0.0f; }
    __device__ static float op(float a, float b) { return a + b; }
};

// Butterfly (xor) reduction: every lane ends with the same bits, because
// each level combines the same two operands in every lane of a pair.
template <class Op, class T>
__device__ __forceinline__ T warp_allreduce(T x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = Op::op(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}

// Tree reduction to lane 0.
template <class Op>
__device__ __forceinline__ double warp_reduce_lane0(double x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = Op::op(x, __shfl_down_sync(0xffffffffu, x, o));
    return x;
}

// Sum (or max) NV FP64 values over all threads of the instance's CTAs; every
// thread gets the totals, bit-identical in every CTA, and the ND scalars
// fin(totals, d) derives from them (computed once, by one thread, and
// broadcast: a divide or square root that every thread repeated would cost
// the narrow FP64 pipe of this GPU hundreds of cycles).  FP64 adds are kept
// few for the same reason.  On one CTA every thread stages its values in
// shared memory and warp 0 sums them (nw values a lane, then one tree).  On
// a cluster each warp reduces its values to lane 0, which publishes them;
// one cluster barrier; warp 0 of every CTA folds all partials of all CTAs
// (lane l reads partials l, l+32, ..., remote ones through distributed
// shared memory, all loads in flight at once), in the same order in every
// CTA.  A block barrier then hands the results to the other warps.  The
// double-buffered slots are rewritten two reductions later, after the next
// barrier, which every reader has passed; the per-thread slots are rewritten
// only after this reduction's last barrier.
template <class Op, int NV, int ND = 0, class Fin = NoFin>
__device__ __forceinline__ void cl_reduce(ClusterCtx &C, double (&v)[NV], double *d = nullptr, Fin fin = Fin{})
{
    static_assert(NV + ND <= RB_SLOTS && NV <= RB_PART, "reduction slots");
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double t[NV];
    if (C.ncta == 1) {
#pragma unroll
        for (int i = 0; i < NV; i++) C.part[i * blockDim.x + threadIdx.x] = v[i];
        __syncthreads();
        if (wid == 0) {
#pragma unroll
            for (int i = 0; i < NV; i++) t[i] = Op::id();
            for (int w = 0; w < nw; w++) {
#pragma unroll
                for (int i = 0; i < NV; i++) t[i] = Op::op(t[i], C.part[i * blockDim.x + 32 * w + lane]);
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < NV; i++) v[i] = warp_reduce_lane0<Op>(v[i]);
        if (lane == 0) {
#pragma unroll
            for (int i = 0; i < NV; i++) C.red[C.rb][i][wid] = v[i];
        }
        unit_sync(C);
        if (wid == 0) {
            const int total = C.ncta * nw;   // <= 8 * 16
#pragma unroll
            for (int i = 0; i < NV; i++) t[i] = Op::id();
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int s = lane + 32 * u;
                if (s < total) {
                    const int r = s / nw, w = s - r * nw;
                    const double *src = C.cl.map_shared_rank(&C.red[C.rb][0][w], r);
#pragma unroll
                    for (int i = 0; i < NV; i++) t[i] = Op::op(t[i], src[i * RB_WARPS]);
                }
            }
        }
    }
    if (wid == 0) {
#pragma unroll
        for (int i = 0; i < NV; i++) t[i] = warp_reduce_lane0<Op>(t[i]);
        if (lane == 0) {
#pragma unroll
            for (int i = 0; i < NV; i++) C.bc[C.rb][i] = t[i];
            if constexpr (ND > 0) {
                double dd[ND];
                fin(t, dd);
#pragma unroll
                for (int i = 0; i < ND; i++) C.bc[C.rb][NV + i] = dd[i];
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NV; i++) v[i] = C.bc[C.rb][i];
    if constexpr (ND > 0) {
#pragma unroll
        for (int i = 0; i < ND; i++) d[i] = C.bc[C.rb][NV + i];
    }
    C.rb ^= 1;
}

// FP32 sums for the inner PCG: FP32 adds are cheap, so every warp folds all
// partials itself (butterflies, identical bits in every lane, warp and CTA)
// and the reduction costs one barrier.
template <int NV>
__device__ __forceinline__ void cl_reduce_f32(ClusterCtx &C, float (&v)[NV])
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; i++) v[i] = warp_allreduce<FSum>(v[i]);
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < NV; i++) C.redf[C.rb][i][wid] = v[i];
    }
    unit_sync(C);
    const int total = C.ncta * nw;
    float t[NV];
#pragma unroll
    for (int i = 0; i < NV; i++) t[i] = FSum::id();
#pragma unroll
    for (int u = 0; u < 4; u++) {
        const int s = lane + 32 * u;
        if (s < total) {
            const int r = s / nw, w = s - r * nw;
            const float *src = C.solo ? &C.redf[C.rb][0][w] : C.cl.map_shared_rank(&C.redf[C.rb][0][w], r);
#pragma unroll
            for (int i = 0; i < NV; i++) t[i] = FSum::op(t[i], src[i * RB_WARPS]);
        }
    }
#pragma unroll
    for (int i = 0; i < NV; i++) v[i] = warp_allreduce<FSum>(t[i]);
    C.rb ^= 1;
}

// The grid fields the FP32 operator reads, held in registers by value.
struct Geo32 {
    FastDiv fx, fxy;
    int nx, ny, nz, sxy;
    float w[3];
};

__device__ __forceinline__ Geo32 geo32(const Grid &g)
{
    return Geo32{g.fx, g.fxy, g.nx, g.ny, g.nz, (int)g.sxy, {g.w32[0], g.w32[1], g.w32[2]}};
}

// FP32 operator of cell p, (A v)_p = cb_p v_p + sum over interior faces of
// w (K_P + K_N)/2 (v_p - v_N), faces recomputed from FP32 K (a neighbour with
// K < 0 is inactive); 32-bit indices.  Both loads of a face issue before the
// inactive test, so a cell costs one memory round trip.
template <class Get>
__device__ __forceinline__ float apply32_i(const Geo32 &g, int p, const float *__restrict__ K32,
                                           const float *__restrict__ cb32, Get get)
{
    const unsigned int u = (unsigned int)p;
    const unsigned int kk = fdiv(u, g.fxy);
    const unsigned int r = u - kk * (unsigned int)g.sxy;
    const unsigned int jj = fdiv(r, g.fx);
    const int i = (int)(r - jj * (unsigned int)g.nx), j = (int)jj, k = (int)kk;
    const float KP = K32[p];
    const float vP = get(p);
    float acc = cb32[p] * vP;
    auto face = [&](bool inside, int q, float w) {
        if (!inside) return;
        const float KN = K32[q];
        const float vN = get(q);
        const float t = fmaf(w * 0.5f * (KP + KN), vP - vN, acc);
        acc = KN < 0.0f ? acc : t;
    };
    face(i > 0, p - 1, g.w[0]);
    face(i < g.nx - 1, p + 1, g.w[0]);
    face(j > 0, p - g.nx, g.w[1]);
    face(j < g.ny - 1, p + g.nx, g.w[1]);
    face(k > 0, p - g.sxy, g.w[2]);
    face(k < g.nz - 1, p + g.sxy, g.w[2]);
    return acc;
}

// Vertical-line preconditioner M: the FP32 operator without its horizontal
// faces.  Per column (i, j) of an instance it is the tridiagonal matrix with
// diagonal cb_k + the two vertical face terms and off-diagonals
// lo_k = -wz (K_{k-1} + K_k)/2 (row k to k - 1) and up_k = lo_{k+1}:
// symmetric and diagonally dominant with cb > 0, so elimination needs no
// pivoting.  A - M is the horizontal graph Laplacian (positive
// semi-definite), so every eigenvalue of M^-1 A is >= 1, and M^-1 is exact on
// residuals that are uniform across the columns, where the horizontal faces
// carry no flux.
//
// Each column is solved by the partition method (substructuring), cut into
// Pn segments of L cells so that a deep column uses many threads: work item
// (column, segment) s = [a, b) with local matrix M_s (the rows of the
// segment without its couplings to cells a - 1 and b) holds, per cell,
// the local factors (1/pivot, c/pivot) and P_k = lo_a (M_s^-1 e_a)_k,
// Q_k = up_{b-1} (M_s^-1 e_{b-1})_k.  With y = M_s^-1 r on the segment, the
// solution is z_k = y_k - P_k z_{a-1} - Q_k z_b, and the segments' end values
// E_s = z_a, F_s = z_{b-1} solve a reduced system with one forward and one
// backward sweep per column over its segments (factors kept at each
// segment's first cell).  Segments: as many as the unit has threads per
// column, at most 32, at least 4 cells each.
constexpr int ZB = 16;      // cells of a segment loaded ahead of its recurrence
constexpr int ZSEG_MAX = 32;

struct ZSeg {
    int L, Pn;              // cells per segment, segments per column
};

__device__ __forceinline__ ZSeg zline_segs(const ClusterCtx &C, const Geo32 &g)
{
    int P = (C.ncta * (int)blockDim.x) / g.sxy;
    P = min(P, ZSEG_MAX);
    P = min(P, g.nz / 4);
    P = max(P, 1);
    const int L = (g.nz + P - 1) / P;
    return ZSeg{L, (g.nz + L - 1) / L};
}

// Factors of every (column, segment), then the reduced system's per column.
// Contains a unit barrier: every thread of the unit calls it.
__device__ __noinline__ void zline_factor32(ClusterCtx &C, const Geo32 g, const float *__restrict__ K32,
                                            const float *__restrict__ cb32, float *__restrict__ lt_inv,
                                            float *__restrict__ lt_c, float *__restrict__ lt_P,
                                            float *__restrict__ lt_Q, float4 *__restrict__ lt_rs)
{
    const int T = C.ncta * (int)blockDim.x, t0 = C.rank * (int)blockDim.x + (int)threadIdx.x;
    const int nz = g.nz, s = g.sxy;
    const float hw = 0.5f * g.w[2];
    const ZSeg zs = zline_segs(C, g);
    for (int w = t0; w < s * zs.Pn; w += T) {
        const int col = w % s, seg = w / s;
        const int a = seg * zs.L, b = min(a + zs.L, nz);
        // forward: pivots, c' and w = M_s^-1 e_a before back substitution (kept in lt_P)
        float Kk = K32[col + a * s], Kb = a > 0 ? K32[col + (a - 1) * s] : 0.0f;   // K of cells k and k - 1
        float lo = 0.0f, cp = 0.0f, wv = 0.0f;   // coupling to the cell below (0 at the segment's start); c'_{k-1}; w_{k-1}
        for (int k0 = a; k0 < b; k0 += ZB) {
            float Kup[ZB], cbv[ZB];
#pragma unroll
            for (int u = 0; u < ZB; u++) {
                const int k = k0 + u;
                Kup[u] = k + 1 < nz && k < b ? K32[col + (k + 1) * s] : 0.0f;
                cbv[u] = k < b ? cb32[col + k * s] : 1.0f;
            }
#pragma unroll
            for (int u = 0; u < ZB; u++) {
                const int k = k0 + u;
                if (k < b) {
                    const float up = k + 1 < nz ? -hw * (Kk + Kup[u]) : 0.0f;   // row k to k + 1 (full operator)
                    const float lof = k > 0 ? -hw * (Kb + Kk) : 0.0f;
                    const float diag = cbv[u] - lof - up;
                    const float upl = k + 1 < b ? up : 0.0f;   // within the segment
                    const float inv = 1.0f / fmaf(-lo, cp, diag);
                    wv = k == a ? inv : -lo * wv * inv;
                    cp = upl * inv;
                    lt_inv[col + k * s] = inv;
                    lt_c[col + k * s] = cp;
                    lt_P[col + k * s] = wv;
                    lo = upl;
                    Kb = Kk;
                    Kk = Kup[u];
                }
            }
        }
        // backward: p = M_s^-1 e_a, q = M_s^-1 e_{b-1}, scaled by the outside couplings
        const float la = a > 0 ? -hw * (K32[col + (a - 1) * s] + K32[col + a * s]) : 0.0f;
        const float ub = b < nz ? -hw * (K32[col + (b - 1) * s] + K32[col + b * s]) : 0.0f;
        float pn = 0.0f, qn = 0.0f;
        for (int k = b - 1; k >= a; k--) {
            const float c = lt_c[col + k * s], wk = lt_P[col + k * s];
            const float pk = k == b - 1 ? wk : fmaf(-c, pn, wk);
            const float qk = k == b - 1 ? lt_inv[col + k * s] : -c * qn;
            lt_P[col + k * s] = la * pk;
            lt_Q[col + k * s] = ub * qk;
            pn = pk;
            qn = qk;
        }
    }
    if (zs.Pn == 1) return;   // one segment: no reduced system (uniform over the unit)
    unit_sync(C);             // every segment's P, Q published
    for (int col = t0; col < s; col += T) {
        float gp = 0.0f;
        for (int seg = 0; seg < zs.Pn; seg++) {
            const int a = seg * zs.L, b = min(a + zs.L, nz);
            const float al = lt_P[col + a * s], ga = lt_P[col + (b - 1) * s];
            const float be = lt_Q[col + a * s], de = lt_Q[col + (b - 1) * s];
            const float iv = 1.0f / fmaf(-al, gp, 1.0f);
            const float h = be * iv;
            const float gn = fmaf(ga * gp, h, de);
            lt_rs[col + a * s] = make_float4(iv, h, gn, ga * gp);
            gp = gn;
        }
    }
}

// z = M^-1 r on this thread's work items: y = M_s^-1 r per segment (into
// z32), the reduced system per column (segment end values into ef), then
// z = y - P F_{s-1} - Q E_{s+1}; returns this thread's share of r . z.
// With several segments per column it contains two unit barriers: every
// thread of the unit calls it.  ef is scratch of the instance's size.
__device__ __noinline__ float zline_solve32(ClusterCtx &C, const Geo32 g, const float *__restrict__ K32,
                                            const float *__restrict__ lt_inv, const float *__restrict__ lt_c,
                                            const float *__restrict__ lt_P, const float *__restrict__ lt_Q,
                                            const float4 *__restrict__ lt_rs, const float *__restrict__ r32,
                                            float *__restrict__ z32, float *__restrict__ ef)
{
    const int T = C.ncta * (int)blockDim.x, t0 = C.rank * (int)blockDim.x + (int)threadIdx.x;
    const int nz = g.nz, s = g.sxy;
    const float hw = 0.5f * g.w[2];
    const ZSeg zs = zline_segs(C, g);
    const bool one = zs.Pn == 1;
    float rz = 0.0f;
    for (int w = t0; w < s * zs.Pn; w += T) {
        const int col = w % s, seg = w / s;
        const int a = seg * zs.L, b = min(a + zs.L, nz);
        // forward: t_k = (r_k - lo_k t_{k-1}) / pivot_k, lo_k = -wz (K_{k-1} + K_k)/2 inside the segment
        float y = 0.0f, Kb = 0.0f;
        for (int k0 = a; k0 < b; k0 += ZB) {
            float rv[ZB], Kv[ZB], iv[ZB];
#pragma unroll
            for (int u = 0; u < ZB; u++) {
                const int k = k0 + u;
                const bool in = k < b;
                rv[u] = in ? r32[col + k * s] : 0.0f;
                Kv[u] = in ? K32[col + k * s] : 0.0f;
                iv[u] = in ? lt_inv[col + k * s] : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < ZB; u++) {
                const int k = k0 + u;
                if (k < b) {
                    const float lo = k > a ? -hw * (Kb + Kv[u]) : 0.0f;
                    y = fmaf(-lo, y, rv[u]) * iv[u];
                    z32[col + k * s] = y;
                    Kb = Kv[u];
                }
            }
        }
        // backward: y_k = t_k - c'_k y_{k+1} (c' = 0 at the segment's last cell)
        float yn = 0.0f;
        for (int k0 = b - 1; k0 >= a; k0 -= ZB) {
            float tv[ZB], cv[ZB], rv[ZB];
#pragma unroll
            for (int u = 0; u < ZB; u++) {
                const int k = k0 - u;
                const bool in = k >= a;
                tv[u] = in ? z32[col + k * s] : 0.0f;
                cv[u] = in ? lt_c[col + k * s] : 0.0f;
                rv[u] = in && one ? r32[col + k * s] : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < ZB; u++) {
                const int k = k0 - u;
                if (k >= a) {
                    yn = fmaf(-cv[u], yn, tv[u]);
                    z32[col + k * s] = yn;
                    rz = fmaf(rv[u], yn, rz);   // one segment: y is z
                }
            }
        }
    }
    if (one) return rz;   // uniform over the unit
    unit_sync(C);
    // reduced system, one thread per column: forward over the segments
    // (e'_s, f'_s into ef at the segment's ends), then backward (E_s, F_s)
    constexpr int ZR = 8;
    for (int col = t0; col < s; col += T) {
        float f = 0.0f;
        for (int s0 = 0; s0 < zs.Pn; s0 += ZR) {
            float ya[ZR], yb[ZR], al[ZR], ga[ZR];
            float4 rs[ZR];
#pragma unroll
            for (int u = 0; u < ZR; u++) {
                const int sg = s0 + u;
                const int a = sg * zs.L, b = min(a + zs.L, nz);
                const bool in = sg < zs.Pn;
                ya[u] = in ? z32[col + a * s] : 0.0f;
                yb[u] = in ? z32[col + (b - 1) * s] : 0.0f;
                al[u] = in ? lt_P[col + a * s] : 0.0f;
                ga[u] = in ? lt_P[col + (b - 1) * s] : 0.0f;
                rs[u] = in ? lt_rs[col + a * s] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            }
#pragma unroll
            for (int u = 0; u < ZR; u++) {
                const int sg = s0 + u;
                if (sg < zs.Pn) {
                    const int a = sg * zs.L, b = min(a + zs.L, nz);
                    const float e = fmaf(-al[u], f, ya[u]) * rs[u].x;
                    f = fmaf(rs[u].w, e, fmaf(-ga[u], f, yb[u]));
                    ef[col + a * s] = e;
                    ef[col + (b - 1) * s] = f;   // the same cell when the segment has one cell (then f = e)
                }
            }
        }
        float En = 0.0f;
        for (int s0 = zs.Pn - 1; s0 >= 0; s0 -= ZR) {
            float ev[ZR], fv[ZR];
            float4 rs[ZR];
#pragma unroll
            for (int u = 0; u < ZR; u++) {
                const int sg = s0 - u;
                const int a = sg * zs.L, b = min(a + zs.L, nz);
                const bool in = sg >= 0;
                ev[u] = in ? ef[col + a * s] : 0.0f;
                fv[u] = in ? ef[col + (b - 1) * s] : 0.0f;
                rs[u] = in ? lt_rs[col + a * s] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            }
#pragma unroll
            for (int u = 0; u < ZR; u++) {
                const int sg = s0 - u;
                if (sg >= 0) {
                    const int a = sg * zs.L, b = min(a + zs.L, nz);
                    const float E = fmaf(-rs[u].y, En, ev[u]), F = fmaf(-rs[u].z, En, fv[u]);
                    ef[col + a * s] = E;
                    ef[col + (b - 1) * s] = F;
                    En = E;
                }
            }
        }
    }
    unit_sync(C);
    // combination, every segment in parallel
    for (int w = t0; w < s * zs.Pn; w += T) {
        const int col = w % s, seg = w / s;
        const int a = seg * zs.L, b = min(a + zs.L, nz);
        const float Fp = seg > 0 ? ef[col + (a - 1) * s] : 0.0f;
        const float En = seg + 1 < zs.Pn ? ef[col + b * s] : 0.0f;
#pragma unroll 4
        for (int k = a; k < b; k++) {
            const int p = col + k * s;
            const float z = fmaf(-lt_Q[p], En, fmaf(-lt_P[p], Fp, z32[p]));
            z32[p] = z;
            rz = fmaf(r32[p], z, rz);
        }
    }
    return rz;
}

// Inner FP32 PCG of one defect-correction pass, A d = r32 from d = 0, on
// this CTA's cells [lo, hi) of an instance (views offset to the instance);
// scalars in FP32 too, since every thread computes them.  Preconditioner:
// Jacobi (z32 and rho = r.z from the caller), or with zline the vertical-line
// solve (factors lt_inv, lt_c).  Kept out of line so that its loops get
// registers of their own, apart from the instance state of the caller.
// Returns false on breakdown; its = inner iterations.
template <bool zline>
__device__ __noinline__ bool inner_pcg32(ClusterCtx &C, const Geo32 g, int lo, int hi, const float *__restrict__ K32,
                                         const float *__restrict__ cb32, const float *__restrict__ di32,
                                         float *__restrict__ r32, float *__restrict__ z32, float *__restrict__ pa_,
                                         float *__restrict__ pb_, float *__restrict__ q32, float *__restrict__ d32,
                                         const float *__restrict__ lt_inv, const float *__restrict__ lt_c,
                                         const float *__restrict__ lt_P, const float *__restrict__ lt_Q,
                                         const float4 *__restrict__ lt_rs, float rho, float stop, int max_it, int &its)
{
    float beta = 0.0f;
    int pi = 0;
    its = 0;
    const int bd = (int)blockDim.x;
    if constexpr (zline) {
        // r32 was published by the caller's reduction barrier
        float w0[1] = {zline_solve32(C, g, K32, lt_inv, lt_c, lt_P, lt_Q, lt_rs, r32, z32, q32)};
        cl_reduce_f32<1>(C, w0);   // also publishes z32
        rho = w0[0];
        if (!(rho > 0.0f) || !isfinite(rho)) return false;
    }
    for (;;) {
        float *pin = pi ? pb_ : pa_, *pout = pi ? pa_ : pb_;
        const bool first = its == 0;
        auto get = [&](int qq) { return first ? z32[qq] : fmaf(beta, pin[qq], z32[qq]); };
        // two cells per thread and pass, all loads of both before any store,
        // so their round trips overlap (same accumulation order as one cell
        // per pass)
        float a0 = 0.0f;
        for (int p = lo + (int)threadIdx.x; p < hi; p += 2 * bd) {
            const bool has2 = p + bd < hi;
            const int p2 = has2 ? p + bd : p;
            const float pp = get(p);
            const float qp = apply32_i(g, p, K32, cb32, get);
            const float pp2 = get(p2);
            const float qp2 = apply32_i(g, p2, K32, cb32, get);
            pout[p] = pp;
            q32[p] = qp;
            a0 = fmaf(pp, qp, a0);
            if (has2) {
                pout[p2] = pp2;
                q32[p2] = qp2;
                a0 = fmaf(pp2, qp2, a0);
            }
        }
        float w1[1] = {a0};
        cl_reduce_f32<1>(C, w1);
        const float af = rho / w1[0];
        if (!(w1[0] > 0.0f) || !isfinite(af)) return false;
        float b0 = 0.0f, b1 = 0.0f;
        if constexpr (zline) {
            for (int p = lo + (int)threadIdx.x; p < hi; p += bd) {
                const float r2 = fmaf(-af, q32[p], r32[p]);
                d32[p] = fmaf(af, pout[p], d32[p]);
                r32[p] = r2;
                b0 = fmaf(r2, r2, b0);
            }
            unit_sync(C);   // the columns cross the CTAs' cell ranges
            b1 = zline_solve32(C, g, K32, lt_inv, lt_c, lt_P, lt_Q, lt_rs, r32, z32, q32);   // q32 is free here
        } else
        for (int p = lo + (int)threadIdx.x; p < hi; p += 2 * bd) {
            const bool has2 = p + bd < hi;
            const int p2 = has2 ? p + bd : p;
            const float pa = pout[p], da = d32[p], qa = q32[p], ra = r32[p], ia = di32[p];
            const float pb = pout[p2], db = d32[p2], qb = q32[p2], rb = r32[p2], ib = di32[p2];
            const float ra2 = fmaf(-af, qa, ra), za2 = ia * ra2;
            d32[p] = fmaf(af, pa, da);
            r32[p] = ra2;
            z32[p] = za2;
            b0 = fmaf(ra2, ra2, b0);
            b1 = fmaf(ra2, za2, b1);
            if (has2) {
                const float rb2 = fmaf(-af, qb, rb), zb2 = ib * rb2;
                d32[p2] = fmaf(af, pb, db);
                r32[p2] = rb2;
                z32[p2] = zb2;
                b0 = fmaf(rb2, rb2, b0);
                b1 = fmaf(rb2, zb2, b1);
            }
        }
        float w2[2] = {b0, b1};
        cl_reduce_f32<2>(C, w2);
        its++;
        pi ^= 1;
        if (!isfinite(w2[0]) || !isfinite(w2[1])) return false;
        if (sqrtf(w2[0]) <= stop || its >= max_it) return true;
        beta = w2[1] / rho;
        rho = w2[1];
    }
}

__device__ __forceinline__ double t_tol_d(double t) { return 1e-9 * (fabs(t) > 1.0 ? fabs(t) : 1.0); }

}  // namespace

template <int PREC, int THREADS>
__global__ void __launch_bounds__(THREADS, 512 / THREADS)
k_ensemble(EnsDesc *__restrict__ D, int n_inst, EnsBuffers B, EnsParams P, const double *t_end_p, unsigned int *queue,
           const int *__restrict__ sched)
{
    const double t_end = *t_end_p;
    static_assert(THREADS <= 32 * RB_WARPS, "partial slots");
    __shared__ double red[2][RB_SLOTS][RB_WARPS];
    __shared__ double bc[2][RB_SLOTS];
    __shared__ float redf[2][RB_SLOTS][RB_WARPS];
    __shared__ int s_inst;
    __shared__ double part[RB_PART * THREADS];
    ClusterCtx C{cg::this_cluster(), 0, 1, false, red, bc, redf, part, 0};
    const int cl_rank = (int)C.cl.block_rank(), cl_size = (int)C.cl.num_blocks();
    C.rank = cl_rank;
    C.ncta = cl_size;

    for (;;) {
        int inst;
        if (!C.solo) {
            if (C.rank == 0 && threadIdx.x == 0) {
                const unsigned int k = atomicAdd(queue, 1u);
                s_inst = k < (unsigned int)n_inst ? sched[k] : -1;
            }
            C.cl.sync();
            const int e = *C.cl.map_shared_rank(&s_inst, 0);
            C.cl.sync();   // no remote shared access after this point when going solo
            if (e < 0) break;
            inst = e & ENS_SCHED_INDEX;
            if (cl_size > 1 && !(e & ENS_SCHED_WIDE)) {
                // the queue has reached the instances that run on single
                // CTAs: rank 0 runs this one alone, the others pop their own
                C.solo = true;
                C.rank = 0;
                C.ncta = 1;
                if (cl_rank != 0) continue;
            }
        } else {
            if (threadIdx.x == 0) {
                const unsigned int k = atomicAdd(queue, 1u);
                s_inst = k < (unsigned int)n_inst ? (sched[k] & ENS_SCHED_INDEX) : -1;
            }
            __syncthreads();
            inst = s_inst;
            __syncthreads();
            if (inst < 0) break;
        }
        unsigned long long t_start = 0;
        if (C.rank == 0 && threadIdx.x == 0) asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_start));

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
        float *LTi = P.zline ? B.lt_inv + off : nullptr, *LTc = P.zline ? B.lt_c + off : nullptr;
        float *LTP = P.zline ? B.lt_P + off : nullptr, *LTQ = P.zline ? B.lt_Q + off : nullptr;
        float4 *LTR = P.zline ? B.lt_rs + off : nullptr;
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
                closure(*soil, Ks[p], hp, g.tab, g.closure64, th, k, c);
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
        auto sqrt3 = [](const double (&t)[4], double *o) {
            o[0] = sqrt(t[0]);
            o[1] = sqrt(t[1]);
            o[2] = sqrt(t[2]);
        };

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
                unit_sync(C);
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
                                            KB[kin], Can, nullptr, P.eps_chord, V_dt, cs);
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
                    double sq[3];   // square roots of the first three sums
                    cl_reduce<OpSum, 4, 3>(C, v, sq, sqrt3);
                    int cg_it = 0;
                    bool lin_ok = true;
                    if (PREC == 0) {
                        // ---- FP64 Jacobi-PCG
                        double rho = v[0];
                        const double stop = P.tol_cg * sq[2];
                        bool done = !(isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]));
                        if (done) lin_ok = false;
                        else done = sq[1] <= stop;
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
                            double alpha;
                            cl_reduce<OpSum, 1, 1>(C, w1, &alpha,
                                                   [&](const double (&t)[1], double *o) { o[0] = rho / t[0]; });
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
                            double fb[2];   // stop test passed (1 or 0), beta
                            cl_reduce<OpSum, 2, 2>(C, w2, fb, [&](const double (&t)[2], double *o) {
                                o[0] = sqrt(t[0]) <= stop ? 1.0 : 0.0;
                                o[1] = t[1] / rho;
                            });
                            cg_it++;
                            pi ^= 1;
                            if (!isfinite(w2[0]) || !isfinite(w2[1])) { lin_ok = false; break; }
                            if (fb[0] != 0.0) break;
                            if (cg_it >= P.cg_max_it) { lin_ok = false; break; }
                            beta = fb[1];
                            rho = w2[1];
                        }
                    } else {
                        // ---- FP32 inner PCG inside FP64 defect correction
                        // (the assembly's reduction barrier published K32, cb32)
                        if (P.zline) zline_factor32(C, geo32(g), K32, cb32, LTi, LTc, LTP, LTQ, LTR);
                        int outer = 1;
                        for (;;) {
                            const bool finite = isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]) && isfinite(v[3]);
                            if (!finite) { lin_ok = false; break; }
                            if (sq[0] <= P.tol_cg * sq[1]) break;
                            if (outer >= P.outer_max_it) { lin_ok = false; break; }
                            // inner solve A d = r32 from d = 0, FP32 throughout
                            int inner_it = 0;
                            if (v[2] > 0.0) {
                                const float stop = (float)(P.tol_inner * sq[2]);
                                lin_ok = P.zline
                                             ? inner_pcg32<true>(C, geo32(g), (int)lo, (int)hi, K32, cb32, di32, r32,
                                                                 z32, P32[0], P32[1], q32, d32, LTi, LTc, LTP, LTQ,
                                                                 LTR, 0.0f, stop, P.inner_max_it, inner_it)
                                             : inner_pcg32<false>(C, geo32(g), (int)lo, (int)hi, K32, cb32, di32, r32,
                                                                  z32, P32[0], P32[1], q32, d32, nullptr, nullptr,
                                                                  nullptr, nullptr, nullptr, (float)v[3], stop,
                                                                  P.inner_max_it, inner_it);
                            }
                            cg_it += inner_it;
                            if (!lin_ok) break;
                            for (long long p = lo + threadIdx.x; p < hi; p += blockDim.x) x[p] += (double)d32[p];
                            unit_sync(C);
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
                            cl_reduce<OpSum, 4, 3>(C, v, sq, sqrt3);
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
                unit_sync(C);
            }
            if (!accepted) break;
        }
        unit_sync(C);
        if (C.rank == 0 && threadIdx.x == 0) {
            unsigned long long t_stop;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_stop));
            d.busy_ns += (long long)(t_stop - t_start);
            d.ctas = C.ncta;
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
        unit_sync(C);
    }
}

template <int PREC>
static void *ensemble_kernel(int threads)
{
    if (threads == 128) return (void *)k_ensemble<PREC, 128>;
    if (threads == 256) return (void *)k_ensemble<PREC, 256>;
    if (threads == 512) return (void *)k_ensemble<PREC, 512>;
    return nullptr;
}

static void *ensemble_kernel(int threads, int precision)
{
    return precision == 0 ? ensemble_kernel<0>(threads) : ensemble_kernel<1>(threads);
}

cudaError_t launch_ensemble(cudaStream_t s, int cluster, int threads, int nclusters, int precision, EnsDesc *D,
                            int n_inst, const EnsBuffers &B, const EnsParams &P, const double *t_end,
                            unsigned int *queue, const int *sched)
{
    void *fn = ensemble_kernel(threads, precision);
    if (!fn) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(cluster * nclusters), 1, 1);
    cfg.blockDim = dim3((unsigned)threads, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void *args[] = {&D, &n_inst, const_cast<EnsBuffers *>(&B), const_cast<EnsParams *>(&P), &t_end, &queue, &sched};
    return cudaLaunchKernelExC(&cfg, fn, args);
}

int ensemble_max_clusters(int cluster, int threads, int precision)
{
    void *fn = ensemble_kernel(threads, precision);
    if (!fn) return 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)cluster, 1, 1);
    cfg.blockDim = dim3((unsigned)threads, 1, 1);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

}  // namespace rf
