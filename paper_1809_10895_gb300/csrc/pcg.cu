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

#include <algorithm>

#include "cell_ops.cuh"
#include "rf_internal.cuh"
#include "rf_reduce.cuh"
#include "tma.cuh"

namespace rf {

#define GRID_STRIDE_LOOP(p)                                                                 \
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < g.N;           \
         p += (long long)gridDim.x * blockDim.x)

// Tiled sweeps for the stencil kernels.  A block owns a TX x TY column tile
// and a range of z planes and walks up through them: the x/y neighbours of a
// plane come from shared memory (the plane plus a one-cell halo, double
// buffered so each plane needs one barrier), the z neighbours from registers
// (the planes below and above), and the plane above is loaded while the
// current one is in use.  Blocks loop over (tile, z-range) items; the grid
// never exceeds the reduction's block count.
constexpr int TX = 32, TY = RED_THREADS / 32;
constexpr int HALO = 2 * TY + 2 * TX;   // x- and y-halo cells of a plane (no corners)

struct Tiles {
    int ntx, nty, zc;       // tiles along x, y; planes per item
    int tx;                 // tile width in x
    long long items;
};

static Tiles make_tiles(const Grid &g, int nblk)
{
    if (g.cap > nblk) nblk = g.cap;
    Tiles t;
    t.tx = TX;
    t.ntx = (g.nx + TX - 1) / TX;
    t.nty = (g.ny + TY - 1) / TY;
    const long long tiles = (long long)t.ntx * t.nty;
    // split z so that the items fill the grid in one wave when the tiles alone
    // do not (every block then walks the same number of planes)
    const long long want_chunks = nblk / tiles;
    const int chunks = (int)std::min<long long>(std::max<long long>(want_chunks, 1), g.nz);
    t.zc = (g.nz + chunks - 1) / chunks;
    t.items = tiles * ((g.nz + t.zc - 1) / t.zc);
    return t;
}

// Tiles with the z split that minimises (waves of `resident` blocks) x
// (planes per item + the two extra planes an item reads); at most `cap` items
// per wave are launched.
static Tiles make_tiles_balanced(const Grid &g, int resident, int tile_x)
{
    Tiles t;
    t.tx = tile_x;
    t.ntx = (g.nx + tile_x - 1) / tile_x;
    t.nty = (g.ny + TY - 1) / TY;
    const long long tiles = (long long)t.ntx * t.nty;
    long long best = -1;
    int best_zc = g.nz;
    for (int ch = 1; ch <= g.nz; ch++) {
        const int zc = (g.nz + ch - 1) / ch;
        const long long items = tiles * ((g.nz + zc - 1) / zc);
        const long long waves = (items + resident - 1) / resident;
        const long long cost = waves * (zc + 2);
        if (best < 0 || cost < best) {
            best = cost;
            best_zc = zc;
        }
    }
    t.zc = best_zc;
    t.items = tiles * ((g.nz + t.zc - 1) / t.zc);
    return t;
}

static int tile_blocks(const Tiles &t, const Grid &g, int nblk)
{
    return (int)std::min<long long>(t.items, g.cap > nblk ? g.cap : nblk);
}

struct TileItem {
    int i0, j0, k0, k1;
};

__device__ __forceinline__ TileItem tile_item(const Grid &g, const Tiles &t, long long item)
{
    const long long per_plane = (long long)t.ntx * t.nty;
    const int chunk = (int)(item / per_plane);
    const long long r = item - chunk * per_plane;
    TileItem it;
    it.j0 = (int)(r / t.ntx) * TY;
    it.i0 = (int)(r % t.ntx) * t.tx;
    it.k0 = chunk * t.zc;
    it.k1 = min(g.nz, it.k0 + t.zc);
    return it;
}

// Halo cell h (0 <= h < HALO) of a tile, as offsets (hx, hy) from (i0, j0):
// -x column, +x column, -y row, +y row.
__device__ __forceinline__ void halo_cell(int h, int &hx, int &hy)
{
    if (h < TY) { hx = -1; hy = h; }
    else if (h < 2 * TY) { hx = TX; hy = h - TY; }
    else if (h < 2 * TY + TX) { hx = h - 2 * TY; hy = -1; }
    else { hx = h - 2 * TY - TX; hy = TY; }
}

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

// One plane of the FP64 operator's face coefficients around a tile, staged by
// the tiled FP64 kernels: Ty of rows j0-1 .. j0+TY-1 and Tx of the -x halo
// column (the +x / +y / +z coefficients of a cell are its own).
struct Faces64 {
    double ty[2][TY + 1][TX];
    double tx[2][TY];
};

// Stage the values v (own cell pc, halo via val) and face coefficients of
// plane k; returns the cell's own coefficients (0 on inactive cells).
template <class Val>
__device__ __forceinline__ void stage64(const Grid &g, const TileItem &it, int k, int buf, int tx, int ty, int hx,
                                        int hy, bool inside, long long c, const uint8_t *__restrict__ flags,
                                        const double *__restrict__ Tx, const double *__restrict__ Ty,
                                        const double *__restrict__ Tz, const double *__restrict__ diag, double pc,
                                        Val val, double (&sP)[2][TY + 2][TX + 2], Faces64 &sF, bool &act,
                                        double &dg, double &txp, double &typ, double &tzp)
{
    sP[buf][ty + 1][tx + 1] = pc;
    act = inside && (flags[c] & FLAG_ACTIVE);
    dg = txp = typ = tzp = 0.0;
    if (act) {
        dg = diag[c];
        txp = Tx[c];
        typ = Ty[c];
        tzp = Tz[c];
    }
    sF.ty[buf][ty + 1][tx] = typ;
    if (threadIdx.x < HALO) {
        const int ii = it.i0 + hx, jj = it.j0 + hy;
        const bool in = ii >= 0 && ii < g.nx && jj >= 0 && jj < g.ny;
        const long long hc = ii + (long long)g.nx * jj + g.sxy * k;
        const bool hact = in && (flags[hc] & FLAG_ACTIVE);
        sP[buf][hy + 1][hx + 1] = hact ? val(hc) : 0.0;
        if (hx == -1) sF.tx[buf][hy] = hact ? Tx[hc] : 0.0;
        if (hy == -1) sF.ty[buf][0][hx] = hact ? Ty[hc] : 0.0;
    }
}

// (A v)_P = diag_P v_P - sum_f T_f v_N with faces in the order -x +x -y +y -z +z.
__device__ __forceinline__ double apply64_tile(const Grid &g, int i, int j, int k, int tx, int ty, int buf,
                                               const double (&sP)[2][TY + 2][TX + 2], const Faces64 &sF,
                                               double txm_lane, double dg, double txp, double typ, double tzm,
                                               double tzp, double vm, double vc, double vn)
{
    const double txm = tx > 0 ? txm_lane : sF.tx[buf][ty];
    double acc = dg * vc;
    if (i > 0) acc -= txm * sP[buf][ty + 1][tx];
    if (i < g.nx - 1) acc -= txp * sP[buf][ty + 1][tx + 2];
    if (j > 0) acc -= sF.ty[buf][ty][tx] * sP[buf][ty][tx + 1];
    if (j < g.ny - 1) acc -= typ * sP[buf][ty + 2][tx + 1];
    if (k > 0) acc -= tzm * vm;
    if (k < g.nz - 1) acc -= tzp * vn;
    return acc;
}

__global__ void __launch_bounds__(RED_THREADS)
k_cg64_spmv(Grid g, Tiles tw, const uint8_t *__restrict__ flags, const double *__restrict__ z,
            const double *__restrict__ p_in, double *__restrict__ p_out, double *__restrict__ q,
            const double *__restrict__ Tx, const double *__restrict__ Ty, const double *__restrict__ Tz,
            const double *__restrict__ diag, double *partials, unsigned int *ticket, CgScal *sc)
{
    count_launch(g, KK_CG64_SPMV);
    if (sc->done) return;
    count_work(g, KK_CG64_SPMV);
    const double beta = sc->beta;
    const bool first = sc->iter == 0;
    auto val = [&](long long c) { return first ? z[c] : fma(beta, p_in[c], z[c]); };
    // p = z + beta p_old on active cells of the grid, 0 elsewhere
    auto pval = [&](int i, int j, int k) -> double {
        if (i >= g.nx || j >= g.ny || k < 0 || k >= g.nz) return 0.0;
        const long long c = i + (long long)g.nx * j + g.sxy * k;
        return (flags[c] & FLAG_ACTIVE) ? val(c) : 0.0;
    };
    __shared__ double sP[2][TY + 2][TX + 2];
    __shared__ Faces64 sF;
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    int hx = 0, hy = 0;
    if (threadIdx.x < HALO) halo_cell(threadIdx.x, hx, hy);
    double v[1] = {0.0};
    for (long long item = blockIdx.x; item < tw.items; item += gridDim.x) {
        const TileItem it = tile_item(g, tw, item);
        const int i = it.i0 + tx, j = it.j0 + ty;
        const bool inside = i < g.nx && j < g.ny;
        double pm = pval(i, j, it.k0 - 1), pc = pval(i, j, it.k0);
        double tzm = 0.0;
        if (inside && it.k0 > 0) {
            const long long cm = i + (long long)g.nx * j + g.sxy * (it.k0 - 1);
            tzm = (flags[cm] & FLAG_ACTIVE) ? Tz[cm] : 0.0;
        }
        // the plane's coefficients and halo, loaded a plane ahead so that
        // their round trip overlaps the previous plane's work (the kernel is
        // latency-bound: few FP64 instructions a cell, one barrier a plane)
        struct Pl {
            bool act, hact;
            double dg, txp, typ, tzp, hp, htx, hty;
        };
        auto load = [&](int k, long long c) {
            Pl l;
            l.act = inside && (flags[c] & FLAG_ACTIVE);
            l.dg = l.txp = l.typ = l.tzp = 0.0;
            if (l.act) {
                l.dg = diag[c];
                l.txp = Tx[c];
                l.typ = Ty[c];
                l.tzp = Tz[c];
            }
            l.hact = false;
            l.hp = l.htx = l.hty = 0.0;
            if (threadIdx.x < HALO) {
                const int ii = it.i0 + hx, jj = it.j0 + hy;
                const bool in = ii >= 0 && ii < g.nx && jj >= 0 && jj < g.ny;
                const long long hc = ii + (long long)g.nx * jj + g.sxy * k;
                l.hact = in && (flags[hc] & FLAG_ACTIVE);
                if (l.hact) {
                    l.hp = val(hc);
                    if (hx == -1) l.htx = Tx[hc];
                    if (hy == -1) l.hty = Ty[hc];
                }
            }
            return l;
        };
        Pl nxt = load(it.k0, i + (long long)g.nx * j + g.sxy * it.k0);
        for (int k = it.k0; k < it.k1; k++) {
            const int buf = k & 1;
            const long long c = i + (long long)g.nx * j + g.sxy * k;
            const Pl cur = nxt;
            if (k + 1 < it.k1) nxt = load(k + 1, c + g.sxy);
            sP[buf][ty + 1][tx + 1] = pc;
            sF.ty[buf][ty + 1][tx] = cur.typ;
            if (threadIdx.x < HALO) {
                sP[buf][hy + 1][hx + 1] = cur.hp;
                if (hx == -1) sF.tx[buf][hy] = cur.htx;
                if (hy == -1) sF.ty[buf][0][hx] = cur.hty;
            }
            const bool act = cur.act;
            const double dg = cur.dg, txp = cur.txp, typ = cur.typ, tzp = cur.tzp;
            const double pn = pval(i, j, k + 1);
            const double txm_lane = __shfl_up_sync(0xffffffffu, txp, 1);
            __syncthreads();
            if (act) {
                const double acc = apply64_tile(g, i, j, k, tx, ty, buf, sP, sF, txm_lane, dg, txp, typ, tzm, tzp,
                                                pm, pc, pn);
                p_out[c] = pc;
                q[c] = acc;
                v[0] += pc * acc;
            } else if (inside) {
                p_out[c] = 0.0;
                q[c] = 0.0;
            }
            tzm = tzp;
            pm = pc;
            pc = pn;
        }
        __syncthreads();
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
// d0 = 0 (so r32 = r, z32 = D^-1 r32).  The residual is formed in FP64; its
// norms (a stopping test and CG seeds) are summed from the FP32 residual in
// FP32 within a block, in FP64 across blocks.  Counts outer iterations and
// fails the solve after outer_max_it residuals without convergence.
__global__ void __launch_bounds__(RED_THREADS)
k_resid64(Grid g, Tiles tw, const uint8_t *__restrict__ flags, const double *__restrict__ x,
          const double *__restrict__ b, const double *__restrict__ Tx, const double *__restrict__ Ty,
          const double *__restrict__ Tz, const double *__restrict__ diag, const float *__restrict__ dinv32,
          float *__restrict__ r32, float *__restrict__ z32, float *__restrict__ d32, double tol, double tol_inner,
          int inner_max_it, int outer_max_it, double *partials, unsigned int *ticket, CgScal *outer, CgScal *inner,
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
    auto val = [&](long long c) { return x[c]; };
    auto xval = [&](int i, int j, int k) -> double {
        if (i >= g.nx || j >= g.ny || k < 0 || k >= g.nz) return 0.0;
        const long long c = i + (long long)g.nx * j + g.sxy * k;
        return (flags[c] & FLAG_ACTIVE) ? x[c] : 0.0;
    };
    __shared__ double sP[2][TY + 2][TX + 2];
    __shared__ Faces64 sF;
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    int hx = 0, hy = 0;
    if (threadIdx.x < HALO) halo_cell(threadIdx.x, hx, hy);
    float a_rr = 0.0f, a_bb = 0.0f, a_rz = 0.0f;   // r32.r32, b.b, r32.z32
    for (long long item = blockIdx.x; item < tw.items; item += gridDim.x) {
        const TileItem it = tile_item(g, tw, item);
        const int i = it.i0 + tx, j = it.j0 + ty;
        const bool inside = i < g.nx && j < g.ny;
        double xm = xval(i, j, it.k0 - 1), xc = xval(i, j, it.k0);
        double tzm = 0.0;
        if (inside && it.k0 > 0) {
            const long long cm = i + (long long)g.nx * j + g.sxy * (it.k0 - 1);
            tzm = (flags[cm] & FLAG_ACTIVE) ? Tz[cm] : 0.0;
        }
        for (int k = it.k0; k < it.k1; k++) {
            const int buf = k & 1;
            const long long c = i + (long long)g.nx * j + g.sxy * k;
            bool act;
            double dg, txp, typ, tzp;
            stage64(g, it, k, buf, tx, ty, hx, hy, inside, c, flags, Tx, Ty, Tz, diag, xc, val, sP, sF, act, dg,
                    txp, typ, tzp);
            const double xn = xval(i, j, k + 1);
            const double bp = act ? b[c] : 0.0;
            const float di = act ? dinv32[c] : 0.0f;
            const double txm_lane = __shfl_up_sync(0xffffffffu, txp, 1);
            __syncthreads();
            if (act) {
                const double rp = bp - apply64_tile(g, i, j, k, tx, ty, buf, sP, sF, txm_lane, dg, txp, typ, tzm,
                                                    tzp, xm, xc, xn);
                const float rf = (float)rp;
                const float zf = di * rf;
                const float bf = (float)bp;
                r32[c] = rf;
                z32[c] = zf;
                d32[c] = 0.0f;
                a_rr = fmaf(rf, rf, a_rr);
                a_bb = fmaf(bf, bf, a_bb);
                a_rz = fmaf(rf, zf, a_rz);
            } else if (inside) {
                r32[c] = 0.0f;
                z32[c] = 0.0f;
                d32[c] = 0.0f;
            }
            tzm = tzp;
            xm = xc;
            xc = xn;
        }
        __syncthreads();
    }
    float vf[3] = {a_rr, a_bb, a_rz};
    double w[3];
    if (grid_reduce_f32<3>(vf, w, partials, ticket) && threadIdx.x == 0) {
        outer->iter += 1;
        const double v[4] = {w[0], w[1], w[0], w[2]};
        outer_residual_scalars(outer, inner, v, tol, tol_inner, inner_max_it, outer_max_it, cond_outer, cond_inner);
    }
}

__global__ void __launch_bounds__(RED_THREADS)
k_cg32_spmv(Grid g, Tiles tw, const float *__restrict__ z, const float *__restrict__ p_in, float *__restrict__ p_out,
            float *__restrict__ q, const float *__restrict__ K32, const float *__restrict__ cb32, double *partials,
            unsigned int *ticket, CgScal *sc)
{
    count_launch(g, KK_CG32_SPMV);
    if (sc->done) return;
    count_work(g, KK_CG32_SPMV);
    const float beta = (float)sc->beta;
    const bool first = sc->iter == 0;
    // (p, K) of a cell: p = z + beta p_old, K < 0 marks inactive / outside cells
    auto load = [&](int i, int j, int k, float &pv, float &kv) {
        pv = 0.0f;
        kv = -1.0f;
        if (i < 0 || i >= g.nx || j < 0 || j >= g.ny || k < 0 || k >= g.nz) return;
        const long long c = i + (long long)g.nx * j + g.sxy * k;
        kv = K32[c];
        if (kv >= 0.0f) pv = first ? z[c] : fmaf(beta, p_in[c], z[c]);
    };
    __shared__ float sP[2][TY + 2][TX + 2], sK[2][TY + 2][TX + 2];
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    int hx = 0, hy = 0;
    if (threadIdx.x < HALO) halo_cell(threadIdx.x, hx, hy);
    const float wx = g.w32[0] * 0.5f, wy = g.w32[1] * 0.5f, wz = g.w32[2] * 0.5f;
    float acc = 0.0f;
    for (long long item = blockIdx.x; item < tw.items; item += gridDim.x) {
        const TileItem it = tile_item(g, tw, item);
        const int i = it.i0 + tx, j = it.j0 + ty;
        const bool inside = i < g.nx && j < g.ny;
        float pm, km, pc, kc;
        load(i, j, it.k0 - 1, pm, km);
        load(i, j, it.k0, pc, kc);
        for (int k = it.k0; k < it.k1; k++) {
            const int buf = k & 1;
            const long long c = i + (long long)g.nx * j + g.sxy * k;
            sP[buf][ty + 1][tx + 1] = pc;
            sK[buf][ty + 1][tx + 1] = kc;
            if (threadIdx.x < HALO) {
                float hp, hk;
                load(it.i0 + hx, it.j0 + hy, k, hp, hk);
                sP[buf][hy + 1][hx + 1] = hp;
                sK[buf][hy + 1][hx + 1] = hk;
            }
            float pn, kn;
            load(i, j, k + 1, pn, kn);
            const float cb = (inside && kc >= 0.0f) ? cb32[c] : 0.0f;
            __syncthreads();
            if (inside && kc >= 0.0f) {
                // (A p)_P = cb_P p_P + sum_f w_f (K_P + K_N)/2 (p_P - p_N), faces -x +x -y +y -z +z
                float qp = cb * pc;
                auto face = [&](float KN, float vN, float w) {
                    if (KN >= 0.0f) qp = fmaf(w * (kc + KN), pc - vN, qp);
                };
                face(sK[buf][ty + 1][tx], sP[buf][ty + 1][tx], wx);
                face(sK[buf][ty + 1][tx + 2], sP[buf][ty + 1][tx + 2], wx);
                face(sK[buf][ty][tx + 1], sP[buf][ty][tx + 1], wy);
                face(sK[buf][ty + 2][tx + 1], sP[buf][ty + 2][tx + 1], wy);
                face(km, pm, wz);
                face(kn, pn, wz);
                p_out[c] = pc;
                q[c] = qp;
                acc = fmaf(pc, qp, acc);
            } else if (inside) {
                p_out[c] = 0.0f;
                q[c] = 0.0f;
            }
            pm = pc;
            km = kc;
            pc = pn;
            kc = kn;
        }
        __syncthreads();
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

// The FP32 stencil step with planes staged by TMA.  Per plane the block
// copies three 136 x 10 boxes (z, p_old, K) around its 128 x 8 tile and the
// tile's own 128 x 8 cb into shared memory with bulk tensor copies; each
// thread owns four x-adjacent cells (one float4), so the per-plane work of
// a thread -- poll, barrier, addressing -- is spread over four cells.  Each
// face term w (K_P + K_N)(p_P - p_N) is formed once: a face between two of a
// thread's cells serves both (with opposite signs), and the face between
// planes k and k + 1 is formed at plane k and carried in registers into
// plane k + 1.  A plane therefore needs only itself and the
// plane above, so the ring of stages holds planes k and k + 1 and keeps the
// next TMA_STAGES - 2 in flight.  Warp 0 alone polls the copy's mbarrier
// (bounded); the others meet it at the one barrier per plane and then
// confirm the completed phase once.  When a plane arrives each thread forms
// p = z + beta p_old (in place of z) for its own cells and at most one halo
// quad or cell.  A
// wait that runs out sets *fault, ends the solve and drains the copies in
// flight.
#ifndef RF_TMA_STAGES
#define RF_TMA_STAGES 4
#endif
constexpr int TMA_WAIT_TRIES = 1 << 20;   // about a second of suspending polls

// TMA_STAGES = planes k, k+1 resident plus TMA_STAGES - 2 in flight.
// Two blocks per SM: 4 stages of 3 x 5504 + 4096 bytes (cb is staged for the
// tile's own cells only), 82.9 KB a block.
template <int TMA_STAGES>
__global__ void __launch_bounds__(RED_THREADS, 2)
k_cg32_spmv_tma(Grid g, Tiles tw, const __grid_constant__ TmaMaps32 maps, int pin_sel, float *__restrict__ p_out,
                float *__restrict__ q, double *partials, unsigned int *ticket, CgScal *sc, int *fault)
{
    static_assert(TMA_STAGES >= 3 && TMA_STAGES <= 8, "the ring needs planes k, k+1 plus one in flight");
    count_launch(g, KK_CG32_SPMV);
    if (sc->done) return;
    count_work(g, KK_CG32_SPMV);
    const float beta = (float)sc->beta;
    const bool first = sc->iter == 0;
    constexpr int SLOT = TMA_SLOT_BYTES / 4;
    constexpr int OWN = TMA_OWN_BYTES / 4;
    __shared__ __align__(128) float sbuf[TMA_STAGES][3][SLOT];   // z (then p), p_old, K around the tile
    __shared__ __align__(128) float cbuf[TMA_STAGES][OWN];       // cb of the tile's own cells
    __shared__ __align__(8) uint64_t bar[TMA_STAGES];
    __shared__ int s_timeout;
    const CUtensorMap *mp = pin_sel ? &maps.p1 : &maps.p0;
    if (threadIdx.x == 0) {
        for (int st = 0; st < TMA_STAGES; st++) mbar_init(&bar[st], 1);
        mbar_init_fence();
        s_timeout = 0;
    }
    __syncthreads();
    const uint32_t tx_bytes = (first ? 2 : 3) * TMA_BOX_BYTES + TMA_OWN_BYTES;
    const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
    const bool poller = threadIdx.x < 32;
    const int idx = (ty + 1) * TMA_BX + 4 * tx + TMA_X0;   // a multiple of 4: the quad is one float4
    const int oidx = ty * TMA_TX + 4 * tx;                 // the quad in the own-cell box
    // halo this thread converts: threads 0-63 a quad of the rows below and
    // above the tile, threads 64-79 one cell left or right of it
    int hidx4 = -1, hidx = -1;
    if (threadIdx.x < 64) {
        const int hy = threadIdx.x < 32 ? -1 : TY;
        hidx4 = (hy + 1) * TMA_BX + 4 * (threadIdx.x % 32) + TMA_X0;
    } else if (threadIdx.x < 64 + 2 * TY) {
        const int h = threadIdx.x - 64;
        const int hx = h < TY ? -1 : TMA_TX, hy = h % TY;
        hidx = (hy + 1) * TMA_BX + hx + TMA_X0;
    }
    const float wx = g.w32[0] * 0.5f, wy = g.w32[1] * 0.5f, wz = g.w32[2] * 0.5f;
    uint32_t phase = 0, pending = 0;   // per stage: parity of its next completion; copy in flight
    float acc = 0.0f;
    auto ld4 = [](const float *a, int e) { return *reinterpret_cast<const float4 *>(a + e); };
    auto fma4 = [](float b, float4 o, float4 z) {
        return make_float4(fmaf(b, o.x, z.x), fmaf(b, o.y, z.y), fmaf(b, o.z, z.z), fmaf(b, o.w, z.w));
    };
    // face term of cell P towards cell N.  Inactive cells carry K = NaN and
    // the K boxes read NaN outside the grid (their p reads 0), so
    // max(w (K_P + K_N), 0) is the face coefficient where both cells are
    // active and 0 where either is not (IEEE max returns the non-NaN operand)
    auto face = [](float kP, float pP, float kN, float pN, float w) -> float {
        return fmaxf(w * (kP + kN), 0.0f) * (pP - pN);
    };
    for (long long item = blockIdx.x; item < tw.items && !s_timeout; item += gridDim.x) {
        const TileItem it = tile_item(g, tw, item);
        const int i = it.i0 + 4 * tx, j = it.j0 + ty;      // first cell of the quad (nx is a multiple of 4)
        const bool inside = i < g.nx && j < g.ny;
        // plane kk = it.k0 - 1 + L goes to stage L % TMA_STAGES (stage
        // indices advance incrementally); planes outside the grid are neither
        // copied nor read
        auto present = [&](int kk) { return kk >= 0 && kk < g.nz && kk <= it.k1; };
        auto issue = [&](int kk, int st) {   // every thread tracks pending; thread 0 copies
            if (!present(kk)) return;
            pending |= 1u << st;
            if (threadIdx.x == 0) {
                mbar_expect_tx(&bar[st], tx_bytes);
                const int x = it.i0 - TMA_X0, y = it.j0 - 1;
                tma_load_3d(sbuf[st][0], &maps.z, &bar[st], x, y, kk);
                if (!first) tma_load_3d(sbuf[st][1], mp, &bar[st], x, y, kk);
                tma_load_3d(sbuf[st][2], &maps.K, &bar[st], x, y, kk);
                tma_load_3d(cbuf[st], &maps.cb, &bar[st], it.i0, it.j0, kk);
            }
        };
        // warp 0: poll stage st (bounded); false when the wait ran out.  The
        // grid's wait_tries (a test limit) replaces the default poll count;
        // negative: a single non-blocking test
        auto poll = [&](int st) -> bool {
            if (!poller || !(pending & (1u << st))) return true;
            if (g.wait_tries < 0) return mbar_test_wait(&bar[st], (phase >> st) & 1u);
            return mbar_wait_bounded(&bar[st], (phase >> st) & 1u, g.wait_tries > 0 ? g.wait_tries : TMA_WAIT_TRIES);
        };
        // after the barrier that follows a successful poll: confirm the phase
        // (completes at once) and form p for the own cells and halo cell of plane kk
        auto take = [&](int kk, int st) {
            if (pending & (1u << st)) {
                mbar_try_wait(&bar[st], (phase >> st) & 1u);
                phase ^= 1u << st;
                pending &= ~(1u << st);
            }
            if (!first && present(kk)) {
                float *pz = sbuf[st][0];
                const float *po = sbuf[st][1];
                *reinterpret_cast<float4 *>(pz + idx) = fma4(beta, ld4(po, idx), ld4(pz, idx));
                if (hidx4 >= 0) *reinterpret_cast<float4 *>(pz + hidx4) = fma4(beta, ld4(po, hidx4), ld4(pz, hidx4));
                if (hidx >= 0) pz[hidx] = fmaf(beta, po[hidx], pz[hidx]);
                fence_proxy_async_smem();   // the stage is refilled by tensor copies later
            }
        };
        auto next = [](int st) { return st + 1 == TMA_STAGES ? 0 : st + 1; };
        for (int L = 0; L < TMA_STAGES; L++) issue(it.k0 - 1 + L, L);
        if (!(poll(0) && poll(1))) s_timeout = 1;
        __syncthreads();
        if (s_timeout) break;
        take(it.k0 - 1, 0);
        take(it.k0, 1);
        // the bottom-face term of plane k0 (from plane k0 - 1, staged for
        // this only); later planes receive it from the plane below
        float4 carry = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (inside && it.k0 > 0) {
            const float4 kc = ld4(sbuf[1][2], idx), pc = ld4(sbuf[1][0], idx);
            const float4 kb = ld4(sbuf[0][2], idx), pb = ld4(sbuf[0][0], idx);
            carry = make_float4(face(kc.x, pc.x, kb.x, pb.x, wz), face(kc.y, pc.y, kb.y, pb.y, wz),
                                face(kc.z, pc.z, kb.z, pb.z, wz), face(kc.w, pc.w, kb.w, pb.w, wz));
        }
        // stages of planes k and k + 1, and the one plane k - 1 held (refilled with plane k + TMA_STAGES - 1)
        int s_c = 1, s_p = 2 % TMA_STAGES, s_i = 0;
        long long c = i + (long long)g.nx * j + g.sxy * it.k0;
        for (int k = it.k0; k < it.k1; k++, c += g.sxy) {
            if (!poll(s_p)) s_timeout = 1;
            __syncthreads();              // plane k+1 landed; plane k-1 is no longer read
            if (s_timeout) break;
            issue(k + TMA_STAGES - 1, s_i);
            take(k + 1, s_p);
            if (inside) {
                const float *P0 = sbuf[s_c][0], *K0 = sbuf[s_c][2];
                const float4 kc = ld4(K0, idx), pc = ld4(P0, idx), cb = ld4(cbuf[s_c], oidx);
                const float4 kym = ld4(K0, idx - TMA_BX), pym = ld4(P0, idx - TMA_BX);
                const float4 kyp = ld4(K0, idx + TMA_BX), pyp = ld4(P0, idx + TMA_BX);
                // (A p)_P = cb_P p_P + sum_f w_f (K_P + K_N)/2 (p_P - p_N); the
                // plane above the grid's top is not staged, so its faces are skipped
                const float t01 = face(kc.x, pc.x, kc.y, pc.y, wx);   // faces inside the quad
                const float t12 = face(kc.y, pc.y, kc.z, pc.z, wx);
                const float t23 = face(kc.z, pc.z, kc.w, pc.w, wx);
                float4 tz = make_float4(0.0f, 0.0f, 0.0f, 0.0f);       // top faces
                if (k < g.nz - 1) {
                    const float4 kzp = ld4(sbuf[s_p][2], idx), pzp = ld4(sbuf[s_p][0], idx);
                    tz = make_float4(face(kc.x, pc.x, kzp.x, pzp.x, wz), face(kc.y, pc.y, kzp.y, pzp.y, wz),
                                     face(kc.z, pc.z, kzp.z, pzp.z, wz), face(kc.w, pc.w, kzp.w, pzp.w, wz));
                }
                float q0 = fmaf(cb.x, pc.x, carry.x) + t01 + tz.x;
                float q1 = fmaf(cb.y, pc.y, carry.y) - t01 + t12 + tz.y;
                float q2 = fmaf(cb.z, pc.z, carry.z) - t12 + t23 + tz.z;
                float q3 = fmaf(cb.w, pc.w, carry.w) - t23 + tz.w;
                q0 += face(kc.x, pc.x, K0[idx - 1], P0[idx - 1], wx);
                q3 += face(kc.w, pc.w, K0[idx + 4], P0[idx + 4], wx);
                q0 += face(kc.x, pc.x, kym.x, pym.x, wy) + face(kc.x, pc.x, kyp.x, pyp.x, wy);
                q1 += face(kc.y, pc.y, kym.y, pym.y, wy) + face(kc.y, pc.y, kyp.y, pyp.y, wy);
                q2 += face(kc.z, pc.z, kym.z, pym.z, wy) + face(kc.z, pc.z, kyp.z, pyp.z, wy);
                q3 += face(kc.w, pc.w, kym.w, pym.w, wy) + face(kc.w, pc.w, kyp.w, pyp.w, wy);
                carry = make_float4(-tz.x, -tz.y, -tz.z, -tz.w);
                const bool a0 = kc.x >= 0.0f, a1 = kc.y >= 0.0f, a2 = kc.z >= 0.0f, a3 = kc.w >= 0.0f;
                const float4 po = make_float4(a0 ? pc.x : 0.0f, a1 ? pc.y : 0.0f, a2 ? pc.z : 0.0f, a3 ? pc.w : 0.0f);
                const float4 qo = make_float4(a0 ? q0 : 0.0f, a1 ? q1 : 0.0f, a2 ? q2 : 0.0f, a3 ? q3 : 0.0f);
                acc = fmaf(po.x, qo.x, fmaf(po.y, qo.y, fmaf(po.z, qo.z, fmaf(po.w, qo.w, acc))));
                *reinterpret_cast<float4 *>(p_out + c) = po;
                *reinterpret_cast<float4 *>(q + c) = qo;
            }
            s_c = s_p;
            s_p = next(s_p);
            s_i = next(s_i);
        }
        __syncthreads();                  // the item's planes are no longer read
    }
    if (s_timeout) {
        // drain the copies in flight (bounded), report, end the solve
        for (int st = 0; st < TMA_STAGES; st++)
            if (pending & (1u << st)) mbar_wait_bounded(&bar[st], (phase >> st) & 1u, TMA_WAIT_TRIES);
        if (threadIdx.x == 0) atomicExch(fault, 1);
    }
    float vf[1] = {acc};
    double v[1];
    if (grid_reduce_f32<1>(vf, v, partials, ticket) && threadIdx.x == 0) {
        sc->pq = v[0];
        const double a = sc->rho / v[0];
        if (!(v[0] > 0.0) || !isfinite(a) || __ldcg(fault)) {
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
    // one cell: inactive cells (dinv 0) keep x and r and hold z = 0 (as set
    // when the inner solve starts), so z is written without being read
    auto cell = [&](float di, float pv, float xv, float qv, float rv, float &xo, float &ro, float &zo) {
        const bool act = di != 0.0f;
        const float rp = fmaf(-alpha, qv, rv), zp = di * rp;
        xo = act ? fmaf(alpha, pv, xv) : xv;
        ro = act ? rp : rv;
        zo = act ? zp : 0.0f;
        if (act) {
            a0 = fmaf(rp, rp, a0);
            a1 = fmaf(rp, zp, a1);
        }
    };
    const long long N = g.N;
    const long long stride = (long long)gridDim.x * blockDim.x, t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool vec = ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(r) | reinterpret_cast<uintptr_t>(z) |
                       reinterpret_cast<uintptr_t>(pd) | reinterpret_cast<uintptr_t>(q) |
                       reinterpret_cast<uintptr_t>(dinv)) & 15u) == 0;
    long long done = 0;
    if (vec) {
        // four cells per thread and pass: 16-byte loads and stores
        const long long n4 = N / 4;
        for (long long v = t0; v < n4; v += stride) {
            const float4 di = reinterpret_cast<const float4 *>(dinv)[v], pv = reinterpret_cast<const float4 *>(pd)[v];
            const float4 xv = reinterpret_cast<const float4 *>(x)[v], qv = reinterpret_cast<const float4 *>(q)[v];
            const float4 rv = reinterpret_cast<const float4 *>(r)[v];
            float4 xo, ro, zo;
            cell(di.x, pv.x, xv.x, qv.x, rv.x, xo.x, ro.x, zo.x);
            cell(di.y, pv.y, xv.y, qv.y, rv.y, xo.y, ro.y, zo.y);
            cell(di.z, pv.z, xv.z, qv.z, rv.z, xo.z, ro.z, zo.z);
            cell(di.w, pv.w, xv.w, qv.w, rv.w, xo.w, ro.w, zo.w);
            reinterpret_cast<float4 *>(x)[v] = xo;
            reinterpret_cast<float4 *>(r)[v] = ro;
            reinterpret_cast<float4 *>(z)[v] = zo;
        }
        done = n4 * 4;
    }
    for (long long p = done + t0; p < N; p += stride) {
        float xo, ro, zo;
        cell(dinv[p], pd[p], x[p], q[p], r[p], xo, ro, zo);
        x[p] = xo;
        r[p] = ro;
        z[p] = zo;
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
    const Tiles tw = make_tiles(g, nblk);
    k_cg64_spmv<<<tile_blocks(tw, g, nblk), RED_THREADS, 0, s>>>(g, tw, flags, z, p_in, p_out, q, Tx, Ty, Tz, diag,
                                                              partials, ticket, sc);
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
    const Tiles tw = make_tiles(g, nblk);
    k_resid64<<<tile_blocks(tw, g, nblk), RED_THREADS, 0, s>>>(g, tw, flags, x, b, Tx, Ty, Tz, diag, dinv32, r32, z32,
                                                            d32, tol, tol_inner, inner_max_it, outer_max_it,
                                                            partials, ticket, outer, inner, cond_outer, cond_inner);
}

void launch_cg32_spmv(cudaStream_t s, int nblk, const Grid &g, const float *z, const float *p_in, float *p_out,
                      float *q, const float *K32, const float *cb32, double *partials, unsigned int *ticket,
                      CgScal *sc, const TmaMaps32 *tma, int *fault)
{
    const Tiles tw = make_tiles(g, nblk);
    if (tma && fault && z == tma->z_ptr && K32 == tma->K_ptr && cb32 == tma->cb_ptr &&
        (p_in == tma->p_ptr[0] || p_in == tma->p_ptr[1]) && TY == 8) {
        // one wave: as many items as blocks resident at this kernel's occupancy
        static int occ = 0;
        if (occ == 0 && (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cg32_spmv_tma<RF_TMA_STAGES>,
                                                                        RED_THREADS, 0) != cudaSuccess || occ < 1))
            occ = 1;
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int resident = std::max(1, std::min(occ * sms, std::max(g.cap, nblk)));
        const Tiles tt = make_tiles_balanced(g, resident, TMA_TX);
        k_cg32_spmv_tma<RF_TMA_STAGES><<<(int)std::min<long long>(tt.items, resident), RED_THREADS, 0, s>>>(
            g, tt, *tma, p_in == tma->p_ptr[1] ? 1 : 0, p_out, q, partials, ticket, sc, fault);
        return;
    }
    k_cg32_spmv<<<tile_blocks(tw, g, nblk), RED_THREADS, 0, s>>>(g, tw, z, p_in, p_out, q, K32, cb32, partials, ticket,
                                                              sc);
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

bool make_tma_maps32(int nx, int ny, int nz, const float *z, const float *p0, const float *p1, const float *K,
                     const float *cb, TmaMaps32 *out)
{
    if (nx % 4 != 0 || nx < 4) return false;
    for (const float *ptr : {z, p0, p1, K, cb})
        if (!ptr || (reinterpret_cast<uintptr_t>(ptr) & 15u) != 0) return false;
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
        return false;
    auto encode = reinterpret_cast<CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                                const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                                const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                                CUtensorMapL2promotion, CUtensorMapFloatOOBfill)>(fn);
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
    const cuuint64_t strides[2] = {(cuuint64_t)nx * 4, (cuuint64_t)nx * ny * 4};
    const cuuint32_t box[3] = {TMA_BX, TMA_BY, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    // boxes outside the grid read 0, except K, which reads NaN like an
    // inactive cell (the stencil's face coefficient max(w (K_P + K_N), 0)
    // then closes the faces at the grid's edge without a test)
    const cuuint32_t own_box[3] = {TMA_TX, TMA_OWN_BY, 1};
    auto one = [&](CUtensorMap *m, const float *ptr, bool nan_fill, const cuuint32_t *bx) {
        return encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(ptr), dims, strides, bx, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                      nan_fill ? CU_TENSOR_MAP_FLOAT_OOB_FILL_NAN_REQUEST_ZERO_FMA : CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
               CUDA_SUCCESS;
    };
    if (!(one(&out->z, z, false, box) && one(&out->p0, p0, false, box) && one(&out->p1, p1, false, box) &&
          one(&out->K, K, true, box) && one(&out->cb, cb, false, own_box)))
        return false;
    out->z_ptr = z;
    out->p_ptr[0] = p0;
    out->p_ptr[1] = p1;
    out->K_ptr = K;
    out->cb_ptr = cb;
    return true;
}

}  // namespace rf
