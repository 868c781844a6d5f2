// cell_ops.cuh -- per-cell device arithmetic shared by the single-domain
// kernels and the batched-ensemble kernel: closures (Eq. 2-4, Eq. A6), grid
// neighbours and the two stencil forms of the Picard operator.
#pragma once

#include <math.h>

#include "f64m.cuh"
#include "rf_internal.cuh"

namespace rf {

// van Genuchten / Mualem closures (Eq. 2-4), evaluated in double-float
// arithmetic (ff.cuh) with FP64 only at the input and the outputs.
// With u = -alpha h, L = log u, x = u^n = exp(n L), l1 = log(1 + x):
//   Se = (1 + x)^-m = exp(-m l1)                               (Eq. 2)
//   u^(n-1) = x / u (since m n = n - 1), so (x/(1+x))^m = (x/u) Se = ys
//   Se^(1/m) = 1/(1+x) = w, so 1 - Se^(1/m) = x/(1+x) and
//   K = Ks Se^(1/2) (1 - ys)^2                                   (Eq. 4)
//     with 1 - ys = -expm1(m log(1 - w)) when ys > 1/2 (dry soil, where
//     1 - ys would cancel)
//   C = (theta_s-theta_r) alpha n m u^(n-1) (1+x)^-(m+1)
//     = (theta_s-theta_r) alpha n m ys w                         (Eq. 3)
// (h < 0 only; closure() below handles h >= 0 and the other models.)
__device__ __forceinline__ void closure_vg_df(const DevSoil &s, double Ks, double h, const FFTables *__restrict__ tab,
                                              double &th, double &K, double &C)
{
    const double dth = s.theta_s - s.theta_r;
    const double ud = -s.alpha * h;
    if (ud < 1e-30) {                     // (-alpha h)^n underflows: the wet limit
        th = s.theta_s;
        K = Ks;
        C = 0.0;
        return;
    }
    const ff u = ff_from_d(ud);
    const ff L = ff_log(u, tab);
    const ff nL = ff_mul(ff_make(s.n_hi, s.n_lo), L);
    if (nL.hi > 80.0f) {                  // x > e^80: Se = x^-m, K and C vanish at double range
        th = s.theta_r + dth * ff_to_d(ff_exp(ff_neg(ff_mul(ff_make(s.m_hi, s.m_lo), nL)), tab));
        K = 0.0;
        C = 0.0;
        return;
    }
    const ff x = ff_exp(nL, tab);
    const ff onepx = ff_add_f(x, 1.0f);
    const ff l1 = ff_log(onepx, tab);
    const ff mm = ff_make(s.m_hi, s.m_lo);
    const ff se = ff_exp(ff_neg(ff_mul(mm, l1)), tab);
    const ff w = ff_div(ff_make(1.0f, 0.0f), onepx);
    const ff ys = ff_mul(ff_div(x, u), se);
    ff omy;
    if (ys.hi <= 0.5f) {
        omy = ff_add_f(ff_neg(ys), 1.0f);
    } else {
        const ff lg = (w.hi < 0.0078125f) ? ff_log1p_small(ff_neg(w)) : ff_log(ff_add_f(ff_neg(w), 1.0f), tab);
        const ff z = ff_mul(mm, lg);
        omy = (z.hi > -0.0078125f) ? ff_neg(ff_expm1_small(z)) : ff_add_f(ff_neg(ff_exp(z, tab)), 1.0f);
    }
    th = s.theta_r + dth * ff_to_d(se);
    K = Ks * ff_to_d(ff_mul(ff_sqrt(se), ff_mul(omy, omy)));
    C = s.cfac * ff_to_d(ff_mul(ys, w));
}

// The same van Genuchten / Mualem closures (h < 0) in FP64, with the
// table-driven exp / log of f64m.cuh: with u = -alpha h, L = log u (as a
// double-double), x = exp(n L), l1 = log1p(x) (double-double):
//   Se = exp(-m l1), w = 1/(1+x), ys = (x/(1+x))^m = (x/u) Se,
//   K = Ks sqrt(Se) (1 - ys)^2 with 1 - ys = -expm1(m log1p(-w)) when
//   ys > 1/2, C = (theta_s-theta_r) alpha n m ys w;
// sqrt(Se) = exp(-m l1 / 2) and Se its square (f64_exp_sqr), 1/u and w
// from the one reciprocal 1/(u (1 + x)), since each divide, square root
// and exponential costs GB300's narrow FP64 pipe a dozen instructions.
// n L and m l1 are formed with their rounding errors (two-product), so x and
// Se keep a few units in the last place however large |L| or l1 are.
// Beyond x = e^700 (a suction far outside any soil state) theta = theta_r +
// dtheta x^-m and K = C = 0; below u = 1e-30 (h within 1e-30/alpha of 0) ys
// is taken as exp(m (n L - l1)), the quotient x/u being out of range.
__device__ __forceinline__ void closure_vg_fp64(const DevSoil &s, double Ks, double h,
                                                const FFTables *__restrict__ tab, double &th, double &K, double &C)
{
    const double dth = s.theta_s - s.theta_r;
    const double u = -s.alpha * h;
    double Lh, Ll;
    f64_log_dd(u, tab, Lh, Ll);
    const double nh = s.n * Lh;
    const double nl = fma(s.n, Lh, -nh) + s.n * Ll;
    if (nh > 700.0) {
        th = s.theta_r + dth * f64_exp_nc(fmax(-s.m * nh, -700.0), tab);
        K = 0.0;
        C = 0.0;
        return;
    }
    // x = u^n; below e^-700 it is 0 to double precision beside 1 (Se = 1)
    const double x = nh >= -700.0 ? f64_exp_dd(nh, nl, tab) : 0.0;
    const double onepx = 1.0 + x;
    // one reciprocal serves w = 1/(1 + x) and 1/u (separate ones where the
    // product would overflow)
    const double uo = u * onepx;
    double w, iu;
    if (uo < 1e300) {
        const double q = rcp64(uo);
        w = q * u;
        iu = q * onepx;
    } else {
        w = rcp64(onepx);
        iu = rcp64(u);
    }
    double l1h, l1l;
    if (x >= 0.0078125) f64_log1p_big_dd(x, onepx, w, tab, l1h, l1l);
    else f64_log1p_dd(x, tab, l1h, l1l);
    // Se^(1/2) = exp(-m l1 / 2), with Se = (Se^(1/2))^2 from the same
    // exponential (K needs the root, theta and C need Se)
    const double hm = 0.5 * s.m;
    const double sh = -hm * l1h;                   // in [-350, 0]
    double s2, se;
    f64_exp_sqr(sh, fma(-hm, l1h, -sh) - hm * l1l, tab, s2, se);
    const double ys = u >= 1e-30 ? (x * iu) * se : f64_exp(s.m * ((nh - l1h) + (nl - l1l)), tab);
    double omy;
    if (ys <= 0.5) {
        omy = 1.0 - ys;
    } else {
        // 1 - ys = -expm1(m log(1 - w)), log(1 - w) = log(x/(1+x)) = n L - l1:
        // l1 inherits the rounding of x (about 1e-16 absolute), so the
        // difference of the two double-doubles serves only while |n L - l1| >
        // log(3/2), i.e. x < 2; beyond, log1p(-w)
        const double lw = x < 2.0 ? (nh - l1h) + (nl - l1l) : f64_log1p(-w, tab);
        omy = -f64_expm1_neg(s.m * lw, tab);
    }
    th = s.theta_r + dth * se;
    K = Ks * s2 * (omy * omy);
    C = s.cfac * (ys * w);
}

// Brooks and Corey's closures (the alternative Sec. 1 names), FP64: air-entry
// head h_b = -1/alpha, pore-size index lambda = n; Se = (h_b / h)^lambda below
// h_b and 1 above; theta = theta_r + (theta_s - theta_r) Se, C = dtheta/dh =
// -lambda (theta_s - theta_r) Se / h, K = Ks Se^((2 + 3 lambda)/lambda).
__device__ __forceinline__ void closure_bc(const DevSoil &s, double Ks, double h, double &th, double &K, double &C)
{
    const double hb = -1.0 / s.alpha, lam = s.n;
    if (h >= hb) {
        th = s.theta_s;
        K = Ks;
        C = 0.0;
        return;
    }
    const double ls = lam * log(hb / h);          // log Se
    const double se = exp(ls);
    const double dth = s.theta_s - s.theta_r;
    th = s.theta_r + dth * se;
    C = -lam * dth * se / h;
    K = Ks * exp(ls * (2.0 + 3.0 * lam) / lam);
}

// Closures of one cell at head h: theta*, K, C.  For h >= 0 (tie included)
// theta* = theta_s + S h, K = Ks, C = S, which makes d(theta*)/dh equal to
// Eq. 3 on both branches.  fp64 selects FP64 van Genuchten arithmetic
// instead of double-float.  Gardner (Eq. A6, a test model): K = Ks e^(alpha
// h), theta = theta_r + (theta_s-theta_r) e^(alpha h), in FP64.
__device__ __forceinline__ void closure(const DevSoil &s, double Ks, double h, const FFTables *__restrict__ tab,
                                        bool fp64, double &th, double &K, double &C)
{
    if (h >= 0.0) {
        th = s.theta_s + s.S * h;
        K = Ks;
        C = s.S;
        return;
    }
    if (s.model == M_GARDNER) {
        const double dth = s.theta_s - s.theta_r;
        const double e = exp(s.alpha * h);
        K = Ks * e;
        th = s.theta_r + dth * e;
        C = dth * s.alpha * e;
        return;
    }
    if (s.model == M_BROOKS_COREY) {
        closure_bc(s, Ks, h, th, K, C);
        return;
    }
    if (fp64) closure_vg_fp64(s, Ks, h, tab, th, K, C);
    else closure_vg_df(s, Ks, h, tab, th, K, C);
}

// Neighbour across face f of cell p = (i,j,k); false when outside the grid.
__device__ __forceinline__ bool neighbour(const Grid &g, long long p, int i, int j, int k, int f, long long &q)
{
    switch (f) {
    case F_XMIN: q = p - 1; return i > 0;
    case F_XMAX: q = p + 1; return i < g.nx - 1;
    case F_YMIN: q = p - g.nx; return j > 0;
    case F_YMAX: q = p + g.nx; return j < g.ny - 1;
    case F_ZMIN: q = p - g.sxy; return k > 0;
    default:     q = p + g.sxy; return k < g.nz - 1;
    }
}

// FP64 stencil with stored coefficients; get(q) supplies the vector value.
template <class Get>
__device__ __forceinline__ double apply64(const Grid &g, long long p, const double *__restrict__ Tx,
                                          const double *__restrict__ Ty, const double *__restrict__ Tz,
                                          const double *__restrict__ diag, Get get)
{
    int i, j, k;
    cell_ijk(g, p, i, j, k);
    double acc = diag[p] * get(p);
    if (i > 0) acc -= Tx[p - 1] * get(p - 1);
    if (i < g.nx - 1) acc -= Tx[p] * get(p + 1);
    if (j > 0) acc -= Ty[p - g.nx] * get(p - g.nx);
    if (j < g.ny - 1) acc -= Ty[p] * get(p + g.nx);
    if (k > 0) acc -= Tz[p - g.sxy] * get(p - g.sxy);
    if (k < g.nz - 1) acc -= Tz[p] * get(p + g.sxy);
    return acc;
}

// One cell of the Picard system (Sec. 2.2; see k_assemble):
//   c = V C^k / dt (chord slope of theta*, or C(h^k) when |h^k - h^n| <= eps),
//   interior faces T_f = Kbar_f A_f/d_f with Kbar_f = (K_P + K_N)/2 (or the
//   harmonic mean 2 K_P K_N / (K_P + K_N)) and explicit gravity
//   gf_f Kbar_f A_f, gf_f the elevation gradient along the face's outward
//   normal (+1 top, -1 bottom, 0 lateral on a z-up grid),
//   boundary terms of the face classes flagged in fl.
// With RESID, sT = sum over interior faces of T_f h^k_N (for b - A h^k).
// thp: theta*(h^{n-1}), read only by the BDF2 storage.
struct CellSystem {
    double c, rhs, diag, cb, sT, KP;
    double s0;        // storage part of rhs
    double Tup[3];
};

template <bool RESID>
__device__ __forceinline__ void assemble_cell(const Grid &g, const DevSoil *__restrict__ soils,
                                              const uint8_t *__restrict__ zone, const double *__restrict__ Ks,
                                              uint8_t fl, const StepParams &sp, long long p, int i, int j, int k,
                                              const double *__restrict__ hk, const double *__restrict__ hn,
                                              const double *__restrict__ thk, const double *__restrict__ thn,
                                              const double *__restrict__ K, const double *__restrict__ Can,
                                              const double *__restrict__ thp, double eps, double V_dt,
                                              CellSystem &out)
{
    const double hkP = hk[p], hnP = hn[p], KP = K[p];
    double C, s0;
    if (sp.bdf2) {
        // variable-step BDF2 (the multistep alternative Sec. 2.2 names) in the
        // mixed form V/dt [a0 theta^{n+1} - a1 theta^n + a2 theta^{n-1}],
        // theta^{n+1} linearised about h^k as in the modified Picard form
        C = sp.a0 * Can[p];
        s0 = V_dt * (C * hkP - (sp.a0 * thk[p] - sp.a1 * thn[p] + sp.a2 * thp[p]));
    } else if (sp.modified) {
        // modified Picard (Sec. 2.2, mass-conservative variant): theta*(h^{k+1})
        // ~ theta*(h^k) + C(h^k) (h^{k+1} - h^k), so the storage term is
        // c (h^{k+1} - h^k) + V (theta*(h^k) - theta*(h^n)) / dt
        C = Can[p];
        s0 = V_dt * C * hkP - V_dt * (thk[p] - thn[p]);
    } else {
        // classical Picard with the chord slope of theta* between h^n and h^k
        const double dh = hkP - hnP;
        // |dh| > eps compared on the IEEE bit patterns (both non-negative)
        const bool chord = (__double_as_longlong(dh) & 0x7fffffffffffffffLL) > __double_as_longlong(eps);
        C = chord ? (thk[p] - thn[p]) * rcp64(dh) : Can[p];
        s0 = V_dt * C * hnP;
    }
    const double c = V_dt * C;
    double diag = c, rhs = s0, cb = c;
    double sT = 0.0;
    double Tup[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int f = 0; f < 6; f++) {
        long long q;
        if (neighbour(g, p, i, j, k, f, q)) {
            const double KN = K[q];
            if (__double_as_longlong(KN) >= 0) {          // active neighbour (K >= 0; inactive K = -1)
                double Ks2 = KP + KN;                      // 2 Kbar
                if (g.harmonic) Ks2 = Ks2 > 0.0 ? 4.0 * KP * KN / Ks2 : 0.0;
                const double T = Ks2 * g.hw[f];            // Kbar A/d
                diag += T;
                if (f >= F_ZMIN || g.tilted) rhs = fma(Ks2, g.hg[f], rhs);   // explicit gravity, gf Kbar A
                if (f & 1) Tup[f >> 1] = T;
                if (RESID) sT = fma(T, hk[q], sT);
                continue;
            }
        }
        const double gs = g.gf[f];
        if (!(fl & (1u << f))) continue;    // closed face (lateral face on an inactive cell)
        int type = sp.bc_type[f];
        double hD = 0.0;
        if (type == BC_SEEPAGE) {
            if (hnP >= 0.0) { type = BC_DIRICHLET; hD = 0.0; }
            else type = BC_ZERO_FLUX;
        } else if (type == BC_DIRICHLET) {
            hD = sp.bc_val[f];
        }
        if (type == BC_DIRICHLET) {
            const DevSoil s = soils[zone[p]];
            double thD, KD, CD;
            closure(s, Ks[p], hD, g.tab, g.closure64, thD, KD, CD);
            const double T = KD * g.wb[f];
            diag += T;
            cb += T;
            rhs += T * hD + gs * KD * g.A[f];
        } else if (type == BC_FLUX) {
            rhs += sp.bc_val[f] * g.A[f];
        } else if (type == BC_FREE_DRAINAGE) {
            rhs += gs * KP * g.A[f];       // unit gradient: gravity outflow K(h^k) A (gs = -1 at a z-up bottom)
        }
    }
    out.c = c;
    out.s0 = s0;
    out.rhs = rhs;
    out.diag = diag;
    out.cb = cb;
    out.sT = sT;
    out.KP = KP;
    out.Tup[0] = Tup[0];
    out.Tup[1] = Tup[1];
    out.Tup[2] = Tup[2];
}

// Boundary inflow (fin >= 0) and outflow (fout >= 0) of one cell's boundary
// faces in the linear system solved for x (the water balance of Sec. 2.2's
// chord-slope scheme): Dirichlet T_D (h_D - x) + gf K(h_D) A, imposed flux,
// free drainage gf K(h^k) A, seepage as Dirichlet 0 while h^n >= 0.
__device__ __forceinline__ void boundary_fluxes(const Grid &g, const DevSoil &s, double Ksp, uint8_t fl,
                                                const StepParams &sp, double xp, double hnP, double Kold,
                                                double &fin, double &fout)
{
    fin = 0.0;
    fout = 0.0;
#pragma unroll
    for (int f = 0; f < 6; f++) {
        if (!(fl & (1u << f))) continue;
        const double gs = g.gf[f];
        int type = sp.bc_type[f];
        double hD = 0.0, flux = 0.0;
        if (type == BC_SEEPAGE) {
            if (hnP >= 0.0) { type = BC_DIRICHLET; hD = 0.0; }
            else type = BC_ZERO_FLUX;
        } else if (type == BC_DIRICHLET) {
            hD = sp.bc_val[f];
        }
        if (type == BC_DIRICHLET) {
            double thD, KD, CD;
            closure(s, Ksp, hD, g.tab, g.closure64, thD, KD, CD);
            const double T = KD * g.wb[f];
            flux = T * hD + gs * KD * g.A[f] - T * xp;
        } else if (type == BC_FLUX) {
            flux = sp.bc_val[f] * g.A[f];
        } else if (type == BC_FREE_DRAINAGE) {
            flux = gs * Kold * g.A[f];
        }
        if (flux > 0.0) fin += flux;
        else fout -= flux;
    }
}

}  // namespace rf
