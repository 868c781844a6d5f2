// f64m.cuh -- FP64 exp, log, log1p and expm1 for the closures of the plain
// FP64 path, by table-driven argument reduction.
//
// Method: P. T. P. Tang, "Table-driven implementation of the exponential
// function in IEEE floating-point arithmetic", ACM TOMS 15 (1989) 144-157,
// and "Table-driven implementation of the logarithm function in IEEE
// floating-point arithmetic", ACM TOMS 16 (1990) 378-400, with 1024-entry
// tables computed on the host in extended precision (F64_TAB below):
//   exp(y)  = 2^M 2^(j/1024) exp(r),  y = (1024 M + j) ln2/1024 + r,
//             |r| <= ln2/2048, exp(r) - 1 by its Taylor series to r^4
//             (truncation < 2^-64);
//   log(u)  = E ln2 + log(F) + log1p(f/F),  u = 2^E m, F = 1 + j/1024
//             nearest to m, f = m - F exact, |f/F| <= 2^-11, log1p by its
//             Taylor series to v^5 (truncation < 2^-57 relative);
// log1p(x) and expm1(z) reuse them with the exact corrections of 1 + x and
// of 2^M 2^(j/1024) - 1, and short Taylor series near 0.  The large tables
// buy the short polynomials: GB300's FP64 pipe, not memory, bounds the
// closures.  Each result is within a few units in the last place; the
// closures' parity tests bound theta* to 1e-15 relative against the
// oracle's pow forms.
//
// The tables live in FFTables (ff.cuh) beside the double-float ones.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ff.cuh"

namespace rf {

#ifdef __CUDACC__
// ln 2 split for exact products with integers of up to 11 bits: L_HI has 42
// significant bits.
constexpr double F64_LN2_HI = 0.6931471805598903;      // 0x3FE62E42FEFA3800
constexpr double F64_LN2_LO = 5.497923018708371e-14;   // ln 2 - F64_LN2_HI
constexpr double F64_INV_LN2_N = 1477.3197218702985;   // F64_TAB / ln 2
constexpr double F64_LN2_N_HI = F64_LN2_HI / F64_TAB;  // exact (a power-of-two scaling)
constexpr double F64_LN2_N_LO = F64_LN2_LO / F64_TAB;

// 2^k for integer k in [-1022, 1023] from its bit pattern.
__device__ __forceinline__ double f64_pow2i(int k)
{
    return __longlong_as_double((long long)(k + 1023) << 52);
}

// exp(y) = (th + th p + tl) 2^M: the table entry 2^(j/1024) = th + tl and
// p = exp(r) - 1, for y in [-745, 709.8].
__device__ __forceinline__ void f64_exp_core(double y, const FFTables *__restrict__ tab, double &th, double &tl,
                                             double &p, int &M)
{
    // N = nearest integer to y 1024/ln2 (round-to-nearest through the 1.5 2^52 shift)
    const double shifter = 6755399441055744.0;
    const double t = fma(y, F64_INV_LN2_N, shifter);
    const int n = (int)(__double_as_longlong(t) & 0xffffffffLL);
    const double N = t - shifter;
    const double r = fma(-N, F64_LN2_N_LO, fma(-N, F64_LN2_N_HI, y));   // |r| <= ln2/2048
    // exp(r) - 1 = r + r^2 (1/2 + r (1/6 + r/24))
    const double q = fma(r, fma(r, 1.0 / 24.0, 1.0 / 6.0), 0.5);
    p = fma(r * r, q, r);
    const int j = n & (F64_TAB - 1);
    M = n >> F64_TAB_BITS;                          // arithmetic shift: floor(n / 1024)
    const double2 T = tab->e2[j];
    th = T.x;
    tl = T.y;
}

// exp(y) for y in [-708, 709] (normal results; the caller keeps y there).
__device__ __forceinline__ double f64_exp_nc(double y, const FFTables *__restrict__ tab)
{
    double th, tl, p;
    int M;
    f64_exp_core(y, tab, th, tl, p, M);
    return (th + fma(th, p, tl)) * f64_pow2i(M);
}

// exp(y) for y in [-1400, 709.7]; 0 below about -745 (underflow), +inf
// above 709.78.
__device__ __forceinline__ double f64_exp(double y, const FFTables *__restrict__ tab)
{
    if (!(y < 709.782712893384)) return y != y ? y : __longlong_as_double(0x7ff0000000000000LL);
    if (y < -745.2) return 0.0;
    double th, tl, p;
    int M;
    f64_exp_core(y, tab, th, tl, p, M);
    const double v = th + fma(th, p, tl);           // 2^(j/1024) exp(r)
    if (M >= -1022) return v * f64_pow2i(M);
    return (v * f64_pow2i(M + 600)) * f64_pow2i(-600);   // subnormal result
}

// E = exp(hi + lo) and E^2, for |lo| <= ulp(hi) and hi in [-350, 350]: with
// E 2^-M = th + vl, vl = tl + th (p + lo) (to within p lo), E rounds th + vl
// once, and E^2 = th^2 + vl (2 th + vl) rounds once, th^2 exact inside the
// fused multiply-add.  Both within about half a unit in the last place.
__device__ __forceinline__ void f64_exp_sqr(double hi, double lo, const FFTables *__restrict__ tab, double &e,
                                            double &e2)
{
    double th, tl, p;
    int M;
    f64_exp_core(hi, tab, th, tl, p, M);
    const double vl = fma(th, p + lo, tl);
    e = (th + vl) * f64_pow2i(M);
    e2 = fma(th, th, vl * fma(2.0, th, vl)) * f64_pow2i(2 * M);
}

// log(u) for u > 0 (finite) as an unevaluated sum hi + lo (|lo| <= ulp(hi)):
// the exact part E ln2_hi + log(F)_hi and the rest, summed once.  u <= 0 or
// non-finite u are handled by the caller.
__device__ __forceinline__ void f64_log_dd(double u, const FFTables *__restrict__ tab, double &hi, double &lo)
{
    long long b = __double_as_longlong(u);
    int E = (int)(b >> 52) - 1023;
    if (E == -1023) {                              // subnormal: scale into the normal range
        b = __double_as_longlong(u * 18014398509481984.0);   // 2^54
        E = (int)(b >> 52) - 1023 - 54;
    }
    const long long mant = b & 0x000fffffffffffffLL;
    const double m = __longlong_as_double(mant | 0x3ff0000000000000LL);    // [1, 2)
    constexpr int SH = 52 - F64_TAB_BITS;
    const int j = (int)((mant + (1LL << (SH - 1))) >> SH);                 // nearest 1 + j/1024, j in [0, 1024]
    const double F = __longlong_as_double(0x3ff0000000000000LL + ((long long)j << SH));   // 2 at j = 1024
    const double f = m - F;                        // exact, |f| <= 2^-11
    const double v = f * tab->invF[j];
    // log1p(v) = v + v^2 (-1/2 + v (1/3 + v (-1/4 + v/5)))
    const double q = fma(v, fma(v, fma(v, 0.2, -0.25), 1.0 / 3.0), -0.5);
    const double p = fma(v * v, q, v);
    const double e = (double)E;
    const double2 LF = tab->lF[j];
    const double A = fma(e, F64_LN2_HI, LF.x);                   // exact: both on a 2^-42 grid
    const double B = fma(e, F64_LN2_LO, LF.y) + p;
    hi = A + B;
    lo = (A - hi) + B;                             // Fast2Sum (|A| >= |B| or A = 0)
}

// log(u) for u > 0 (finite); -inf at 0, NaN below.
__device__ __forceinline__ double f64_log(double u, const FFTables *__restrict__ tab)
{
    if (!(u > 0.0)) return u == 0.0 ? __longlong_as_double(0xfff0000000000000LL) : __longlong_as_double(0x7ff8000000000000LL);
    if (u == __longlong_as_double(0x7ff0000000000000LL)) return u;
    double hi, lo;
    f64_log_dd(u, tab, hi, lo);
    return hi;
}

// exp(hi + lo) for |lo| <= ulp(hi) and hi in [-708, 709]: exp(hi) (1 + lo).
__device__ __forceinline__ double f64_exp_dd(double hi, double lo, const FFTables *__restrict__ tab)
{
    const double e = f64_exp_nc(hi, tab);
    return fma(e, lo, e);
}

// log(1 + x) for x >= 2^-7 as hi + lo, given u = 1 + x (rounded) and an
// approximation rinv of 1/u (a few units in the last place suffice: it only
// scales the correction c/u, |c/u| < 2^-53).
__device__ __forceinline__ void f64_log1p_big_dd(double x, double u, double rinv, const FFTables *__restrict__ tab,
                                                 double &hi, double &lo)
{
    const double c = x - (u - 1.0);               // 1 + x = u + c exactly
    f64_log_dd(u, tab, hi, lo);
    lo = fma(c, rinv, lo);
}

// log(1 + x) for x > -1 as hi + lo.
__device__ __forceinline__ void f64_log1p_dd(double x, const FFTables *__restrict__ tab, double &hi, double &lo)
{
    if (fabs(x) < 0.0078125) {
        // x - x^2/2 + ... + x^8 / 8 (truncation < 2^-63 relative)
        const double q = fma(x, fma(x, fma(x, fma(x, fma(x, fma(x, -0.125, 1.0 / 7.0), -1.0 / 6.0), 0.2), -0.25),
                                    1.0 / 3.0), -0.5);
        hi = fma(x * x, q, x);
        lo = 0.0;
        return;
    }
    const double u = 1.0 + x;
    // 1 + x = u + c exactly (c = 0 for x in [-1, 1]); log(u + c) = log u + c/u
    // to first order (|c/u| < 2^-53); an FP32 quotient serves the correction,
    // which falls below the last place of log u once u exceeds 1e30
    const double c = x - (u - 1.0);
    f64_log_dd(u, tab, hi, lo);
    if (u < 1e30) lo += (double)((float)c * __frcp_rn((float)u));
}

__device__ __forceinline__ double f64_log1p(double x, const FFTables *__restrict__ tab)
{
    double hi, lo;
    f64_log1p_dd(x, tab, hi, lo);
    return hi + lo;
}

// exp(z) - 1 for z in [-745, 0].
__device__ __forceinline__ double f64_expm1_neg(double z, const FFTables *__restrict__ tab)
{
    if (z > -0.0078125) {
        // z + z^2/2 + ... + z^7/7! (truncation < 2^-66 relative)
        const double q = fma(z, fma(z, fma(z, fma(z, fma(z, 1.0 / 5040.0, 1.0 / 720.0), 1.0 / 120.0), 1.0 / 24.0),
                                    1.0 / 6.0), 0.5);
        return fma(z * z, q, z);
    }
    if (z < -40.0) return -1.0 + f64_exp_nc(fmax(z, -700.0), tab);
    double th, tl, p;
    int M;
    f64_exp_core(z, tab, th, tl, p, M);
    const double s = f64_pow2i(M);
    const double Th = th * s, Tl = tl * s;
    // 2^M 2^(j/1024) (1 + p) - 1 = (Th - 1) + (Tl + Th p); Th - 1 is exact for Th in [1/2, 2]
    return (Th - 1.0) + fma(Th, p, Tl);
}
#endif

}  // namespace rf
