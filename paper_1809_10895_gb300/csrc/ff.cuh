// ff.cuh -- double-float ("float-float") arithmetic for the closures.
//
// GB300 issues FP64 at 2 thread-ops/clk/SM, 64x below FP32, so the van
// Genuchten closures are evaluated with pairs of floats (hi + lo, about 48
// significant bits) and only converted to FP64 at their inputs and outputs.
// Building blocks (published methods):
//   * error-free transformations: TwoSum (Knuth, TAOCP vol. 2), Fast2Sum
//     (Dekker 1971), TwoProduct through a fused multiply-add;
//   * double-float add / multiply / divide / sqrt (Dekker 1971);
//   * exp and log by table-driven argument reduction (P. T. P. Tang, ACM
//     TOMS 15 (1989) 144-157 and 16 (1990) 378-400) with 64-entry tables of
//     2^(j/64), log(c_j) and 1/c_j computed on the host in double, and short
//     Taylor series of exp(r) - 1 and log(1 + t) for |r|, |t| < 1/128.
// The individual float operations use round-to-nearest intrinsics so the
// compiler cannot contract them into FMAs.
#pragma once

#include <cuda_runtime.h>

namespace rf {

struct ff {
    float hi, lo;
};

// 64-entry tables, filled on the host (see make_ff_tables).
// Entries of the FP64 argument-reduction tables (f64m.cuh).
constexpr int F64_TAB_BITS = 10;
constexpr int F64_TAB = 1 << F64_TAB_BITS;

struct FFTables {
    float2 exp2j[64];   // 2^(j/64)
    float2 logc[64];    // log(c_j), c_j = 1 + (j + 1/2)/64
    float2 invc[64];    // 1/c_j
    // FP64 tables of f64m.cuh (N = F64_TAB): e2[j] = (hi, lo) with
    // 2^(j/N) = hi + lo; lF[j] = (hi, lo) with log(1 + j/N) = hi + lo, hi on
    // the 2^-42 grid; invF = 1/(1 + j/N) rounded.  Each pair is one 16-byte
    // load: the lookups are gathers, one L1 wavefront per lane's line.
    double2 e2[F64_TAB];
    double2 lF[F64_TAB + 1];
    double invF[F64_TAB + 1];
};

#ifdef __CUDACC__
__device__ __forceinline__ ff ff_make(float hi, float lo) { return ff{hi, lo}; }

__device__ __forceinline__ ff two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return ff{s, e};
}

__device__ __forceinline__ ff fast_two_sum(float a, float b)   // |a| >= |b|
{
    const float s = __fadd_rn(a, b);
    const float e = __fsub_rn(b, __fsub_rn(s, a));
    return ff{s, e};
}

__device__ __forceinline__ ff two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);
    return ff{p, e};
}

__device__ __forceinline__ ff ff_add(ff a, ff b)
{
    ff s = two_sum(a.hi, b.hi);
    const ff t = two_sum(a.lo, b.lo);
    s.lo = __fadd_rn(s.lo, t.hi);
    s = fast_two_sum(s.hi, s.lo);
    s.lo = __fadd_rn(s.lo, t.lo);
    return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ ff ff_neg(ff a) { return ff{-a.hi, -a.lo}; }
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }

__device__ __forceinline__ ff ff_add_f(ff a, float b)
{
    ff s = two_sum(a.hi, b);
    s.lo = __fadd_rn(s.lo, a.lo);
    return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ ff ff_mul(ff a, ff b)
{
    ff p = two_prod(a.hi, b.hi);
    p.lo = __fmaf_rn(a.hi, b.lo, p.lo);
    p.lo = __fmaf_rn(a.lo, b.hi, p.lo);
    return fast_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ ff ff_mul_f(ff a, float b)
{
    ff p = two_prod(a.hi, b);
    p.lo = __fmaf_rn(a.lo, b, p.lo);
    return fast_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ ff ff_div(ff a, ff b)
{
    const float q1 = __fdiv_rn(a.hi, b.hi);
    const ff r = ff_sub(a, ff_mul_f(b, q1));
    const float q2 = __fdiv_rn(r.hi, b.hi);
    const ff r2 = ff_sub(r, ff_mul_f(b, q2));
    const float q3 = __fdiv_rn(r2.hi, b.hi);
    ff q = fast_two_sum(q1, q2);
    return ff_add_f(q, q3);
}

__device__ __forceinline__ ff ff_sqrt(ff a)
{
    if (!(a.hi > 0.0f)) return ff{0.0f, 0.0f};
    const float s = __fsqrt_rn(a.hi);
    const ff e = ff_sub(a, two_prod(s, s));
    return fast_two_sum(s, __fdiv_rn(e.hi, __fmul_rn(2.0f, s)));
}

__device__ __forceinline__ ff ff_from_d(double d)
{
    const float hi = __double2float_rn(d);
    const float lo = __double2float_rn(d - (double)hi);
    return ff{hi, lo};
}

__device__ __forceinline__ double ff_to_d(ff a) { return (double)a.hi + (double)a.lo; }

// exp(r) - 1 for |r| < 1/128: r + r^2 (1/2 + r (1/6 + r g)), with
// g = 1/24 + r/120 + r^2/720 + r^3/5040 in float (its rounding enters at
// order r^4 * 1e-7 < 1e-16).
__device__ __forceinline__ ff ff_expm1_small(ff r)
{
    const float x = r.hi;
    const float g = __fmaf_rn(x, __fmaf_rn(x, __fmaf_rn(x, 1.0f / 5040.0f, 1.0f / 720.0f), 1.0f / 120.0f),
                              1.0f / 24.0f);
    ff u = ff_add(ff_make(0x1.555556p-3f, -0x1.555556p-28f), ff_mul_f(r, g));   // 1/6 + r g
    u = ff_add_f(ff_mul(r, u), 0.5f);                                            // 1/2 + r (...)
    return ff_add(r, ff_mul(ff_mul(r, r), u));
}

// log(1 + t) for |t| < 1/128: t - t^2 (1/2 - t (1/3 - t h)), with
// h = 1/4 - t/5 + t^2/6 - t^3/7 + t^4/8 in float.
__device__ __forceinline__ ff ff_log1p_small(ff t)
{
    const float x = t.hi;
    const float h = __fmaf_rn(x, __fmaf_rn(x, __fmaf_rn(x, __fmaf_rn(x, 1.0f / 8.0f, -1.0f / 7.0f), 1.0f / 6.0f),
                                        -1.0f / 5.0f), 0.25f);
    ff u = ff_sub(ff_make(0x1.555556p-2f, -0x1.555556p-27f), ff_mul_f(t, h));   // 1/3 - t h
    u = ff_sub(ff_make(0.5f, 0.0f), ff_mul(t, u));                               // 1/2 - t (...)
    return ff_sub(t, ff_mul(ff_mul(t, t), u));
}

// exp(a) = 2^k 2^(j/64) exp(r), 64 k + j = round(a 64/ln2), |r| <= ln2/128.
__device__ __forceinline__ ff ff_exp(ff a, const FFTables *__restrict__ tab)
{
    if (a.hi > 88.0f) return ff{__int_as_float(0x7f800000), 0.0f};
    if (a.hi < -87.0f) return ff{0.0f, 0.0f};
    const float t = rintf(__fmul_rn(a.hi, 0x1.715476p+6f));
    const int N = (int)t;
    // r = a - t ln2/64 with ln2/64 = L1 + L2 + L3 (L1 has 11 bits, so t L1 is exact)
    const float r1 = __fsub_rn(a.hi, __fmul_rn(t, 0x1.63p-7f));
    ff r = two_sum(r1, a.lo);
    r = ff_sub(r, two_prod(t, -0x1.bd0106p-19f));
    r = ff_add_f(r, -__fmul_rn(t, 0x1.cf79acp-46f));
    const ff em1 = ff_expm1_small(r);
    const int j = N & 63;
    const int k = (N - j) >> 6;
    const float2 Tj = __ldg(&tab->exp2j[j]);
    const ff T = ff_make(Tj.x, Tj.y);
    ff res = ff_add(T, ff_mul(T, em1));
    res.hi = ldexpf(res.hi, k);
    res.lo = ldexpf(res.lo, k);
    return res;
}

// log(a), a > 0 (a.hi a normal float): a = 2^e m, m in [1, 2);
// log a = e ln2 + log c_j + log(1 + (m - c_j)/c_j), |m - c_j| <= 1/128.
__device__ __forceinline__ ff ff_log(ff a, const FFTables *__restrict__ tab)
{
    const int bits = __float_as_int(a.hi);
    const int e = ((bits >> 23) & 0xff) - 127;
    const float m = __int_as_float((bits & 0x007fffff) | 0x3f800000);
    const float lo = ldexpf(a.lo, -e);
    const int j = (bits >> 17) & 63;                       // leading 6 fraction bits
    const float c = 1.0f + ((float)j + 0.5f) * (1.0f / 64.0f);
    const ff f = two_sum(__fsub_rn(m, c), lo);             // m - c is exact
    const float2 ic = __ldg(&tab->invc[j]);
    const ff t = ff_mul(f, ff_make(ic.x, ic.y));
    const ff l1p = ff_log1p_small(t);
    const float2 lc = __ldg(&tab->logc[j]);
    const float ef = (float)e;
    ff el = two_prod(ef, 0x1.62e43p-1f);                   // e ln2 (hi part exact product)
    el.lo = __fmaf_rn(ef, -0x1.05c61p-29f, el.lo);
    el = fast_two_sum(el.hi, el.lo);
    return ff_add(ff_add(el, ff_make(lc.x, lc.y)), l1p);
}
#endif

// Host: fill the tables from double-precision libm values.
void make_ff_tables(FFTables *t);

}  // namespace rf
