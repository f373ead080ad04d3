// df64.cuh -- double-float arithmetic: a value is the unevaluated sum hi + lo
// of two FP32 numbers with |lo| <= ulp(hi) / 2, about 48 significant bits on
// the FP32 pipes.  This is NOT IEEE FP64: the exponent range is FP32's (values
// below about 1e-31 lose their low part, below 1e-38 become subnormal or 0),
// and every operation below rounds differently from FP64.
//
// The operations are built from error-free transformations that hold in IEEE
// FP32 with round-to-nearest (the compiler neither reassociates nor drops
// these operations; contraction into FMA only makes them more accurate):
// - TwoSum (Knuth, TAOCP vol. 2, 4.2.2): s + e = a + b exactly;
// - Fast2Sum (Dekker 1971): the same for |a| >= |b|, in three operations;
// - TwoProd with an FMA: p + e = a b exactly.
// Sum and product of two double-float numbers follow the "accurate" sum and
// the FMA-based product of Joldes, Muller and Popescu (ACM TOMS 44, 2017):
// relative errors below 3 u^2 and 5 u^2 (u = 2^-24).  The reciprocal takes
// one Newton correction of the correctly rounded FP32 reciprocal, whose
// residual 1 - b q is exact with an FMA; the square root one Karp-Markstein
// correction of the correctly rounded FP32 square root, whose residual
// a - s^2 is exact with an FMA.  Both land near 2^-47 relative.
//
// The overloads below let the stage's templated face flux (face_flux2) run
// on this type unchanged, for the evaluation of a double-float flux phase
// (moses_debug_flux_eval); no stepping launch uses it.  Include it after
// stage.cuh: the double-float fma would otherwise hide the FP64 one from the
// stage's non-template functions.
#pragma once
#include <cuda_runtime.h>

namespace moses {

struct df {
    float hi, lo;
    df() = default;
    __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
    // nearest double-float of an FP64 value (hi rounded to nearest, then the
    // exact remainder x - hi rounded: 48 of its 53 bits)
    __device__ explicit df(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
    __device__ double to_double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ df df_two_sum(float a, float b)
{
    const float s = a + b, bb = s - a;
    return df(s, (a - (s - bb)) + (b - bb));
}
__device__ __forceinline__ df df_fast_two_sum(float a, float b)  // |a| >= |b| (or a == 0)
{
    const float s = a + b;
    return df(s, b - (s - a));
}
__device__ __forceinline__ df df_two_prod(float a, float b)
{
    const float p = a * b;
    return df(p, fmaf(a, b, -p));
}

__device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }
__device__ __forceinline__ df operator+(df a, df b)
{
    const df s = df_two_sum(a.hi, b.hi), t = df_two_sum(a.lo, b.lo);
    const df v = df_fast_two_sum(s.hi, s.lo + t.hi);
    return df_fast_two_sum(v.hi, t.lo + v.lo);
}
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
__device__ __forceinline__ df operator*(df a, df b)
{
    const df c = df_two_prod(a.hi, b.hi);
    const float t = fmaf(a.hi, b.lo, a.lo * b.lo);
    return df_fast_two_sum(c.hi, c.lo + fmaf(a.lo, b.hi, t));
}
// a b + c, as a product and a sum (two roundings of the double-float result)
__device__ __forceinline__ df fma(df a, df b, df c) { return a * b + c; }

// 1/b for b > 0 normal: q = rn(1/b.hi), e = (1 - b.hi q) - b.lo q (the first
// difference exact with the FMA), 1/b = q (1 + e + ...) ~ q + q e
__device__ __forceinline__ df frcp(df b)
{
    const float q = __frcp_rn(b.hi);
    const float e = fmaf(-b.lo, q, fmaf(-b.hi, q, 1.0f));
    return df_fast_two_sum(q, q * e);
}
// sqrt(a), 0 for a <= 0: s = rn(sqrt(a.hi)), r = (a.hi - s^2) + a.lo (the
// first difference exact with the FMA), sqrt(a) = s + r / (2 s) + O(r^2)
__device__ __forceinline__ df fsqrt(df a)
{
    if (!(a.hi > 0.0f)) return df(0.0f, 0.0f);
    const float s = __fsqrt_rn(a.hi);
    const float r = fmaf(-s, s, a.hi) + a.lo;
    return df_fast_two_sum(s, r * (0.5f * __frcp_rn(s)));
}

// comparisons and the helpers of the flux (values normalised: the order of
// hi decides unless the two are equal)
__device__ __forceinline__ bool df_greater(df a, df b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }
__device__ __forceinline__ bool gtp(df a, df b) { return df_greater(a, b); }
__device__ __forceinline__ df maxnn(df a, df b) { return df_greater(a, b) ? a : b; }
__device__ __forceinline__ df tabs(df a) { return a.hi < 0.0f ? -a : a; }

}  // namespace moses
