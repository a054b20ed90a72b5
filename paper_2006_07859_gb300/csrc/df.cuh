// Double-float arithmetic: a value is an unevaluated sum hi + lo of two floats with |lo| <= ulp(hi) / 2,
// about 48 significant bits.  The error-free transformations are Knuth's two-sum, Dekker's fast two-sum
// (|a| >= |b|) and the product error through fma; every operation below rounds each float operation
// to nearest and must not be reassociated (no fast-math).
#pragma once

#include <cuda_runtime.h>

namespace tpe {

struct df {
    float hi, lo;
};

__device__ __forceinline__ df df_make(float a) { return df{a, 0.f}; }

// s + e = a + b exactly (any magnitudes)
__device__ __forceinline__ df two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return df{s, e};
}

// s + e = a + b exactly when |a| >= |b| (or a = 0)
__device__ __forceinline__ df fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return df{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df df_add(df x, df y)
{
    const df s = two_sum(x.hi, y.hi);
    const df t = two_sum(x.lo, y.lo);
    df r = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
    return fast_two_sum(r.hi, __fadd_rn(r.lo, t.lo));
}

// Sum of two values of the same sign (weights, squares): one two-sum on the high parts is enough, the
// error stays a few units of 2^-44 relative to the result.
__device__ __forceinline__ df df_add_pos(df x, df y)
{
    const df s = two_sum(x.hi, y.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}

__device__ __forceinline__ df df_neg(df x) { return df{-x.hi, -x.lo}; }
__device__ __forceinline__ df df_sub(df x, df y) { return df_add(x, df_neg(y)); }

__device__ __forceinline__ df df_mul(df x, df y)
{
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ df df_mul_f(df x, float f)
{
    const float p = __fmul_rn(x.hi, f);
    float e = __fmaf_rn(x.hi, f, -p);
    e = __fmaf_rn(x.lo, f, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ df df_sqr(df x)
{
    const float p = __fmul_rn(x.hi, x.hi);
    float e = __fmaf_rn(x.hi, x.hi, -p);
    e = __fmaf_rn(__fmul_rn(2.f, x.hi), x.lo, e);
    return fast_two_sum(p, e);
}

// x (1 + f) for a small f (|f| < 1e-5): the correction only touches the low part
__device__ __forceinline__ df df_scale1p(df x, float f) { return fast_two_sum(x.hi, __fmaf_rn(x.hi, f, x.lo)); }

__device__ __forceinline__ double df_to_double(df x) { return (double)x.hi + (double)x.lo; }

__device__ __forceinline__ df df_from_double(double v)
{
    const float h = (float)v;
    return df{h, (float)(v - (double)h)};
}

// a - b of two double-float values given as (hi, lo) float pairs
__device__ __forceinline__ df df_diff(float ah, float al, float bh, float bl) { return df_sub(df{ah, al}, df{bh, bl}); }

}  // namespace tpe
