// df32.cuh -- double-float ("two-FP32") arithmetic for the compensated
// accumulation mode. A value is the unevaluated sum hi + lo of two floats
// with |lo| <= ulp(hi)/2, giving about 44-48 significant bits.
//
// Built from the error-free transformations of Knuth (TwoSum) and Dekker
// (FastTwoSum; TwoProd via a fused multiply-add), the standard basis of
// double-float and double-double libraries. B300's FP64 rate is a small
// fraction of its FP32 rate, so the compensated mode keeps the cancelling
// J - S and flux-divergence steps on the FP32 pipes.
#pragma once
#include <cuda_runtime.h>

namespace rts {

struct df32 {
    float hi, lo;
};

// s + e = a + b exactly (no ordering requirement)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// s + e = a + b exactly when |a| >= |b|
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

// p + e = a * b exactly
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e)
{
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

// packed FP32 pairs: one instruction for both lanes, each lane rounded as its
// scalar form (Blackwell's FFMA2 / FMUL2 / FADD2)
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b as one packed FMA (b times -1 is exact, so a single rounding of a - b)
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.f), a); }

// two_sum on both lanes
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2 &s, float2 &e)
{
    s = add2(a, b);
    const float2 bb = sub2(s, a);
    e = add2(sub2(a, sub2(s, bb)), sub2(b, bb));
}

__device__ __forceinline__ df32 df_make(float a) { return {a, 0.f}; }

__device__ __forceinline__ df32 df_add(df32 a, df32 b)
{
    float s, e, t, f;
    two_sum(a.hi, b.hi, s, e);
    two_sum(a.lo, b.lo, t, f);
    e = __fadd_rn(e, t);
    fast_two_sum(s, e, s, e);
    e = __fadd_rn(e, f);
    fast_two_sum(s, e, s, e);
    return {s, e};
}

__device__ __forceinline__ df32 df_add(df32 a, float b)
{
    float s, e;
    two_sum(a.hi, b, s, e);
    e = __fadd_rn(e, a.lo);
    fast_two_sum(s, e, s, e);
    return {s, e};
}

__device__ __forceinline__ df32 df_neg(df32 a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df32 df_sub(df32 a, df32 b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ df32 df_mul(df32 a, float b)
{
    float p, e;
    two_prod(a.hi, b, p, e);
    e = __fmaf_rn(a.lo, b, e);
    fast_two_sum(p, e, p, e);
    return {p, e};
}

__device__ __forceinline__ df32 df_mul(df32 a, df32 b)
{
    float p, e;
    two_prod(a.hi, b.hi, p, e);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    fast_two_sum(p, e, p, e);
    return {p, e};
}

__device__ __forceinline__ double df_to_double(df32 a) { return (double)a.hi + (double)a.lo; }

// Double-float values of two points (lane x: the first, lane y: the second),
// each operation the df32 one above lane by lane with the same roundings.
// Negated operands are passed in where an error term needs one, so that the
// exact product errors come out negated (fma(a, -b, p) = -(a b - p)) and no
// packed negation is spent; results differ from the scalar forms at most in
// the sign of a zero.
struct df2 {
    float2 hi, lo;
};
__device__ __forceinline__ float2 neg2(float2 a) { return mul2(a, f2(-1.f)); }
__device__ __forceinline__ df2 df2_neg(df2 a) { return {neg2(a.hi), neg2(a.lo)}; }
__device__ __forceinline__ void fast_two_sum2(float2 a, float2 b, float2 &s, float2 &e)
{
    s = add2(a, b);
    e = sub2(b, sub2(s, a));
}
// s + e = a - b exactly (two_sum of a and -b)
__device__ __forceinline__ void two_diff2(float2 a, float2 b, float2 &s, float2 &e)
{
    s = sub2(a, b);
    const float2 bb = sub2(s, a);
    e = sub2(sub2(a, sub2(s, bb)), add2(b, bb));
}
// p + e with e given negated (ne = -e): fast_two_sum(p, e)
__device__ __forceinline__ df2 fast_two_sum2_ne(float2 p, float2 ne)
{
    const float2 s = sub2(p, ne);
    return {s, fma2(ne, f2(-1.f), sub2(p, s))};
}
__device__ __forceinline__ df2 df2_add(df2 a, df2 b)
{
    float2 s, e, t, f;
    two_sum2(a.hi, b.hi, s, e);
    two_sum2(a.lo, b.lo, t, f);
    e = add2(e, t);
    fast_two_sum2(s, e, s, e);
    e = add2(e, f);
    fast_two_sum2(s, e, s, e);
    return {s, e};
}
__device__ __forceinline__ df2 df2_sub(df2 a, df2 b)
{
    float2 s, e, t, f;
    two_diff2(a.hi, b.hi, s, e);
    two_diff2(a.lo, b.lo, t, f);
    e = add2(e, t);
    fast_two_sum2(s, e, s, e);
    e = add2(e, f);
    fast_two_sum2(s, e, s, e);
    return {s, e};
}
// a - (b, 0): the low-part steps of df_sub with a zero there are identities
__device__ __forceinline__ df2 df2_sub(df2 a, float2 b)
{
    float2 s, e;
    two_diff2(a.hi, b, s, e);
    e = add2(e, a.lo);
    fast_two_sum2(s, e, s, e);
    return {s, e};
}
// a * b, nb = -b
__device__ __forceinline__ df2 df2_mul(df2 a, df2 b, df2 nb)
{
    const float2 p = mul2(a.hi, b.hi);
    float2 ne = fma2(a.hi, nb.hi, p);
    ne = fma2(a.hi, nb.lo, ne);
    ne = fma2(a.lo, nb.hi, ne);
    return fast_two_sum2_ne(p, ne);
}
// (x, 0) * b, nx = -x (the zero low part's product is dropped)
__device__ __forceinline__ df2 df2_mul(float2 x, float2 nx, df2 b)
{
    const float2 p = mul2(x, b.hi);
    float2 ne = fma2(nx, b.hi, p);
    ne = fma2(nx, b.lo, ne);
    return fast_two_sum2_ne(p, ne);
}
// a * (y, 0), na = -a (the zero low part's product is dropped)
__device__ __forceinline__ df2 df2_mul(df2 a, df2 na, float2 y)
{
    const float2 p = mul2(a.hi, y);
    float2 ne = fma2(na.hi, y, p);
    ne = fma2(na.lo, y, ne);
    return fast_two_sum2_ne(p, ne);
}
__device__ __forceinline__ df2 df2_splat(df32 a) { return {f2(a.hi), f2(a.lo)}; }
__device__ __forceinline__ df2 df2_pair(df32 a, df32 b) { return {f2(a.hi, b.hi), f2(a.lo, b.lo)}; }

// Arithmetic-type shims so the Q step is written once for double and df32.
__device__ __forceinline__ double acc_zero(double *) { return 0.0; }
__device__ __forceinline__ df32 acc_zero(df32 *) { return {0.f, 0.f}; }
__device__ __forceinline__ double acc_add(double a, double b) { return a + b; }
__device__ __forceinline__ df32 acc_add(df32 a, df32 b) { return df_add(a, b); }
__device__ __forceinline__ double acc_sub(double a, double b) { return a - b; }
__device__ __forceinline__ df32 acc_sub(df32 a, df32 b) { return df_sub(a, b); }
__device__ __forceinline__ double acc_mul(double a, double b) { return a * b; }
__device__ __forceinline__ df32 acc_mul(df32 a, df32 b) { return df_mul(a, b); }
__device__ __forceinline__ double acc_to_double(double a) { return a; }
__device__ __forceinline__ double acc_to_double(df32 a) { return df_to_double(a); }
__device__ __forceinline__ double acc_from(double *, double v) { return v; }
__device__ __forceinline__ df32 acc_from(df32 *, float v) { return df_make(v); }
__device__ __forceinline__ df32 acc_from(df32 *, double v)
{
    float h = (float)v;
    return {h, (float)(v - (double)h)};
}

}  // namespace rts
