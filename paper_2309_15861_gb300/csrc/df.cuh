// df.cuh -- double-float ("FP32 pair") arithmetic for the few steps of the
// ray path that need more than binary32: absolute positions tens of km from
// the array, path lengths of up to ~60 km held to a millimetre, and arrival
// times of ~1e5 ns held to 0.01 ns.
//
// A value is hi + lo with |lo| <= ulp(hi)/2 after normalisation.  The error-
// free transformations are the classical ones: Knuth's TwoSum, Dekker's
// Fast2Sum and the FMA-based exact product.  GB300 runs binary64 at a small
// fraction of its binary32 rate, so these pairs are the cheap way to carry
// ~44 significant bits where the path needs them.
#pragma once
#include <cuda_runtime.h>

struct df {
    float hi, lo;
};

__device__ __forceinline__ df df_make(float a) { return {a, 0.0f}; }

// Knuth TwoSum: s + e == a + b exactly.
__device__ __forceinline__ df two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

// Dekker Fast2Sum (requires |a| >= |b| or a == 0).
__device__ __forceinline__ df fast_two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return {s, e};
}

// Exact product through one fused multiply-add.
__device__ __forceinline__ df two_prod(float a, float b)
{
    float p = __fmul_rn(a, b);
    float e = __fmaf_rn(a, b, -p);
    return {p, e};
}

// From a binary64 value (used once per segment, at ingest).
__device__ __forceinline__ df df_from_double(double x)
{
    float hi = __double2float_rn(x);
    float lo = __double2float_rn(x - (double)hi);
    return {hi, lo};
}

__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ df operator+(df a, df b)
{
    df s = two_sum(a.hi, b.hi);
    df t = two_sum(a.lo, b.lo);
    s.lo = __fadd_rn(s.lo, t.hi);
    s = fast_two_sum(s.hi, s.lo);
    s.lo = __fadd_rn(s.lo, t.lo);
    return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df operator+(df a, float b)
{
    df s = two_sum(a.hi, b);
    s.lo = __fadd_rn(s.lo, a.lo);
    return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df operator-(df a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
__device__ __forceinline__ df operator-(df a, float b) { return a + (-b); }

__device__ __forceinline__ df operator*(df a, df b)
{
    df p = two_prod(a.hi, b.hi);
    p.lo = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
    return fast_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ df operator*(df a, float b)
{
    df p = two_prod(a.hi, b);
    p.lo = __fmaf_rn(a.lo, b, p.lo);
    return fast_two_sum(p.hi, p.lo);
}

// Quotient with two correction steps (~44 bits).
__device__ __forceinline__ df operator/(df a, df b)
{
    float q1 = __fdiv_rn(a.hi, b.hi);
    df r = a - b * q1;
    float q2 = __fdiv_rn(r.hi, b.hi);
    r = r - b * q2;
    float q3 = __fdiv_rn(r.hi, b.hi);
    df q = fast_two_sum(q1, q2);
    return q + q3;
}

// Square root: binary32 root plus one Newton correction in pair arithmetic.
__device__ __forceinline__ df df_sqrt(df a)
{
    if (a.hi <= 0.0f) return {0.0f, 0.0f};
    float s = __fsqrt_rn(a.hi);
    df r = a - two_prod(s, s);
    float c = __fdiv_rn(r.hi, 2.0f * s);
    return fast_two_sum(s, c);
}

__device__ __forceinline__ bool df_gt0(df a) { return a.hi > 0.0f || (a.hi == 0.0f && a.lo > 0.0f); }
__device__ __forceinline__ float df_f(df a) { return __fadd_rn(a.hi, a.lo); }
