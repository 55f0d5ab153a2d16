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

// Hardware reciprocal estimate (MUFU.RCP, about 1 ulp), no IEEE fix-up path.
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

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

// The same split with integer instructions only (GB300's binary64 pipe is
// narrow): hi is x rounded to nearest-even binary32, lo the rest rounded to
// binary32.  Valid for |x| in [2^-74, 2^127]; zero maps to zero, and smaller
// magnitudes (which no position or time reaches) to zero as well.
// df_hi_from_double_bits gives the same hi alone.
__device__ __forceinline__ float df_hi_from_double_bits(double x)
{
    unsigned long long b = (unsigned long long)__double_as_longlong(x);
    uint32_t sign = (uint32_t)(b >> 63) << 31;
    int e = (int)((b >> 52) & 0x7ff);
    if (e < 949) return __uint_as_float(sign);
    unsigned long long M = (1ull << 52) | (b & 0xFFFFFFFFFFFFFull);
    uint32_t top = (uint32_t)(M >> 29);
    uint32_t rem = (uint32_t)(M & 0x1FFFFFFFull);
    bool up = rem > (1u << 28) || (rem == (1u << 28) && (top & 1u));
    int fe = e - 1023 + 127;
    top += up ? 1u : 0u;
    if (top == (1u << 24)) { top >>= 1; fe += 1; }
    return __uint_as_float(sign | ((uint32_t)fe << 23) | (top & 0x7FFFFFu));
}

__device__ __forceinline__ df df_from_double_bits(double x)
{
    unsigned long long b = (unsigned long long)__double_as_longlong(x);
    uint32_t sign = (uint32_t)(b >> 63) << 31;
    int e = (int)((b >> 52) & 0x7ff);
    if (e < 949) return {__uint_as_float(sign), 0.0f};
    unsigned long long M = (1ull << 52) | (b & 0xFFFFFFFFFFFFFull);
    uint32_t top = (uint32_t)(M >> 29);                 // 24 significant bits
    uint32_t rem = (uint32_t)(M & 0x1FFFFFFFull);       // the 29 dropped bits
    bool up = rem > (1u << 28) || (rem == (1u << 28) && (top & 1u));
    int fe = e - 1023 + 127;
    top += up ? 1u : 0u;
    if (top == (1u << 24)) { top >>= 1; fe += 1; }
    float hi = __uint_as_float(sign | ((uint32_t)fe << 23) | (top & 0x7FFFFFu));
    int32_t r = (int32_t)rem - (up ? (1 << 29) : 0);    // x - hi in units of 2^(e-1075)
    float scale = __uint_as_float((uint32_t)(e - 948) << 23);
    float lo = __int2float_rn(r) * scale;
    return {hi, sign ? -lo : lo};
}

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

// Quotient: a hardware reciprocal estimate (MUFU, ~1 ulp) and two correction
// steps in pair arithmetic, each removing the residual of the previous
// estimate (~44 bits).  No IEEE-rounded binary32 division is involved.
__device__ __forceinline__ df operator/(df a, df b)
{
    float rb = rcp_approx(b.hi);
    rb = __fmaf_rn(rb, __fmaf_rn(-b.hi, rb, 1.0f), rb);    // one Newton step on 1/b.hi
    float q1 = a.hi * rb;
    df r = a - b * q1;
    float q2 = r.hi * rb;
    r = r - b * q2;
    float q3 = r.hi * rb;
    df q = fast_two_sum(q1, q2);
    return q + q3;
}

// Square root: s = a rsqrt(a) from the hardware estimate, then two Newton
// corrections in pair arithmetic.
__device__ __forceinline__ df df_sqrt(df a)
{
    if (a.hi <= 0.0f) return {0.0f, 0.0f};
    float rs = rsqrtf(a.hi);
    float s = a.hi * rs;
    df r = a - two_prod(s, s);
    float c = 0.5f * r.hi * rs;
    df x = fast_two_sum(s, c);
    r = a - x * x;
    return x + 0.5f * r.hi * rs;
}

__device__ __forceinline__ bool df_gt0(df a) { return a.hi > 0.0f || (a.hi == 0.0f && a.lo > 0.0f); }
__device__ __forceinline__ float df_f(df a) { return __fadd_rn(a.hi, a.lo); }
