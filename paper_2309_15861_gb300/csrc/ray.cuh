// ray.cuh -- device code shared by the forward kernels (trace_kernels.cuh)
// and the tangent-linear adjoint (adjoint_kernels.cu): numerics, Philox,
// the atmosphere, the segment set-up, one ray, the hit test.
//
// Paper: Baack & Alameddine, "Comparison and efficiency of GPU accelerated
// optical light propagation in CORSIKA 8" (ICRC 2023).
//   Sec. 1.2      Frank-Tamm yield with its threshold, n constant over a step
//   Sec. 1.1      fluorescence yield N = Y dE (Eq. 1), isotropic emission
//   Sec. 1.2.1    cone vector p and the rotation M_Rod (here applied as
//                 cos(theta_c) d + sin(theta_c)(cos c M x + sin c M y))
//   Fig. 1        create at the origin, rotate, move to the emission point
//   Sec. 2        propagation to the ground with refraction
//
// Propagation.  Sec. 2 runs a straight line and then applies refraction
// corrections.  Here the correction is computed, not approximated: the
// straight vacuum line from the emission point is intersected with the
// observation level exactly (FP32 pairs), and the refracted ray's deviation
// from it -- angle (or distance), optical path and optical depth -- comes
// from the Snell / Bouguer invariant as integrals over altitude, written in
// a form free of cancellation and evaluated by 3-node Gauss-Legendre on
// altitude cells no wider than a fixed multiple of the local scale height.
// The bulk of the arithmetic is binary32; FP32 pairs (or binary64, by
// parameter) carry only the emission point, the vacuum path, the landing
// point and the arrival time.
//
// Geometry (flat / spherical Earth) and refraction (on / off) are template
// parameters, so each launch runs a kernel holding only its own branch.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "df.cuh"
#include "internal.h"

namespace clight {

#define FULL_MASK 0xffffffffu

// ------------------------------------------------------------------ numerics
__device__ __forceinline__ float ex2_approx(float x)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rsqrt_approx(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float sqrt_approx(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
// floor of 0 <= x < 2^23 as an integer, by one add rounded down (no F2I)
__device__ __forceinline__ int floor_small(float x)
{
    return (int)(__float_as_uint(__fadd_rd(x, 8388608.0f)) - 0x4B000000u);
}

template <class T> struct Num;
template <> struct Num<float> {
    static __device__ __forceinline__ float div(float a, float b) { return a * rcp_approx(b); }
    static __device__ __forceinline__ float rsq(float x) { return rsqrt_approx(x); }
    static __device__ __forceinline__ float sqr(float x) { return sqrtf(x); }
    static __device__ __forceinline__ void sincos2pi(float u, float *s, float *c) { sincospif(2.0f * u, s, c); }
};
template <> struct Num<double> {
    static __device__ __forceinline__ double div(double a, double b) { return a / b; }
    static __device__ __forceinline__ double rsq(double x) { return rsqrt(x); }
    static __device__ __forceinline__ double sqr(double x) { return sqrt(x); }
    static __device__ __forceinline__ void sincos2pi(double u, double *s, double *c) { sincospi(2.0 * u, s, c); }
};

// exact widening of a bulk-precision value into the pair/binary64 type
__device__ __forceinline__ void p_set(df &o, float x) { o = df_make(x); }
__device__ __forceinline__ void p_set(double &o, float x) { o = (double)x; }
__device__ __forceinline__ void p_set(double &o, double x) { o = x; }
template <class P, class T> __device__ __forceinline__ P p_of(T x)
{
    P o;
    p_set(o, x);
    return o;
}
// constants held both as FP32 pairs and binary64
__device__ __forceinline__ void p_const(df &o, float hi, float lo, double) { o = {hi, lo}; }
__device__ __forceinline__ void p_const(double &o, float, float, double d) { o = d; }
template <class P> __device__ __forceinline__ P pc(float hi, float lo, double d)
{
    P o;
    p_const(o, hi, lo, d);
    return o;
}
__device__ __forceinline__ float p_f(df a) { return __fadd_rn(a.hi, a.lo); }
__device__ __forceinline__ float p_f(double a) { return (float)a; }
__device__ __forceinline__ double p_d(df a) { return df_to_double(a); }
__device__ __forceinline__ double p_d(double a) { return a; }
template <class T> __device__ __forceinline__ T to_t(df a);
template <> __device__ __forceinline__ float to_t<float>(df a) { return p_f(a); }
template <class T> __device__ __forceinline__ T to_t(double a) { return (T)a; }
// a pair as the precise type (the FP64-guard variant widens it to binary64)
__device__ __forceinline__ void p_from_pair(df &o, df a) { o = a; }
__device__ __forceinline__ void p_from_pair(double &o, df a) { o = df_to_double(a); }

// ------------------------------------------------------------------ Philox
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): per round two 32x32->64
// products with 0xD2511F53 and 0xCD9E8D57, the Weyl key increments
// 0x9E3779B9 and 0xBB67AE85.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// (m + 1/2) 2^-23 from the top 23 bits: exact in binary32 and binary64.
template <class T> __device__ __forceinline__ T u01(uint32_t x)
{
    return (T)(x >> 9) * (T)1.1920928955078125e-07 + (T)5.9604644775390625e-08;
}
// binary32: 1 + m 2^-23 from the bits, minus 1, plus 2^-24 (all exact)
template <> __device__ __forceinline__ float u01<float>(uint32_t x)
{
    return (__uint_as_float((x >> 9) | 0x3f800000u) - 1.0f) + 5.9604644775390625e-08f;
}

// ------------------------------------------------------------------ atmosphere
// delta = n - 1 at one altitude (binary32 through the library exp2f, 2 ulp;
// the quadrature nodes use the raw MUFU estimate).
template <class T> struct AtmT;
template <> struct AtmT<float> {
    static __device__ __forceinline__ float delta(const DevAtm &A, float h)
    {
        if (h >= A.h_top) return 0.0f;
        // the layer's constants picked by selects (every parameter read at a
        // constant index, so no lane-dependent constant-bank access)
        float kb = A.kb[0], nl = A.nl2c[0];
#pragma unroll
        for (int j = 1; j < kMaxLayers; ++j) {
            const bool in = j < A.n_layers && h >= A.h_lo[j];
            kb = in ? A.kb[j] : kb;
            nl = in ? A.nl2c[j] : nl;
        }
        return kb * exp2f(h * nl);
    }
};
template <> struct AtmT<double> {
    static __device__ __forceinline__ double delta(const DevAtm &A, double h)
    {
        if (h >= A.h_top_d) return 0.0;
        int i = 0;
        for (int j = 1; j < A.n_layers; ++j)
            if (h >= A.h_lo_d[j]) i = j;
        return A.kb_d[i] * exp(-h * A.inv_c_d[i]);
    }
};

template <class T> __device__ __forceinline__ T earth_radius(const DevAtm &A)
{
    return sizeof(T) == 4 ? (T)A.R_E : (T)A.R_E_d;
}

// Altitude without cancellation: |r + R_E z| - R_E = (x^2 + y^2 + z (z + 2 R_E)) / (|r + R_E z| + R_E).
template <class T, bool SPH> __device__ __forceinline__ T altitude(const DevAtm &A, T x, T y, T z)
{
    if (!SPH) return z;
    const T RE = earth_radius<T>(A);
    T num = x * x + y * y + z * (z + (T)2 * RE);
    T zc = z + RE;
    return Num<T>::div(num, Num<T>::sqr(x * x + y * y + zc * zc) + RE);
}

// ------------------------------------------------------------------ pair refractivity
// Near the Cherenkov threshold beta n - 1 = delta - eps - eps delta is a
// small difference, whose relative error is that of delta times about
// kappa / 2, kappa = (delta + eps) / (beta n - 1).  binary32 delta is good to
// ~1e-6 (the millimetre rounding of the altitude, the exponential), so where
// kappa is large the step's refractivity is recomputed in FP32 pairs.
struct DfConst { float hi, lo; };
__host__ __device__ constexpr DfConst df_const(double x) { return {(float)x, (float)(x - (double)(float)x)}; }

// 2^a for a pair a (|a| < 120): a = n + f with n the integer nearest a.hi;
// 2^f = (e^x)^8 with x = f ln(2) / 8 (|x| < 0.044), e^x by its Taylor
// polynomial of degree 7 (truncation below 4e-16) in pair arithmetic, then
// three squarings and an exact scaling by 2^n.
__device__ __forceinline__ df df_exp2(df a)
{
    constexpr DfConst ln2_8 = df_const(0.69314718055994530942 / 8.0);
    constexpr DfConst c3 = df_const(1.0 / 6.0), c4 = df_const(1.0 / 24.0), c5 = df_const(1.0 / 120.0),
                      c6 = df_const(1.0 / 720.0), c7 = df_const(1.0 / 5040.0);
    const float n = rintf(a.hi);
    const df f = two_sum(a.hi - n, a.lo);              // a.hi - n is exact
    const df x = f * df{ln2_8.hi, ln2_8.lo};
    df p = df{c7.hi, c7.lo};
    p = p * x + df{c6.hi, c6.lo};
    p = p * x + df{c5.hi, c5.lo};
    p = p * x + df{c4.hi, c4.lo};
    p = p * x + df{c3.hi, c3.lo};
    p = p * x + 0.5f;
    p = p * x + 1.0f;
    p = p * x + 1.0f;
    p = p * p;
    p = p * p;
    p = p * p;
    const float sc = __uint_as_float((uint32_t)((int)n + 127) << 23);   // 2^n, exact
    return {p.hi * sc, p.lo * sc};
}

// Refractivity at the midpoint of a step (start x0, y0, z0 and unit
// direction d as pairs, length L) in FP32 pairs: the altitude without
// cancellation, delta = kb 2^(h nl2c) with both constants as pairs.
template <bool SPH>
__device__ __forceinline__ df delta_pair(const DevAtm &A, df x0, df y0, df z0, df dx, df dy, df dz, float L)
{
    const float hL = 0.5f * L;
    const df xm = x0 + dx * hL, ym = y0 + dy * hL, zm = z0 + dz * hL;
    df h = zm;
    if (SPH) {
        const df RE = {A.re_hi, A.re_lo};
        const df zc = zm + RE;
        const df num = xm * xm + ym * ym + zm * (zc + RE);
        h = num / (df_sqrt(xm * xm + ym * ym + zc * zc) + RE);
    }
    if (h.hi >= A.h_top) return {0.0f, 0.0f};
    int i = 0;
#pragma unroll
    for (int j = 1; j < kMaxLayers; ++j)
        if (j < A.n_layers && h.hi >= A.h_lo[j]) i = j;
    return df{A.kb[i], A.kb_lo[i]} * df_exp2(df{A.nl2c[i], A.nl2c_lo[i]} * h);
}

// ------------------------------------------------------------------ segment
// Everything one track step contributes to its photons (Sec. 1.2: the
// atmosphere is homogeneous over a step, so theta_c and the yield are
// per-step quantities).
template <class T, class P> struct Seg {
    P x0, y0, z0, t0;
    P rz0;               // z0 + R_E (spherical): Earth-centred height of the start
    P A0, C0;            // spherical: d . R0 and |R0|^2 - r_obs^2, R0 = (x0, y0, z0 + R_E)
    T dx, dy, dz;        // unit direction (binary32 part)
    T lx, ly, lz;        // its normalisation correction (pair low part)
    T e1x, e1y, e1z, e2x, e2y, e2z;   // M_Rod x, M_Rod y
    T sin_tc, kappa;     // sin(theta_c), 1 - cos(theta_c)
    T gerr;              // bound on the error of the beta n - 1 they came from (0: binary64)
    T L, inv_bc;         // step length, 1/(beta c) in ns/m
    T w_c, w_f;
    T h_mid;             // midpoint altitude
    uint32_t n_c, n_f;
    uint32_t shower;
    int bad;             // 0 ok, else CLIGHT_ERR_* code
    int guarded;
    int cut;             // 1: the angular cut removed the step's Cherenkov light
    T bux, buy, buz;     // beamed fluorescence: cone axis
    T bomc;              // and 1 - cos(half-angle); 0 = isotropic emission
};

constexpr double kInvC = 3.3356409519815204;    // ns/m

__device__ __forceinline__ bool finite_f(float v) { return (__float_as_uint(v) & 0x7f800000u) != 0x7f800000u; }
__device__ __forceinline__ bool finite_d(double v)
{
    return ((unsigned long long)__double_as_longlong(v) & 0x7ff0000000000000ull) != 0x7ff0000000000000ull;
}

// A step record from its four 16-byte words, field by field, so that it
// stays in registers (no copy through local memory).
__device__ __forceinline__ clight_segment seg_from_words(float4 a, float4 b, float4 c, float4 d)
{
    clight_segment s;
    s.x = __hiloint2double(__float_as_int(a.y), __float_as_int(a.x));
    s.y = __hiloint2double(__float_as_int(a.w), __float_as_int(a.z));
    s.z = __hiloint2double(__float_as_int(b.y), __float_as_int(b.x));
    s.t0 = __hiloint2double(__float_as_int(b.w), __float_as_int(b.z));
    s.dx = c.x; s.dy = c.y; s.dz = c.z; s.L = c.w;
    s.eps = d.x; s.dE = d.y;
    s.charge = __float_as_int(d.z);
    s.shower = __float_as_uint(d.w);
    return s;
}

__device__ __forceinline__ bool segment_ok(const clight_segment &s, const DevPar &P)
{
    return finite_d(s.x) && finite_d(s.y) && finite_d(s.z) && finite_d(s.t0) && finite_f(s.dx) &&
           finite_f(s.dy) && finite_f(s.dz) && finite_f(s.L) && finite_f(s.eps) && finite_f(s.dE) &&
           s.L >= 0.0f && s.eps >= 0.0f && s.eps < 1.0f && (int)s.shower < P.n_showers && s.shower < 0x7fffffffu;
}

// ------------------------------------------------------------------ fluorescence beaming
// Sec. 1.1.1 (optimisation): a step whose midpoint m lies at D = |C - m| >=
// 2 R_b from the array centre C emits its fluorescence into the cone about
// C - m of half-angle alpha = asin(R_b / D) + 5e-3 + L / D, uniformly in
// solid angle, with its photon number scaled by sin^2(alpha / 2).
// binary64: the decision and the cone as the oracle forms them.
__device__ __forceinline__ int beam_cone_d(double mx, double my, double mz, double L, const DevPar &P, double &ux,
                                           double &uy, double &uz, double &omc)
{
    double vx = __dsub_rn(P.beam_cx_d, mx), vy = __dsub_rn(P.beam_cy_d, my), vz = __dsub_rn(P.beam_cz_d, mz);
    double D2 = __dadd_rn(__dadd_rn(__dmul_rn(vx, vx), __dmul_rn(vy, vy)), __dmul_rn(vz, vz));
    double R = P.beam_r_d;
    if (!(D2 >= __dmul_rn(__dmul_rn(4.0, R), R))) return 0;
    double D = __dsqrt_rn(D2);
    double a = asin(R / D) + 5e-3 + L / D;
    double sh = sin(0.5 * a);
    omc = 2.0 * sh * sh;
    ux = vx / D; uy = vy / D; uz = vz / D;
    return 1;
}

// binary32, with the switch decided in binary64 where binary32 is not certain
template <class P>
__device__ __forceinline__ int beam_cone_t(const Seg<float, P> &g, const DevPar &Pp, float &ux, float &uy, float &uz,
                                           float &omc)
{
    float hl = 0.5f * g.L;
    float mx = p_f(g.x0) + hl * g.dx, my = p_f(g.y0) + hl * g.dy, mz = p_f(g.z0) + hl * g.dz;
    float vx = Pp.beam_cx - mx, vy = Pp.beam_cy - my, vz = Pp.beam_cz - mz;
    float D2 = vx * vx + vy * vy + vz * vz;
    float R = Pp.beam_r, F = 4.0f * R * R;
    if (fabsf(D2 - F) <= 1.0e-5f * (D2 + F)) {
        double dx = (double)g.dx + g.lx, dy = (double)g.dy + g.ly, dz = (double)g.dz + g.lz;
        double hd = 0.5 * (double)g.L, a, b, c, o;
        if (!beam_cone_d(p_d(g.x0) + hd * dx, p_d(g.y0) + hd * dy, p_d(g.z0) + hd * dz, (double)g.L, Pp, a, b, c, o))
            return 0;
    } else if (!(D2 > F)) {
        return 0;
    }
    float D = sqrtf(D2), iD = 1.0f / D;
    float a = asinf(R * iD) + 5.0e-3f + g.L * iD;
    float sh = sinf(0.5f * a);
    omc = 2.0f * sh * sh;
    ux = vx * iD; uy = vy * iD; uz = vz * iD;
    return 1;
}
__device__ __forceinline__ int beam_cone_t(const Seg<double, double> &g, const DevPar &Pp, double &ux, double &uy,
                                           double &uz, double &omc)
{
    double hd = 0.5 * g.L;
    return beam_cone_d(g.x0 + hd * g.dx, g.y0 + hd * g.dy, g.z0 + hd * g.dz, g.L, Pp, ux, uy, uz, omc);
}

// A direction at polar angle acos(ct) and azimuth 2 pi u about the axis u,
// rotated like the Cherenkov cone (M_Rod of the axis, Sec. 1.2.1).
template <class T>
__device__ __forceinline__ void cone_direction(T ux, T uy, T uz, T omct, T sp, T cp, T &x, T &y, T &z)
{
    // omct = 1 - cos(theta), small near the axis: no cancellation in sin(theta)
    T ct = (T)1 - omct;
    T ax = ux, ay = uy, az = uz - (T)1;
    T na2 = ax * ax + ay * ay + az * az;
    if (na2 > (T)0) {
        T inv = (T)1 / sqrt(na2);
        ax *= inv; ay *= inv; az *= inv;
    } else {
        ax = (T)1; ay = (T)0; az = (T)0;
    }
    T st = sqrt(omct * ((T)2 - omct));
    T e1x = (T)2 * ax * ax - (T)1, e1y = (T)2 * ax * ay, e1z = (T)2 * ax * az;
    T e2x = (T)2 * ay * ax, e2y = (T)2 * ay * ay - (T)1, e2z = (T)2 * ay * az;
    x = ct * ux + st * (cp * e1x + sp * e2x);
    y = ct * uy + st * (cp * e1y + sp * e2y);
    z = ct * uz + st * (cp * e1z + sp * e2z);
}

template <class T> __device__ __forceinline__ T fmax_t(T a, T b) { return a > b ? a : b; }

// ------------------------------------------------------------------ dispersion
// Sec. 1.2 keeps n(lambda) inside the Frank-Tamm integral.  With
// n - 1 = delta(h) g(lambda), g = (1 + B u^2) ig0 and u = 1/lambda (1/nm),
// beta n(u) - 1 = db g(u) - eps with db = delta (1 - eps); the yield is
// 2 pi alpha z^2 L int (1 - 1/(beta n)^2) du over the band where beta n > 1,
// and a photon's u has that integrand as its density.
template <class T> __device__ __forceinline__ T disp_gu(const DevAtm &A, T u)
{
    return sizeof(T) == 4 ? ((T)1 + (T)A.disp_B * u * u) * (T)A.disp_ig0
                          : ((T)1 + (T)A.disp_B_d * u * u) * (T)A.disp_ig0_d;
}
template <class T> __device__ __forceinline__ T disp_f(const DevAtm &A, T db, T eps, T u)
{
    T g1 = db * disp_gu<T>(A, u) - eps;
    if (!(g1 > (T)0)) return (T)0;
    T ib = (T)1 / ((T)1 + g1);
    return g1 * ((T)2 + g1) * ib * ib;
}
// the band [ulo, uhi] of u above threshold; false if empty
template <class T> __device__ __forceinline__ bool disp_band(const DevAtm &A, const DevPar &P, T db, T eps, T &ulo,
                                                             T &uhi)
{
    if (!(db > (T)0)) return false;
    const T B = sizeof(T) == 4 ? (T)A.disp_B : (T)A.disp_B_d;
    const T ig0 = sizeof(T) == 4 ? (T)A.disp_ig0 : (T)A.disp_ig0_d;
    const T il1 = sizeof(T) == 4 ? (T)P.il1 : (T)P.il1_d, dil = sizeof(T) == 4 ? (T)P.dil : (T)P.dil_d;
    T t = (eps / (db * ig0) - (T)1) / B;             // u_threshold^2
    T ut = t > (T)0 ? sqrt(t) : (T)0;
    T u2 = il1 - dil;
    ulo = ut > u2 ? ut : u2;
    uhi = il1;
    return ulo < uhi;
}
// int_ulo^uhi (1 - 1/(beta n)^2) du, 3-node Gauss-Legendre on `panels` panels
template <class T> __device__ __forceinline__ T disp_integral(const DevAtm &A, T db, T eps, T ulo, T uhi, int panels)
{
    T h = (uhi - ulo) / (T)panels, s = (T)0;
    for (int q = 0; q < panels; ++q) {
        T mid = ulo + ((T)q + (T)0.5) * h;
#pragma unroll
        for (int i = 0; i < kGLNodes; ++i) {
            T xg = sizeof(T) == 4 ? (T)A.gl_x[i] : (T)A.gl_x_d[i];
            T wg = sizeof(T) == 4 ? (T)A.gl_w[i] : (T)A.gl_w_d[i];
            s += wg * disp_f<T>(A, db, eps, mid + (T)0.5 * h * xg);
        }
    }
    return (T)0.5 * h * s;
}
// binary64 acceptance of a wavelength proposal, in the oracle's form
// (g1 = delta g - eps - eps delta g), for proposals binary32 cannot decide
__device__ __forceinline__ bool disp_accept_d(const DevAtm &A, const DevPar &P, double delta, double eps, double v,
                                              double w)
{
    double db = delta * (1.0 - eps), ulo, uhi;
    if (!disp_band<double>(A, P, db, eps, ulo, uhi)) return false;
    auto f = [&](double u) {
        double dg = delta * disp_gu<double>(A, u);
        double g1 = dg - eps - eps * dg;
        return g1 > 0 ? g1 * (2.0 + g1) / ((1.0 + g1) * (1.0 + g1)) : 0.0;
    };
    double u = ulo + v * (uhi - ulo);
    return w * f(uhi) < f(u);
}

// Wavelength of a Cherenkov photon with dispersion: u = 1/lambda by
// rejection on the band above threshold.  Proposal 0 uses (u0, u3); proposal
// m >= 1 uses word pair (m - 1) % 2 of Philox with counter word 3 =
// 2 + (m - 1) / 2; after 64 proposals the last one stands.  binary32, with
// proposals too close to call decided in binary64 from the midpoint
// refractivity recomputed at (xm, ym, zm).
static __device__ __noinline__ float disp_sample_f(const DevAtm &A, const DevPar &P, float db, float eps, float u0,
                                                   float u3, int64_t seg_global, uint32_t kk, double xm, double ym,
                                                   double zm, bool sph)
{
    float ulo, uhi;
    disp_band<float>(A, P, db, eps, ulo, uhi);
    float fmax = disp_f<float>(A, db, eps, uhi);
    float gt = db * disp_gu<float>(A, uhi);
    float band = 1.0e-6f * (1.0f + (gt + eps) / fmaxf(gt - eps, 1e-30f)) * fmax;
    float v = u0, wv = u3, u = ulo;
    uint4 xr = make_uint4(0u, 0u, 0u, 0u);
    double dmid = -1.0;
    for (int m = 0;; ++m) {
        u = ulo + v * (uhi - ulo);
        float diff = wv * fmax - disp_f<float>(A, db, eps, u);
        bool acc;
        if (fabsf(diff) <= band) {
            if (dmid < 0.0)
                dmid = AtmT<double>::delta(A, sph ? altitude<double, true>(A, xm, ym, zm) : zm);
            acc = disp_accept_d(A, P, dmid, (double)eps, (double)v, (double)wv);
        } else {
            acc = diff < 0.0f;
        }
        if (acc || m == 64) break;
        if ((m & 1) == 0) {
            xr = philox4x32_10(make_uint4((uint32_t)(uint64_t)seg_global, (uint32_t)((uint64_t)seg_global >> 32), kk,
                                          2u + (uint32_t)(m >> 1)),
                               P.seed, P.stream);
            v = u01<float>(xr.x); wv = u01<float>(xr.y);
        } else {
            v = u01<float>(xr.z); wv = u01<float>(xr.w);
        }
    }
    return u;
}

// the same in binary64 (plain path)
static __device__ __noinline__ double disp_sample_d(const DevAtm &A, const DevPar &P, double db, double eps,
                                                    double u0, double u3, int64_t seg_global, uint32_t kk)
{
    double ulo, uhi;
    disp_band<double>(A, P, db, eps, ulo, uhi);
    double fmax = disp_f<double>(A, db, eps, uhi);
    double v = u0, wv = u3, u = ulo;
    uint4 xr = make_uint4(0u, 0u, 0u, 0u);
    for (int m = 0;; ++m) {
        u = ulo + v * (uhi - ulo);
        if (wv * fmax < disp_f<double>(A, db, eps, u) || m == 64) break;
        if ((m & 1) == 0) {
            xr = philox4x32_10(make_uint4((uint32_t)(uint64_t)seg_global, (uint32_t)((uint64_t)seg_global >> 32), kk,
                                          2u + (uint32_t)(m >> 1)),
                               P.seed, P.stream);
            v = u01<double>(xr.x); wv = u01<double>(xr.y);
        } else {
            v = u01<double>(xr.z); wv = u01<double>(xr.w);
        }
    }
    return u;
}


// Yield and bunch count in binary64 (the plain path, and the guard of the
// FP32 path when its count is not certain).  Frank-Tamm (Sec. 1.2):
// N = 2 pi alpha z^2 (1/l1 - 1/l2) (1 - 1/(beta n)^2) L for beta n > 1.
template <bool SPH>
__device__ __forceinline__ void yield_fp64(const clight_segment &s, const DevAtm &A, const DevPar &P,
                                           double ux, double uy, double uz, double *Nc, double *sin2,
                                           double *kappa, double *Nf)
{
    double xm = s.x + 0.5 * (double)s.L * ux, ym = s.y + 0.5 * (double)s.L * uy,
           zm = s.z + 0.5 * (double)s.L * uz;
    // the altitude without cancellation (near the threshold the yield's
    // relative error is the refractivity's times kappa / 2)
    double h;
    if (SPH) {
        double zc = zm + A.R_E_d;
        h = (xm * xm + ym * ym + zm * (zm + 2.0 * A.R_E_d)) / (sqrt(xm * xm + ym * ym + zc * zc) + A.R_E_d);
    } else {
        h = zm;
    }
    double dl = AtmT<double>::delta(A, h);
    double eps = (double)s.eps;
    double g1 = dl - eps - eps * dl;               // beta n - 1
    double z2 = (double)s.charge * (double)s.charge;
    *Nc = 0.0;
    *sin2 = 0.0;
    *kappa = 0.0;
    double ulo, uhi;
    if (A.disp) {
        // the wavelength integral; the angle is per photon (db and eps passed on)
        double db = dl * (1.0 - eps);
        if (z2 > 0.0 && s.L > 0.0f && disp_band<double>(A, P, db, eps, ulo, uhi))
            *Nc = P.fta_d * z2 * disp_integral<double>(A, db, eps, ulo, uhi, 16) * (double)s.L;
        *sin2 = db;
        *kappa = eps;
    } else if (z2 > 0.0 && g1 > 0.0 && s.L > 0.0f) {
        double bn = 1.0 + g1;
        *kappa = g1 / bn;                           // 1 - cos(theta_c)
        *sin2 = g1 * (2.0 + g1) / (bn * bn);        // 1 - 1/(beta n)^2
        *Nc = P.band_d * z2 * (*sin2) * (double)s.L;
    }
    *Nf = (P.fyield_d > 0.0 && s.dE > 0.0f && s.L > 0.0f) ? P.fyield_d * (double)s.dE : 0.0;
    if (*Nf > 0.0 && P.beam) {
        double a, b, c, omc;
        if (beam_cone_d(xm, ym, zm, (double)s.L, P, a, b, c, omc)) *Nf *= 0.5 * omc;
    }
}

// ------------------------------------------------------------------ angular cut
// Sec. 1.2.1 (optimisation): a step keeps its Cherenkov light when its
// flight direction d is within the cut angle of the vector v from the step
// midpoint m to a target centre C, i.e. d . v >= |v| cos(cut).  The binary64
// form below is the decision (the oracle evaluates the same expression, in
// the same order, without contraction); binary32 decides only when its
// error bound leaves no doubt.
__device__ __forceinline__ bool cut_keep_d(const double d[3], const double m[3], double cx, double cy, double cz,
                                           double cosc)
{
    double vx = __dsub_rn(cx, m[0]), vy = __dsub_rn(cy, m[1]), vz = __dsub_rn(cz, m[2]);
    double dot = __dadd_rn(__dadd_rn(__dmul_rn(d[0], vx), __dmul_rn(d[1], vy)), __dmul_rn(d[2], vz));
    double nv = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(vx, vx), __dmul_rn(vy, vy)), __dmul_rn(vz, vz)));
    return __dsub_rn(dot, __dmul_rn(nv, cosc)) >= 0.0;
}

// +1 keep, -1 drop, 0 not certain in binary32.  Without a square root: for
// a cut below 90 degrees, d . v >= |v| cos <=> d . v >= 0 and
// (d . v)^2 - cos^2 |v|^2 >= 0.  mabs bounds |m|_1 + |c|_1 (the absolute
// error of v is below 1.2e-7 mabs).
__device__ __forceinline__ int cut_test_f(float dx, float dy, float dz, float mx, float my, float mz, float cx,
                                          float cy, float cz, float cos2, float mabs)
{
    float vx = cx - mx, vy = cy - my, vz = cz - mz;
    float dot = dx * vx + dy * vy + dz * vz;
    float v2 = vx * vx + vy * vy + vz * vz;
    float f = dot * fabsf(dot) - cos2 * v2;          // sign(dot) (d.v)^2 - cos^2 |v|^2
    float eb = 4.0e-6f * (v2 + mabs * mabs);
    return f > eb ? 1 : (f < -eb ? -1 : 0);
}

// Does the step keep its Cherenkov light?  (dxf, dyf, dzf): the unit
// direction in binary32.  The binary64 direction and midpoint (rounded as
// the oracle rounds them) are formed only when binary32 is not certain.
__device__ __forceinline__ void cut_exact_dm(const clight_segment &s, double d[3], double m[3])
{
    double n = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn((double)s.dx, (double)s.dx),
                                              __dmul_rn((double)s.dy, (double)s.dy)),
                                    __dmul_rn((double)s.dz, (double)s.dz)));
    d[0] = __ddiv_rn((double)s.dx, n); d[1] = __ddiv_rn((double)s.dy, n); d[2] = __ddiv_rn((double)s.dz, n);
    double hl = __dmul_rn(0.5, (double)s.L);
    m[0] = __dadd_rn(s.x, __dmul_rn(hl, d[0]));
    m[1] = __dadd_rn(s.y, __dmul_rn(hl, d[1]));
    m[2] = __dadd_rn(s.z, __dmul_rn(hl, d[2]));
}

static __device__ __noinline__ bool cut_keeps_v(double sx, double sy, double sz, float sL, float sdx, float sdy,
                                                float sdz, float dxf, float dyf, float dzf, const DevPar &P)
{
    clight_segment s;
    s.x = sx; s.y = sy; s.z = sz; s.L = sL; s.dx = sdx; s.dy = sdy; s.dz = sdz;
    float hl = 0.5f * s.L;
    float mx = (float)s.x + hl * dxf, my = (float)s.y + hl * dyf, mz = (float)s.z + hl * dzf;
    const float cos2 = P.cut_cos * P.cut_cos;
    float mabs = fabsf(mx) + fabsf(my) + fabsf(mz) + P.cut_cabs;
    double d[3], m[3];
    if (P.cut_mode == CLIGHT_CUT_CENTRE) {
        int r = cut_test_f(dxf, dyf, dzf, mx, my, mz, P.cut_cx, P.cut_cy, P.cut_cz, cos2, mabs);
        if (r != 0) return r > 0;
        cut_exact_dm(s, d, m);
        return cut_keep_d(d, m, P.cut_cx_d, P.cut_cy_d, P.cut_cz_d, P.cut_cos_d);
    }
    // the whole array first: seen from m, every telescope centre lies within
    // rho = asin(r / |v0|) of the mean centre, so the smallest angle to a
    // telescope is within [a0 - rho, a0 + rho] (2e-3 rad of margin)
    {
        float vx = P.cut_tx - mx, vy = P.cut_ty - my, vz = P.cut_tz - mz;
        float nv = sqrtf(vx * vx + vy * vy + vz * vz);
        if (nv > 2.0f * P.cut_tr) {
            float iv = 1.0f / nv;
            float ex = dxf - vx * iv, ey = dyf - vy * iv, ez = dzf - vz * iv;
            float a0 = 2.0f * asinf(fminf(1.0f, 0.5f * sqrtf(ex * ex + ey * ey + ez * ez)));
            float rho = asinf(P.cut_tr * iv);
            if (a0 - rho > P.cut_rad + 2e-3f) return false;
            if (a0 + rho < P.cut_rad - 2e-3f) return true;
        }
    }
    // the telescopes around the point where the step's line meets the array
    // plane are the likeliest to be inside the cone: a quick accept
    if (dzf < -0.05f) {
        float tp = (P.cut_tz - mz) / dzf;
        if (tp > 0.0f) {
            float px = mx + tp * dxf, py = my + tp * dyf;
            int ix = (int)floorf((px - P.cut_gx0) * P.cut_inv_gs), iy = (int)floorf((py - P.cut_gy0) * P.cut_inv_gs);
            for (int cy = max(iy - 1, 0); cy <= min(iy + 1, P.cut_ny - 1); ++cy)
                for (int cx = max(ix - 1, 0); cx <= min(ix + 1, P.cut_nx - 1); ++cx) {
                    int c = cy * P.cut_nx + cx;
                    int b = __ldg(P.cut_cell_start + c), e = __ldg(P.cut_cell_start + c + 1);
                    for (int q = b; q < e; ++q) {
                        float4 t = __ldg(P.cut_tel + __ldg(P.cut_cell_tel + q));
                        if (cut_test_f(dxf, dyf, dzf, mx, my, mz, t.x, t.y, t.z, cos2, mabs) > 0) return true;
                    }
                }
        }
    }
    // all telescopes, four at a time
    bool unsure = false;
    int j = 0;
    for (; j + 4 <= P.cut_n_tel; j += 4) {
        float4 t0 = __ldg(P.cut_tel + j), t1 = __ldg(P.cut_tel + j + 1);
        float4 t2 = __ldg(P.cut_tel + j + 2), t3 = __ldg(P.cut_tel + j + 3);
        int r0 = cut_test_f(dxf, dyf, dzf, mx, my, mz, t0.x, t0.y, t0.z, cos2, mabs);
        int r1 = cut_test_f(dxf, dyf, dzf, mx, my, mz, t1.x, t1.y, t1.z, cos2, mabs);
        int r2 = cut_test_f(dxf, dyf, dzf, mx, my, mz, t2.x, t2.y, t2.z, cos2, mabs);
        int r3 = cut_test_f(dxf, dyf, dzf, mx, my, mz, t3.x, t3.y, t3.z, cos2, mabs);
        if (r0 > 0 || r1 > 0 || r2 > 0 || r3 > 0) return true;
        if (r0 == 0 || r1 == 0 || r2 == 0 || r3 == 0) unsure = true;
    }
    for (; j < P.cut_n_tel; ++j) {
        float4 t = __ldg(P.cut_tel + j);
        int r = cut_test_f(dxf, dyf, dzf, mx, my, mz, t.x, t.y, t.z, cos2, mabs);
        if (r > 0) return true;
        if (r == 0) unsure = true;
    }
    if (!unsure) return false;
    cut_exact_dm(s, d, m);
    for (int j = 0; j < P.cut_n_tel; ++j) {
        float4 t = __ldg(P.cut_tel + j);
        if (cut_keep_d(d, m, (double)t.x, (double)t.y, (double)t.z, P.cut_cos_d)) return true;
    }
    return false;
}

template <class T, class P>
__device__ __forceinline__ void make_frame(Seg<T, P> &g)
{
    // A = unit bisector of the flight direction and -z; M x = 2 A_x A - x,
    // M y = 2 A_y A - y (columns of M_Rod = 2 A A^T - 1).
    T ax = g.dx, ay = g.dy, az = g.dz - (T)1;
    T na2 = ax * ax + ay * ay + az * az;
    if (na2 > (T)0) {
        T inv = sizeof(T) == 4 ? (T)rsqrtf((float)na2) : (T)1 / Num<T>::sqr(na2);
        ax *= inv; ay *= inv; az *= inv;
    } else {
        ax = (T)1; ay = (T)0; az = (T)0;
    }
    g.e1x = (T)2 * ax * ax - (T)1; g.e1y = (T)2 * ax * ay;        g.e1z = (T)2 * ax * az;
    g.e2x = (T)2 * ay * ax;        g.e2y = (T)2 * ay * ay - (T)1; g.e2z = (T)2 * ay * az;
}

// binary32 segment set-up with the binary64 guard on the integer bunch count.
// EXT = false drops the optional angular cut and fluorescence beaming from
// the compiled code (the launcher picks it when neither is on).
// Fluorescence count rule 1: the number that decides whether a step with
// fewer photons than one bunch emits a bunch of weight B (counter word 2 is
// 0xFFFFFFFF, outside the photon counters, word 3 the fluorescence process).
template <class T> __device__ __forceinline__ T roulette_u(int64_t seg_global, const DevPar &P)
{
    uint4 r = philox4x32_10(make_uint4((uint32_t)(uint64_t)seg_global, (uint32_t)((uint64_t)seg_global >> 32),
                                       0xFFFFFFFFu, 1u), P.seed, P.stream);
    return u01<T>(r.x);
}

// The low words of the pair direction of a binary32 unit vector d: the
// normalisation residual -(|d|^2 - 1)/2 d, from exact products.
__device__ __forceinline__ void dir_residual(float dx, float dy, float dz, float &lx, float &ly, float &lz)
{
    const df r2 = two_prod(dx, dx) + two_prod(dy, dy) + two_prod(dz, dz);
    const float e2 = p_f(r2 - 1.0f);
    lx = -0.5f * e2 * dx; ly = -0.5f * e2 * dy; lz = -0.5f * e2 * dz;
}

// FULL = false (the first pass of the two-pass path): the same bunch counts,
// Cherenkov cone and binary32 step, without what only a traced ray needs --
// the low words of the start, the direction residual, the time, the vacuum-
// line constants A0, C0 (zero, or the binary32 values).  The guard branches
// form the pairs they need with the same arithmetic, so the counts are
// identical in both passes.
template <bool SPH, bool EXT = true, bool DISP = true, bool FULL = true>
__device__ __forceinline__ void load_segment_f(const clight_segment &s, int64_t seg_global, const DevAtm &A,
                                               const DevPar &P, Seg<float, df> &g)
{
    g.bad = 0;
    g.guarded = 0;
    g.cut = 0;
    g.n_c = g.n_f = 0;
    g.w_c = g.w_f = 0.0f;
    g.shower = s.shower;
    g.h_mid = 0.0f;
    g.bux = g.buy = g.buz = g.bomc = 0.0f;
    float n2 = s.dx * s.dx + s.dy * s.dy + s.dz * s.dz;
    if (!segment_ok(s, P) || !(n2 > 0.0f)) {
        g.bad = CLIGHT_ERR_BAD_SEGMENT;
        g.dx = 0; g.dy = 0; g.dz = -1; g.lx = g.ly = g.lz = 0;
        g.x0 = g.y0 = g.z0 = g.t0 = g.rz0 = g.A0 = g.C0 = df_make(0.0f);
        g.L = 0; g.inv_bc = 0; g.sin_tc = 0; g.kappa = 0;
        make_frame(g);
        return;
    }
    // unit direction as a pair: the binary32 part normalised by one rsqrt,
    // the residual -(|d|^2 - 1)/2 d (from exact products) as the low part
    const float f = rsqrtf(n2);
    g.dx = s.dx * f; g.dy = s.dy * f; g.dz = s.dz * f;
    if (FULL) {
        dir_residual(g.dx, g.dy, g.dz, g.lx, g.ly, g.lz);
        g.x0 = df_from_double_bits(s.x);
        g.y0 = df_from_double_bits(s.y);
        g.z0 = df_from_double_bits(s.z);
        g.t0 = df_from_double_bits(s.t0);
    } else {
        g.lx = g.ly = g.lz = 0.0f;
        g.x0 = df_make(df_hi_from_double_bits(s.x));
        g.y0 = df_make(df_hi_from_double_bits(s.y));
        g.z0 = df_make(df_hi_from_double_bits(s.z));
        g.t0 = df_make(0.0f);
    }
    g.rz0 = SPH ? g.z0 + df{A.re_hi, A.re_lo} : g.z0;
    if (SPH && FULL) {
        // for the vacuum line of every Cherenkov photon of the step:
        // |R0 + l d|^2 - r_obs^2 = C0 + l (2 A0 + l)
        g.A0 = df{g.dz, g.lz} * g.rz0 + (g.dx * g.x0.hi + g.dy * g.y0.hi);
        g.C0 = (g.z0 - df{A.hobs_hi, A.hobs_lo}) * (g.z0 + df{A.k2_hi, A.k2_lo}) +
               (g.x0.hi * g.x0.hi + g.y0.hi * g.y0.hi);
    } else {
        g.A0 = g.C0 = df_make(0.0f);
    }
    g.L = s.L;
    g.inv_bc = Num<float>::div(3.3356409519815204f, 1.0f - s.eps);   // 1/(beta c), ns/m
    make_frame(g);

    // midpoint altitude and refractivity (n constant over the step)
    float hL = 0.5f * s.L;
    float xm = g.x0.hi + hL * g.dx, ym = g.y0.hi + hL * g.dy, zm = g.z0.hi + hL * g.dz;
    float hm = altitude<float, SPH>(A, xm, ym, zm);
    g.h_mid = hm;
    float dl = AtmT<float>::delta(A, hm);
    float eps = s.eps;
    float z2 = (float)s.charge * (float)s.charge;
    if (EXT && P.cut_mode != CLIGHT_CUT_OFF && z2 > 0.0f &&
        !cut_keeps_v(s.x, s.y, s.z, s.L, s.dx, s.dy, s.dz, g.dx, g.dy, g.dz, P)) {
        g.cut = 1;
        z2 = 0.0f;
    }
    // beta n - 1 = delta - eps - eps delta, kept as a small number
    float g1 = __fmaf_rn(-eps, dl, dl - eps);
    // error bound of g1 (delta known to ~1.5e-6 relative; generous factor)
    float eg = 4.0e-6f * dl + 2.4e-7f * (dl + eps);
    // near the threshold (kappa = (delta + eps) / g1 above 16, or the sign of
    // g1 not certain) the refractivity in FP32 pairs: g1 to ~1e-12 relative.
    // The lean set-up (FULL = false: counts and cone bounds only) keeps the
    // binary32 g1 and its bound eg: its counts are exact all the same (the
    // guard takes what eg leaves uncertain), and the classification carries
    // the cone's resulting direction error (gerr)
    if (FULL && !(DISP && A.disp) && z2 > 0.0f && s.L > 0.0f && g1 > -eg && 16.0f * g1 < dl + eps) {
        const df dlp = delta_pair<SPH>(A, g.x0, g.y0, g.z0, df{g.dx, g.lx}, df{g.dy, g.ly}, df{g.dz, g.lz}, s.L);
        const df g1p = (dlp - eps) - dlp * eps;
        dl = p_f(dlp);
        g1 = p_f(g1p);
        eg = 1.0e-11f * (dl + eps);
    }
    bool guard = false;
    float Nc = 0.0f;
    g.gerr = eg;
    if (DISP && A.disp) {
        // dispersion: the band integral; per-photon angles from (db, eps)
        float db = dl * (1.0f - eps), ulo, uhi;
        if (z2 > 0.0f && s.L > 0.0f) {
            bool band = disp_band<float>(A, P, db, eps, ulo, uhi);
            if (band) {
                Nc = P.fta * z2 * disp_integral<float>(A, db, eps, ulo, uhi, 4) * s.L;
                float gt = db * disp_gu<float>(A, uhi);
                float kap = (gt + eps) / fmaxf(gt - eps, 1e-30f);   // condition at the band top
                float x = Nc * P.inv_bunch;
                float ex = x * (2.0e-5f + 4.0e-6f * kap) + 1.0e-6f;
                if (ceilf(x - ex) != ceilf(x + ex)) guard = true;
                else g.n_c = (uint32_t)ceilf(x);
            } else if (ulo < uhi * (1.0f + 1.0e-5f)) {
                guard = true;                // the threshold sits at the band edge
            }
        }
        g.sin_tc = db;
        g.kappa = eps;
    } else if (z2 > 0.0f && s.L > 0.0f) {
        if (g1 > eg) {
            float bn = 1.0f + g1;
            float ib = rcp_approx(bn);
            float sin2 = g1 * (2.0f + g1) * ib * ib;
            Nc = P.band * z2 * sin2 * s.L;
            g.sin_tc = sqrtf(sin2);
            g.kappa = g1 * ib;
            float x = Nc * P.inv_bunch;
            float ex = x * (eg * rcp_approx(g1) * 2.0f + 2.0e-6f) + 1.0e-6f;
            // an uncertain integer count, or a cone so narrow that its binary32
            // angle would move photons by millimetres: recompute in binary64
            if (ceilf(x - ex) != ceilf(x + ex) || g1 < 1.0e-6f * dl) guard = true;
            else g.n_c = (uint32_t)ceilf(x);
        } else if (g1 > -eg) {
            guard = true;
        }
    }
    if (!guard && g.n_c == 0 && !(DISP && A.disp)) { g.sin_tc = 0.0f; g.kappa = 0.0f; }
    float Nf = 0.0f;
    bool fguard = false, roul = false;
    if (P.fyield > 0.0f && s.dE > 0.0f && s.L > 0.0f) {
        Nf = P.fyield * s.dE;
        float rel = 1.0e-6f;
        if (EXT && P.beam && beam_cone_t(g, P, g.bux, g.buy, g.buz, g.bomc)) {
            Nf *= 0.5f * g.bomc;
            rel = 1.0e-5f;                   // asin, sin and the geometry in binary32
        }
        float x = Nf * P.inv_bunch;
        float ex = x * rel + 1.0e-7f;
        if (ceilf(x - ex) != ceilf(x + ex)) {
            fguard = true;
        } else if (EXT && P.roulette && x < 1.0f) {
            float u = roulette_u<float>(seg_global, P);
            if (fabsf(u - x) <= ex) fguard = true;    // decided in binary64 below
            else { g.n_f = u < x ? 1u : 0u; roul = true; }
        } else {
            g.n_f = (uint32_t)ceilf(x);
        }
    }
    if (g.cut) guard = false;
    if (guard || fguard) {
        g.guarded = 1;
        float lx = g.lx, ly = g.ly, lz = g.lz;
        if (!FULL) dir_residual(g.dx, g.dy, g.dz, lx, ly, lz);
        double Ncd, sin2d, kapd, Nfd;
        yield_fp64<SPH>(s, A, P, (double)g.dx + (double)lx, (double)g.dy + (double)ly, (double)g.dz + (double)lz,
                        &Ncd, &sin2d, &kapd, &Nfd);
        if (guard) {
            double nb = ceil(Ncd / P.bunch_d);
            g.n_c = (uint32_t)nb;
            Nc = (float)Ncd;
            g.sin_tc = (DISP && A.disp) ? (float)sin2d : (float)sqrt(sin2d);
            g.kappa = (float)kapd;
            g.gerr = 0.0f;
            if (g.n_c > 0) g.w_c = (float)(Ncd / nb);
        }
        if (fguard) {
            double xd = Nfd / P.bunch_d;
            if (EXT && P.roulette && xd < 1.0) {
                g.n_f = roulette_u<double>(seg_global, P) < xd ? 1u : 0u;
                roul = true;
            } else {
                double nb = ceil(xd);
                g.n_f = (uint32_t)nb;
                Nf = (float)Nfd;
                if (g.n_f > 0) g.w_f = (float)(Nfd / nb);
            }
        }
    }
    if (!guard && g.n_c > 0) g.w_c = Nc * rcp_approx((float)g.n_c);
    if (roul) g.w_f = g.n_f > 0 ? (float)P.bunch_d : 0.0f;
    else if (!fguard && g.n_f > 0) g.w_f = Nf * rcp_approx((float)g.n_f);
}

// binary64 segment set-up (plain path).
template <bool SPH>
__device__ void load_segment_d(const clight_segment &s, int64_t seg_global, const DevAtm &A, const DevPar &P,
                               Seg<double, double> &g)
{
    g.bad = 0;
    g.gerr = 0.0;
    g.guarded = 0;
    g.cut = 0;
    g.n_c = g.n_f = 0;
    g.w_c = g.w_f = 0.0;
    g.shower = s.shower;
    g.bux = g.buy = g.buz = g.bomc = 0.0;
    double n2 = (double)s.dx * s.dx + (double)s.dy * s.dy + (double)s.dz * s.dz;
    if (!segment_ok(s, P) || !(n2 > 0.0)) {
        g.bad = CLIGHT_ERR_BAD_SEGMENT;
        return;
    }
    double inv = 1.0 / sqrt(n2);
    g.dx = s.dx * inv; g.dy = s.dy * inv; g.dz = s.dz * inv;
    g.lx = g.ly = g.lz = 0.0;
    g.x0 = s.x; g.y0 = s.y; g.z0 = s.z; g.t0 = s.t0;
    g.rz0 = SPH ? s.z + A.R_E_d : s.z;
    g.A0 = SPH ? g.dx * s.x + g.dy * s.y + g.dz * g.rz0 : 0.0;
    g.C0 = SPH ? (s.z - A.h_obs_d) * (s.z + A.k2_d) + s.x * s.x + s.y * s.y : 0.0;
    g.L = s.L;
    g.inv_bc = kInvC / (1.0 - (double)s.eps);
    make_frame(g);
    double Nc, sin2, kap, Nf;
    yield_fp64<SPH>(s, A, P, g.dx, g.dy, g.dz, &Nc, &sin2, &kap, &Nf);
    if (P.cut_mode != CLIGHT_CUT_OFF && s.charge != 0 && !cut_keeps_v(s.x, s.y, s.z, s.L, s.dx, s.dy, s.dz, (float)g.dx, (float)g.dy, (float)g.dz, P)) {
        g.cut = 1;
        Nc = 0.0;
    }
    if (Nf > 0.0 && P.beam && !beam_cone_t(g, P, g.bux, g.buy, g.buz, g.bomc)) g.bomc = 0.0;
    g.sin_tc = A.disp ? sin2 : sqrt(sin2);          // dispersion: (db, eps) for per-photon angles
    g.kappa = kap;
    if (Nc > 0.0) {
        double nb = ceil(Nc / P.bunch_d);
        g.n_c = (uint32_t)nb;
        g.w_c = Nc / nb;
    }
    if (Nf > 0.0 && P.roulette && Nf < P.bunch_d) {
        g.n_f = roulette_u<double>(seg_global, P) < Nf / P.bunch_d ? 1u : 0u;
        g.w_f = g.n_f ? P.bunch_d : 0.0;
    } else if (Nf > 0.0) {
        double nb = ceil(Nf / P.bunch_d);
        g.n_f = (uint32_t)nb;
        g.w_f = Nf / nb;
    }
}

// The step with its pairs widened to binary64 (the FP64-guard precision:
// native binary64 at the steps that carry pairs otherwise).
__device__ __forceinline__ void widen_seg(const Seg<float, df> &q, Seg<float, double> &qd)
{
    p_from_pair(qd.x0, q.x0); p_from_pair(qd.y0, q.y0); p_from_pair(qd.z0, q.z0);
    p_from_pair(qd.t0, q.t0); p_from_pair(qd.rz0, q.rz0);
    p_from_pair(qd.A0, q.A0); p_from_pair(qd.C0, q.C0);
    qd.dx = q.dx; qd.dy = q.dy; qd.dz = q.dz; qd.lx = q.lx; qd.ly = q.ly; qd.lz = q.lz;
    qd.e1x = q.e1x; qd.e1y = q.e1y; qd.e1z = q.e1z; qd.e2x = q.e2x; qd.e2y = q.e2y; qd.e2z = q.e2z;
    qd.sin_tc = q.sin_tc; qd.kappa = q.kappa; qd.gerr = q.gerr; qd.L = q.L; qd.inv_bc = q.inv_bc;
    qd.w_c = q.w_c; qd.w_f = q.w_f; qd.n_c = q.n_c; qd.n_f = q.n_f; qd.shower = q.shower;
    qd.bux = q.bux; qd.buy = q.buy; qd.buz = q.buz; qd.bomc = q.bomc;
    qd.h_mid = q.h_mid; qd.bad = q.bad; qd.guarded = q.guarded; qd.cut = q.cut;
}

// ------------------------------------------------------------------ one ray
template <class T, class P> struct RayOut {
    P X, Y;            // crossing of the plane z = h_obs
    P t;               // arrival time there
    T cx, cy, cz;      // arrival direction
    T lambda, weight;
    int status;        // 0 reached, 1 escaped, 2 under, 3 turned, 4 idle lane, 5 reached (grazing, not landed)
    uint32_t cells;    // quadrature cells integrated
};

// Quadrature of the refracted ray's deviation from the vacuum line.
//   I0: integral whose p_v multiple is the angle (spherical) or horizontal
//       distance (flat) the refracted ray falls short of the vacuum line;
//   I1: optical path minus vacuum path length;
//   I2: density-weighted path (rho / rho_ref) ds.
// r = R_E + h (spherical) or 1 (flat); q_v = r^2 - p_v^2,
// q = n^2 q_v + (n^2 - n_e^2) p_v^2 = n^2 r^2 - (n_e p_v)^2.
template <class T, bool WARP, bool SPH, bool REFR>
__device__ __forceinline__ void ray_quadrature(const DevAtm &A, T hcap, T he, T de, T pv2, T bf2, T gl, T &I0,
                                               T &I1, T &I2, uint32_t &ncell)
{
    I0 = I1 = I2 = (T)0;
    const T RE = earth_radius<T>(A);
    const T ne = (T)1 + de;
    for (int c = 0; c < A.n_cells; ++c) {
        const DevCell &C = A.cells[c];
        T lo = sizeof(T) == 4 ? (T)C.lo : (T)A.cell_lo_d[c];
        bool act = hcap > lo;
        if (WARP) {
            if (!__any_sync(FULL_MASK, act)) break;
        } else {
            if (!act) break;
        }
        if (!act) continue;
        ++ncell;
        T chi = sizeof(T) == 4 ? (T)C.hi : (T)A.cell_hi_d[c];
        T hi = hcap < chi ? hcap : chi;
        T mid = (T)0.5 * (lo + hi), half = (T)0.5 * (hi - lo);
        T kb = (sizeof(T) == 4 ? (T)C.kb : (T)A.cell_kb_d[c]) * gl;
        T rb = sizeof(T) == 4 ? (T)C.rb : (T)A.cell_rb_d[c];
        T nl = sizeof(T) == 4 ? (T)C.nl2c : (T)-A.cell_ic_d[c];
        T s0 = 0, s1 = 0, s2 = 0;
#pragma unroll
        for (int gi = 0; gi < kGLNodes; ++gi) {
            T xg, wg;
            if (sizeof(T) == 4) { xg = (T)A.gl_x[gi]; wg = (T)A.gl_w[gi]; }
            else { xg = (T)A.gl_x_d[gi]; wg = (T)A.gl_w_d[gi]; }
            T h = mid + half * xg;
            // float: 2^(h nl) with nl = -log2(e)/c; double: e^(h nl) with nl = -1/c
            T ex = sizeof(T) == 4 ? (T)ex2_approx((float)(h * nl)) : (T)exp((double)(h * nl));
            T dl = kb * ex;
            T rr = rb * ex;
            T r = SPH ? RE + h : (T)1;
            T qv = SPH ? (h - he) * ((T)2 * RE + h + he) + bf2 : bf2;
            if (REFR) {
                T n = (T)1 + dl;
                T n2 = n * n;
                T gg = (dl - de) * ((T)2 + dl + de);          // n^2 - n_e^2
                T q = n2 * qv + gg * pv2;
                T rq = Num<T>::rsq(q), rqv = Num<T>::rsq(qv);
                T sq = q * rq, sqv = qv * rqv;
                T cm = rq * rqv;
                T a = dl * ((T)2 + dl);                         // n^2 - 1
                s0 += wg * Num<T>::div(-r * gg * cm, ne * sqv + sq);
                s1 += wg * Num<T>::div(r * (n2 * a * qv - gg * pv2) * cm, n2 * sqv + sq);
                s2 += wg * (rr * n * r * rq);
            } else {
                T rqv = Num<T>::rsq(qv);
                s1 += wg * (dl * r * rqv);
                s2 += wg * (rr * r * rqv);
            }
        }
        I0 += s0 * half;
        I1 += s1 * half;
        I2 += s2 * half;
    }
}

// First-order straight-line corrections in the form the landing code takes
// (I0: the flat horizontal shortfall per unit sin, or the spherical angle
// shortfall per unit p_v; I1: optical excess; I2: density path).
template <class T, bool SPH, bool REFR>
__device__ __forceinline__ void straight_corrections(const DevAtm &A, T he, T de, T pv2, T bf2, T gl, T &I0,
                                                     T &I1, T &I2)
{
    const float hf = (float)he;
    float Dh, Rh;                                     // int_h^top delta, rho / rho_ref
    if (hf >= A.h_top) {
        Dh = 0.0f; Rh = 0.0f;
    } else {
        int i = 0;
#pragma unroll
        for (int j = 1; j < kMaxLayers; ++j)
            if (j < A.n_layers && hf >= A.h_lo[j]) i = j;
        float ex = ex2_approx(hf * A.nl2c[i]);
        Dh = A.lay_c[i] * A.kb[i] * ex + A.lay_E[i];
        Rh = A.lay_c[i] * A.rb[i] * ex + A.lay_F[i];
    }
    T J = (T)(A.D_obs - Dh) * gl, Jr = (T)(A.R_obs - Rh);
    const T h_obs = sizeof(T) == 4 ? (T)A.h_obs : (T)A.h_obs_d;
    T corr = de * (he - h_obs) - J;
    T mu2, s2, r2 = (T)1;
    if (SPH) {
        T re2 = bf2 + pv2;                            // r_e^2
        mu2 = bf2 / re2;
        s2 = pv2 / re2;
        r2 = re2;
    } else {
        mu2 = bf2;
        s2 = pv2;
    }
    T imu = Num<T>::rsq(mu2);                         // 1 / mu
    T imu3 = imu * imu * imu;
    I0 = SPH ? corr * imu3 * Num<T>::rsq(r2) * Num<T>::div((T)1, sizeof(T) == 4 ? (T)A.r_obs : (T)A.r_obs_d)
             : corr * imu3;
    I1 = REFR ? J * imu + s2 * corr * imu3 : J * imu; // a straight ray only gains delta ds
    I2 = Jr * imu;
}

// Optional features of the per-ray code, fixed at compile time so that the
// default kernel carries none of them: FEAT_EXT the angular cut and the
// fluorescence beaming; FEAT_STRAIGHT the straight-line propagator only (no
// quadrature); FEAT_RUNTIME both propagators, chosen by DevPar::prop;
// FEAT_DISP dispersion, active when DevAtm::disp.
constexpr int FEAT_EXT = 1, FEAT_STRAIGHT = 2, FEAT_RUNTIME = 4, FEAT_DISP = 8,
              FEAT_ALL = FEAT_EXT | FEAT_RUNTIME | FEAT_DISP;

// Rays that cannot land near a telescope skip the quadrature.  Bouguer's
// invariant n r sin(psi) with n growing downward makes the refracted ray
// steeper than its vacuum line at every radius; the vacuum line's zenith
// angle is largest at its landing point (sin psi = p_v / r grows as r
// falls).  With mu that smallest cosine, s = sqrt(1 - mu^2) and delta_max
// the largest refractivity, tan(psi_v) - tan(psi) <= s delta_max / mu^3 at
// every height, so the refracted crossing of the plane z = h_obs lies within
// s delta_max (h_e - h_obs + zeta) / mu^3 of the vacuum crossing (zeta, the
// depth of the sphere below the plane, adds the stretch from the sphere back
// up to the plane), and the arrival direction within s delta_max / mu of the
// vacuum one.  With a factor 1.25 and 5 cm for binary32 rounding: if no
// centre lies within that distance plus the hit test's search radius of the
// vacuum crossing, the ray hits nothing.  Returns true for such a ray.
// derr > 0: (dx, dy, dz) is known only to within that angle (cos_obs is
// then already a lower bound); the vacuum crossing moves by up to
// tp derr (1 + tan) and |d_z| by up to derr.
template <bool FINE>
__device__ __forceinline__ bool clr_clear(const DevTel &Tl, const uint8_t *clr, float x, float y, float rs);
template <bool FINE = false>
__device__ __forceinline__ bool clear_miss(float xe, float ye, float ze, float dx, float dy, float dz, float he,
                                           float cos_obs, float gl, const DevAtm &A, const DevTel &Tl,
                                           const uint8_t *clr, bool sph, bool refr, float widen = 0.0f,
                                           float derr = 0.0f)
{
    const float tp = (ze - A.h_obs) * rcp_approx(-dz);
    const float Xv = xe + tp * dx, Yv = ye + tp * dy;
    float mu = (sph ? fminf(cos_obs, -dz - derr) : -dz - derr) - 1.0e-3f;
    if (!(mu > 0.05f)) return false;
    const float s = sqrt_approx(1.0f - mu * mu);           // mu < 0.999
    const float im = rcp_approx(mu);
    const float sd = refr ? 1.25f * s * A.delta_max * gl : 0.0f;
    const float zeta = sph ? (Xv * Xv + Yv * Yv) * A.inv_r_obs : 0.0f;
    const float B = sd * ((he - A.h_obs) + zeta) * (im * im * im) + 0.05f + 1.05f * derr * tp * (1.0f + im);
    const float czb = -dz - derr - sd * im - 1.0e-5f;     // below the arrival |cz|
    if (!(czb > 0.05f)) return false;
    const float dzmax = fmaxf(fabsf(Tl.zmax - A.h_obs), fabsf(Tl.zmin - A.h_obs));
    const float rs = (Tl.Rmax + widen + dzmax * sqrt_approx(1.0f - czb * czb)) * rcp_approx(czb) + 2.0e-3f + B;
    if (Xv + rs < Tl.xmin || Xv - rs > Tl.xmax || Yv + rs < Tl.ymin || Yv - rs > Tl.ymax) return true;
    return clr_clear<FINE>(Tl, clr, Xv, Yv, rs);
}

// Does the clearance map rule out every centre within rs of (x, y)?  FINE:
// the fine map (global memory); else the coarse one at clr
// (shared memory; nullptr: no map).
template <bool FINE>
__device__ __forceinline__ bool clr_clear(const DevTel &Tl, const uint8_t *clr, float x, float y, float rs)
{
    const uint8_t *m = FINE ? Tl.fclr : clr;
    if (!m) return false;
    const float inv = FINE ? Tl.finv_cgs : Tl.inv_cgs;
    const float fx = (x - (FINE ? Tl.fcx0 : Tl.cx0)) * inv, fy = (y - (FINE ? Tl.fcy0 : Tl.cy0)) * inv;
    const int nx = FINE ? Tl.fcnx : Tl.cnx, ny = FINE ? Tl.fcny : Tl.cny;
    if (!(fx >= 0.0f && fy >= 0.0f && fx < (float)nx && fy < (float)ny)) return false;
    const int ci = floor_small(fy) * nx + floor_small(fx);
    return rs < (float)(FINE ? __ldg(m + ci) : m[ci]) * kClrQuantum;
}

// CULL (binary32 only): skip the quadrature for rays clear_miss rejects;
// they end with status 6 (reached the observation level, no telescope near;
// `widen` enlarges the telescopes' radius for that test).
template <class T, class P, bool WARP, bool SPH, bool REFR, int FEAT = FEAT_ALL, bool CULL = false>
__device__ __forceinline__ void trace_ray(const Seg<T, P> &g, int64_t seg_global, uint32_t k, bool active,
                                          const DevAtm &A, const DevPar &Pp, RayOut<T, P> &o,
                                          const DevTel *Tl = nullptr, const uint8_t *clr = nullptr,
                                          float widen = 0.0f)
{
    // ---- generation (Sec. 1.1, 1.2, 1.2.1; Fig. 1)
    uint32_t proc = k < g.n_c ? 0u : 1u;
    uint32_t kk = proc ? k - g.n_c : k;
    uint4 x = philox4x32_10(make_uint4((uint32_t)(uint64_t)seg_global,
                                       (uint32_t)((uint64_t)seg_global >> 32), kk, proc),
                            Pp.seed, Pp.stream);
    T u0 = u01<T>(x.x), u1 = u01<T>(x.y), u2 = u01<T>(x.z), u3 = u01<T>(x.w);
    P dgx, dgy, dgz;
    T lam, w;
    T kapc = (T)0, stc = (T)0, ccc = (T)0, scc = (T)0;      // the Cherenkov cone, for the vacuum line
    if (proc == 0) {
        T st = g.sin_tc, kap = g.kappa;
        if ((FEAT & FEAT_DISP) && A.disp) {
            // dispersion: u = 1/lambda by rejection on the band above threshold
            // (proposal 0 from (u0, u3); proposal m >= 1 from word pair (m - 1) % 2
            // of Philox with counter word 3 = 2 + (m - 1) / 2; the 64th stands)
            T db = g.sin_tc, eps = g.kappa;
            T u;
            if (sizeof(T) == 4) {
                double hl = 0.5 * (double)g.L;
                u = (T)disp_sample_f(A, Pp, (float)db, (float)eps, (float)u0, (float)u3, seg_global, kk,
                                     p_d(g.x0) + hl * ((double)g.dx + (double)g.lx),
                                     p_d(g.y0) + hl * ((double)g.dy + (double)g.ly),
                                     p_d(g.z0) + hl * ((double)g.dz + (double)g.lz), SPH);
            } else {
                u = (T)disp_sample_d(A, Pp, (double)db, (double)eps, (double)u0, (double)u3, seg_global, kk);
            }
            lam = (T)1 / u;
            T g1 = db * disp_gu<T>(A, u) - eps;
            T ib = (T)1 / ((T)1 + g1);
            st = sqrt(g1 * ((T)2 + g1)) * ib;
            kap = g1 * ib;
        } else {
            T il1 = sizeof(T) == 4 ? (T)Pp.il1 : (T)Pp.il1_d;
            T dil = sizeof(T) == 4 ? (T)Pp.dil : (T)Pp.dil_d;
            lam = Num<T>::div((T)1, il1 - u0 * dil);       // density ~ 1/lambda^2
        }
        T sc, cc;
        Num<T>::sincos2pi(u2, &sc, &cc);
        kapc = kap; stc = st; ccc = cc; scc = sc;
        T sx = -kap * g.dx + st * (cc * g.e1x + sc * g.e2x);
        T sy = -kap * g.dy + st * (cc * g.e1y + sc * g.e2y);
        T sz = -kap * g.dz + st * (cc * g.e1z + sc * g.e2z);
        // cos(theta_c) d + sin(theta_c)(cos c e1 + sin c e2), d kept as a pair
        dgx = p_of<P>(g.dx) + (g.lx + sx);
        dgy = p_of<P>(g.dy) + (g.ly + sy);
        dgz = p_of<P>(g.dz) + (g.lz + sz);
        w = g.w_c;
    } else {
        T fl1 = sizeof(T) == 4 ? (T)Pp.fl1 : (T)Pp.fl1_d;
        T fdl = sizeof(T) == 4 ? (T)Pp.fdl : (T)Pp.fdl_d;
        lam = fl1 + u0 * fdl;
        T sp, cp;
        Num<T>::sincos2pi(u2, &sp, &cp);
        if ((FEAT & FEAT_EXT) && g.bomc > (T)0) {
            T bx, by, bz;
            cone_direction<T>(g.bux, g.buy, g.buz, u3 * g.bomc, sp, cp, bx, by, bz);
            dgx = p_of<P>(bx);
            dgy = p_of<P>(by);
            dgz = p_of<P>(bz);
        } else {
            T cz = (T)2 * u3 - (T)1;                        // exact
            T sz = Num<T>::sqr(((T)1 - cz) * ((T)1 + cz));
            dgx = p_of<P>(sz * cp);
            dgy = p_of<P>(sz * sp);
            dgz = p_of<P>(cz);
        }
        w = g.w_f;
    }
    // dispersion: this photon's refractivity is delta(h) g(lambda)
    const T gl = ((FEAT & FEAT_DISP) && A.disp) ? disp_gu<T>(A, (T)1 / lam) : (T)1;
    T ell = u1 * g.L;
    P xe = g.x0 + ell * (g.dx + g.lx);
    P ye = g.y0 + ell * (g.dy + g.ly);
    P ze = g.z0 + ell * (g.dz + g.lz);
    P te = g.t0 + ell * g.inv_bc;
    o.lambda = lam;
    o.status = 0;

    T dx = to_t<T>(dgx), dy = to_t<T>(dgy), dz = to_t<T>(dgz);
    // spherical: z of the emission point enters only binary32 quantities here
    // (the pairs that need it use C0 and A0, or compute it below)
    T xef = to_t<T>(xe), yef = to_t<T>(ye);
    T zef = SPH ? to_t<T>(g.z0) + ell * (g.dz + g.lz) : to_t<T>(ze);
    const T h_obs = sizeof(T) == 4 ? (T)A.h_obs : (T)A.h_obs_d;
    const P Hobs = pc<P>(A.hobs_hi, A.hobs_lo, A.h_obs_d);     // exact constants for the pair arithmetic

    // ---- vacuum straight line to the observation level (exact geometry)
    P s_v;
    T he, de, pv2, bf2, bf, sqf = 0;
    bool esc = false, under = false, turned = false, grazing = false;
    if (SPH) {
        // b = -(d . R_e) = r_e cos(psi_e); C = |R_e|^2 - r_obs^2
        P b, C;
        const T A0f = to_t<T>(g.A0);
        if (proc == 0) {
            // Cherenkov: d_g = (1 - kappa) d + sin(theta_c)(cos c e1 + sin c e2) with
            // e1, e2 orthogonal to d, so d_g . R_e = A0 - kappa A0 + sin(theta_c)(cos c
            // e1 + sin c e2) . R0 + l (1 - kappa); only A0 and C0 need the pairs
            const T RZf = to_t<T>(g.z0) + earth_radius<T>(A);
            T E1 = g.e1x * to_t<T>(g.x0) + g.e1y * to_t<T>(g.y0) + g.e1z * RZf;
            T E2 = g.e2x * to_t<T>(g.x0) + g.e2y * to_t<T>(g.y0) + g.e2z * RZf;
            b = (-g.A0) + (kapc * A0f - stc * (ccc * E1 + scc * E2) - ell * ((T)1 - kapc));
            C = g.C0 + ell * ((T)2 * A0f + ell);
        } else {
            P Rz = g.rz0 + ell * (g.dz + g.lz);             // z_e + R_E
            b = -(dgz * Rz) - (dx * xef + dy * yef);
            P dzo = ze - Hobs;
            C = dzo * (ze + pc<P>(A.k2_hi, A.k2_lo, A.k2_d)) + (xef * xef + yef * yef);
        }
        he = altitude<T, SPH>(A, xef, yef, zef);
        de = AtmT<T>::delta(A, he) * gl;                     // n_e - 1
        esc = !(p_f(b) > 0.0f);
        under = he <= h_obs;
        T Rzf = zef + earth_radius<T>(A);
        T c1 = dy * Rzf - dz * yef, c2 = dz * xef - dx * Rzf, c3 = dx * yef - dy * xef;
        pv2 = c1 * c1 + c2 * c2 + c3 * c3;                   // (r_e sin psi_e)^2
        bf = to_t<T>(b);
        bf2 = bf * bf;                                       // (r_e cos psi_e)^2
        // s_v = b - sqrt(b^2 - C) = (C / b) / (1 + sqrt(1 - x)), x = C / b^2,
        // and 1 / (1 + sqrt(1 - x)) = 1/2 + g with g = x / (2 (1 + sqrt(1 - x))^2)
        // small enough that binary32 carries it to ~1e-9 absolute.
        T xx = Num<T>::div(to_t<T>(C), bf2);
        T om = (T)1 - xx;                                    // disc / b^2
        T discf = bf2 * om;
        if (REFR) {
            // reaches the observation sphere iff q(r_obs) > 0, with
            // q_v(r_obs) = disc: q(r_obs) = n_obs^2 disc + (n_obs^2 - n_e^2) p_v^2
            T dob = (sizeof(T) == 4 ? (T)A.delta_obs : (T)A.delta_obs_d) * gl;
            T nob = (T)1 + dob;
            T qL = nob * nob * discf + (dob - de) * ((T)2 + dob + de) * pv2;
            turned = !(qL > (T)0);
            grazing = !turned && !(om > (T)0);   // reaches, but the vacuum line misses: not landed
        } else {
            turned = !(om > (T)0);
        }
        if (!(esc || under || turned || grazing)) {
            T so = Num<T>::sqr(om);
            T gx = Num<T>::div(xx, (T)2 * ((T)1 + so) * ((T)1 + so));
            P f;
            if (sizeof(T) == 4) p_from_pair(f, df{0.5f, (float)gx});
            else f = p_of<P>((T)0.5 + gx);
            s_v = (C / b) * f;
            sqf = bf * so;                                   // r_obs cos(psi) of the vacuum line
        } else {
            s_v = p_of<P>((T)0);
        }
    } else {
        he = zef;
        de = AtmT<T>::delta(A, he) * gl;
        esc = !(p_f(dgz) < 0.0f);
        under = !(p_f(ze - Hobs) > 0.0f);
        if (!(esc || under)) s_v = (ze - Hobs) / (-dgz);
        else s_v = p_of<P>((T)0);
        pv2 = dx * dx + dy * dy;                             // sin^2 theta_e
        bf = -dz;
        bf2 = bf * bf;                                       // cos^2 theta_e
    }
    if (!active) { o.status = 4; }
    else if (esc) { o.status = 1; }
    else if (under) { o.status = 2; }
    else if (turned) { o.status = 3; }
    else if (grazing) { o.status = 5; }
    bool go = o.status == 0;
    if (CULL && sizeof(T) == 4 && go && Pp.cull &&
        clear_miss((float)xef, (float)yef, (float)zef, (float)dx, (float)dy, (float)dz, (float)he,
                   SPH ? (float)sqf * A.inv_r_obs : 0.0f, (float)gl, A, *Tl, clr, SPH, REFR, widen)) {
        o.status = 6;
        go = false;
    }

    // ---- refraction, optical path and optical depth by quadrature
    T htop = sizeof(T) == 4 ? (T)A.h_top : (T)A.h_top_d;
    T hcap = go ? (he < htop ? he : htop) : (T)-1e30;
    T I0, I1, I2;
    o.cells = 0;
    if ((FEAT & FEAT_STRAIGHT) || ((FEAT & FEAT_RUNTIME) && Pp.prop == CLIGHT_PROP_STRAIGHT)) {
        // straight line plus first-order corrections (Sec. 2): with
        // mu = cos(zenith at emission), J = int_{h_obs}^{h_e} delta dh and
        // corr = delta_e (h_e - h_obs) - J, to first order in delta the flat
        // ray falls short horizontally by sin / mu^3 * corr, its optical path
        // exceeds the vacuum one by J / mu + sin^2 / mu^3 * corr, and its
        // density path is int rho / rho_ref dh / mu (layer closed forms).
        straight_corrections<T, SPH, REFR>(A, go ? he : h_obs, de, pv2, bf2, gl, I0, I1, I2);
    } else {
        ray_quadrature<T, WARP, SPH, REFR>(A, hcap, he, de, pv2, bf2, gl, I0, I1, I2, o.cells);
    }
    if (!go) return;

    const T d_obs = (sizeof(T) == 4 ? (T)A.delta_obs : (T)A.delta_obs_d) * gl;
    const T n_obs = (T)1 + d_obs;
    const T ne = (T)1 + de;
    T dLx, dLy, dLz;
    P X, Y, tt;
    T chord = 0;
    if (SPH) {
        const T r_obs = sizeof(T) == 4 ? (T)A.r_obs : (T)A.r_obs_d;
        // the vacuum landing point on the observation sphere; its height
        // below the tangent plane follows from its horizontal distance
        // (zv = rho^2 / (r_obs + sqrt(r_obs^2 - rho^2))), so z needs no pair
        P Pvx = xe + s_v * dgx;
        P Pvy = ye + s_v * dgy;
        T RLx = to_t<T>(Pvx), RLy = to_t<T>(Pvy);
        T rho2 = RLx * RLx + RLy * RLy;
        T zv = Num<T>::div(rho2, r_obs + Num<T>::sqr(r_obs * r_obs - rho2));
        T RLz = r_obs - zv;
        T ir = sizeof(T) == 4 ? (T)A.inv_r_obs : (T)A.inv_r_obs_d;
        // T_v = r_obs d + cos(psi_v) R_L: in-plane tangent scaled by p_v
        T Tx = r_obs * dx + sqf * ir * RLx, Ty = r_obs * dy + sqf * ir * RLy, Tz = r_obs * dz + sqf * ir * RLz;
        T Rhx = RLx * ir, Rhy = RLy * ir, Rhz = RLz * ir;
        P PLx = Pvx, PLy = Pvy;
        T zeta = zv;                                          // h_obs - z of the landing point
        if (REFR) {
            T pv = Num<T>::sqr(pv2);
            T dphi = I0 * pv;
            T sfac = r_obs * I0;                              // r_obs dphi / p_v
            T c2 = (T)0.5 * r_obs * dphi * dphi;
            PLx = Pvx + (sfac * Tx - c2 * Rhx);
            PLy = Pvy + (sfac * Ty - c2 * Rhy);
            zeta = zv - (sfac * Tz - c2 * Rhz);
            T qvL = sqf * sqf;
            T gL = (d_obs - de) * ((T)2 + d_obs + de);
            T qL = n_obs * n_obs * qvL + gL * pv2;
            T inr = Num<T>::div((T)1, n_obs * r_obs);
            T cpsi = Num<T>::sqr(qL) * inr;
            T spsi = ne * pv * inr;
            T at = ne * inr - cpsi * I0;
            T ar = cpsi + spsi * dphi;
            dLx = at * Tx - ar * Rhx;
            dLy = at * Ty - ar * Rhy;
            dLz = at * Tz - ar * Rhz;
        } else {
            dLx = dx; dLy = dy; dLz = dz;
        }
        // from the observation sphere back to the tangent plane z = h_obs
        chord = Num<T>::div(zeta, dLz);
        X = PLx + chord * dLx;
        Y = PLy + chord * dLy;
    } else {
        X = xe + s_v * dgx;
        Y = ye + s_v * dgy;
        if (REFR) {
            X = X + I0 * dx;
            Y = Y + I0 * dy;
            T qL = n_obs * n_obs * bf2 + (d_obs - de) * ((T)2 + d_obs + de) * pv2;
            T f = Num<T>::div(ne, n_obs);
            dLx = f * dx;
            dLy = f * dy;
            dLz = -Num<T>::div(Num<T>::sqr(qL), n_obs);
        } else {
            dLx = dx; dLy = dy; dLz = dz;
        }
    }
    // time: t_e + (vacuum path + optical excess + chord) / c
    const T invc = (T)kInvC;
    P sv_t = s_v * pc<P>(A.invc_hi, A.invc_lo, kInvC);
    tt = te + sv_t + (I1 + n_obs * chord) * invc;
    T tau = 0;
    if (A.absorption) {
        T lr = Num<T>::div(sizeof(T) == 4 ? (T)A.lambda_ref : (T)A.lambda_ref_d, lam);
        T lr2 = lr * lr;
        tau = I2 * lr2 * lr2 * (sizeof(T) == 4 ? (T)A.inv_L0 : (T)A.inv_L0_d);
    }
    o.X = X;
    o.Y = Y;
    o.t = tt;
    o.cx = dLx; o.cy = dLy; o.cz = dLz;
    o.weight = A.absorption ? w * (sizeof(T) == 4 ? (T)expf((float)-tau) : (T)exp((double)-tau)) : w;
}

// ------------------------------------------------------------------ hits
__device__ __forceinline__ void write_hit(const DevOut &O, unsigned long long idx, int64_t seg, uint32_t k,
                                          uint32_t tel, float xr, float yr, float cx, float cy, float lam,
                                          float w, double t, unsigned long long key)
{
    if ((int64_t)idx >= O.capacity) return;
    float4 *p = reinterpret_cast<float4 *>(O.rec + idx);
    uint32_t slo = (uint32_t)(uint64_t)seg, shi = (uint32_t)((uint64_t)seg >> 32);
    p[0] = make_float4(__uint_as_float(slo), __uint_as_float(shi), __uint_as_float(k), __uint_as_float(tel));
    p[1] = make_float4(xr, yr, cx, cy);
    unsigned long long tb = (unsigned long long)__double_as_longlong(t);
    p[2] = make_float4(lam, w, __uint_as_float((uint32_t)tb), __uint_as_float((uint32_t)(tb >> 32)));
    O.keys[idx] = key;
    O.vals[idx] = (uint32_t)idx;
}

// The record alone, for the entry point that keeps no sort keys.
__device__ __forceinline__ void write_hit_record(clight_hit *rec, int64_t capacity, unsigned long long idx,
                                                 int64_t seg, uint32_t k, uint32_t tel, float xr, float yr,
                                                 float cx, float cy, float lam, float w, double t)
{
    if ((int64_t)idx >= capacity) return;
    float4 *p = reinterpret_cast<float4 *>(rec + idx);
    uint32_t slo = (uint32_t)(uint64_t)seg, shi = (uint32_t)((uint64_t)seg >> 32);
    p[0] = make_float4(__uint_as_float(slo), __uint_as_float(shi), __uint_as_float(k), __uint_as_float(tel));
    p[1] = make_float4(xr, yr, cx, cy);
    unsigned long long tb = (unsigned long long)__double_as_longlong(t);
    p[2] = make_float4(lam, w, __uint_as_float((uint32_t)tb), __uint_as_float((uint32_t)(tb >> 32)));
}

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Test the arrival line against the telescopes near the crossing point and
// append every hit.  A sphere of radius R is hit when the line passes closer
// than R to its centre; its centre can then lie at most R / |cz| from the
// crossing point, which bounds the cells searched.
template <class T, class P, bool WARP, bool NOALLOC = false>
__device__ __forceinline__ int hit_test(const RayOut<T, P> &o, int64_t seg_local, int64_t seg_global, uint32_t k,
                                        uint32_t shower, const DevAtm &A, const DevTel &Tl, const DevPar &Pp,
                                        const DevOut &O, unsigned &status_bits, const uint8_t *clr = nullptr)
{
    if (o.status != 0) return 0;
    float Xf = p_f(o.X), Yf = p_f(o.Y);
    float cz = (float)o.cz, cx = (float)o.cx, cy = (float)o.cy;
    if (!(finite_f(Xf) && finite_f(Yf) && cz < 0.0f)) return 0;
    float acz = fabsf(cz);
    float dzmax = fmaxf(fabsf(Tl.zmax - A.h_obs), fabsf(Tl.zmin - A.h_obs));
    float rs = (Tl.Rmax + dzmax * sqrtf(fmaxf(0.0f, 1.0f - acz * acz))) * rcp_approx(fmaxf(acz, 1e-6f)) + 1e-3f;
    if (Xf + rs < Tl.xmin || Xf - rs > Tl.xmax || Yf + rs < Tl.ymin || Yf - rs > Tl.ymax) return 0;
    if (clr) {
        // every centre the line can pass within R of lies within rs of the
        // crossing point; the clearance map bounds the nearest centre from below
        float fx = (Xf - Tl.cx0) * Tl.inv_cgs, fy = (Yf - Tl.cy0) * Tl.inv_cgs;
        if (fx >= 0.0f && fy >= 0.0f && fx < (float)Tl.cnx && fy < (float)Tl.cny) {
            int ci = (int)fy * Tl.cnx + (int)fx;
            if (rs < (float)clr[ci] * kClrQuantum) return 0;
        }
    }
    int ix0 = max(0, (int)floorf((Xf - rs - Tl.gx0) * Tl.inv_gs));
    int ix1 = min(Tl.nx - 1, (int)floorf((Xf + rs - Tl.gx0) * Tl.inv_gs));
    int iy0 = max(0, (int)floorf((Yf - rs - Tl.gy0) * Tl.inv_gs));
    int iy1 = min(Tl.ny - 1, (int)floorf((Yf + rs - Tl.gy0) * Tl.inv_gs));
    int nh = 0;
    for (int iy = iy0; iy <= iy1; ++iy) {
        for (int ix = ix0; ix <= ix1; ++ix) {
            int cell = iy * Tl.nx + ix;
            int b = __ldg(Tl.cell_start + cell), e = __ldg(Tl.cell_start + cell + 1);
            for (int q = b; q < e; ++q) {
                int j = __ldg(Tl.cell_tel + q);
                float4 tp = __ldg(Tl.tel + j);
                // crossing point relative to the centre, at the plane z = z_j
                float dzj = tp.z - A.h_obs;
                float sj = Num<float>::div(dzj, cz);
                float xr = p_f(o.X - (T)tp.x) + sj * cx;
                float yr = p_f(o.Y - (T)tp.y) + sj * cy;
                // impact parameter
                float wd = xr * cx + yr * cy;
                float d2 = xr * xr + yr * yr - wd * wd;
                if (d2 < tp.w * tp.w) {
                    ++nh;
                    P tjp = o.t + (T)(A.n_obs * sj) * (T)kInvC;
                    double tj = p_d(tjp);                        // one conversion per hit
                    uint32_t group = shower * (uint32_t)Tl.n_tel + (uint32_t)j;
                    if (NOALLOC) {
                        // no sort keys: the record goes straight to the caller's
                        // buffer and O.keys holds one hit counter per group
                        unsigned m = __activemask();
                        int leader = __ffs(m) - 1;
                        unsigned long long base = 0;
                        if ((int)(threadIdx.x & 31) == leader) base = atomicAdd(O.ctr + CTR_CURSOR, (unsigned long long)__popc(m));
                        base = __shfl_sync(m, base, leader);
                        unsigned long long idx = base + __popc(m & lanemask_lt());
                        write_hit_record(O.rec, O.capacity, idx, seg_global, k, (uint32_t)j, xr, yr, cx, cy,
                                         (float)o.lambda, (float)o.weight, tj);
                        // one atomic per group among the lanes hitting together
                        const unsigned same = __match_any_sync(m, group);
                        if ((int)(threadIdx.x & 31) == __ffs(same) - 1)
                            atomicAdd(O.keys + group, (unsigned long long)__popc(same));
                        continue;
                    }
                    unsigned long long key;
                    if (Pp.k_bits < 32 && k >= (1u << Pp.k_bits)) {
                        status_bits |= 1u << CLIGHT_ERR_LIMIT;
                        key = ~0ull;
                    } else {
                        key = ((unsigned long long)group << (Pp.seg_bits + Pp.k_bits)) |
                              ((unsigned long long)seg_local << Pp.k_bits) | (unsigned long long)k;
                    }
                    unsigned long long idx;
                    if (WARP) {
                        unsigned m = __activemask();
                        int leader = __ffs(m) - 1;
                        unsigned long long base = 0;
                        if ((int)(threadIdx.x & 31) == leader) base = atomicAdd(O.ctr + CTR_CURSOR, (unsigned long long)__popc(m));
                        base = __shfl_sync(m, base, leader);
                        idx = base + __popc(m & lanemask_lt());
                    } else {
                        idx = atomicAdd(O.ctr + CTR_CURSOR, 1ull);
                    }
                    write_hit(O, idx, seg_global, k, (uint32_t)j, xr, yr, cx, cy, (float)o.lambda,
                              (float)o.weight, tj, key);
                }
            }
        }
    }
    return nh;
}

// Candidate test of the soft-yield adjoint: does the arrival line pass
// within R_j + W of some telescope centre?  The same search as hit_test with
// every radius widened by W.
template <class T, class P>
__device__ __forceinline__ bool soft_candidate(const RayOut<T, P> &o, const DevAtm &A, const DevTel &Tl, float W,
                                               const uint8_t *clr)
{
    if (o.status != 0) return false;
    float Xf = p_f(o.X), Yf = p_f(o.Y);
    float cz = (float)o.cz, cx = (float)o.cx, cy = (float)o.cy;
    if (!(finite_f(Xf) && finite_f(Yf) && cz < 0.0f)) return false;
    float acz = fabsf(cz);
    float dzmax = fmaxf(fabsf(Tl.zmax - A.h_obs), fabsf(Tl.zmin - A.h_obs));
    float rs = (Tl.Rmax + W + dzmax * sqrtf(fmaxf(0.0f, 1.0f - acz * acz))) * rcp_approx(fmaxf(acz, 1e-6f)) + 1e-3f;
    if (Xf + rs < Tl.xmin || Xf - rs > Tl.xmax || Yf + rs < Tl.ymin || Yf - rs > Tl.ymax) return false;
    if (clr) {
        float fx = (Xf - Tl.cx0) * Tl.inv_cgs, fy = (Yf - Tl.cy0) * Tl.inv_cgs;
        if (fx >= 0.0f && fy >= 0.0f && fx < (float)Tl.cnx && fy < (float)Tl.cny) {
            int ci = (int)fy * Tl.cnx + (int)fx;
            if (rs < (float)clr[ci] * kClrQuantum) return false;
        }
    }
    int ix0 = max(0, (int)floorf((Xf - rs - Tl.gx0) * Tl.inv_gs));
    int ix1 = min(Tl.nx - 1, (int)floorf((Xf + rs - Tl.gx0) * Tl.inv_gs));
    int iy0 = max(0, (int)floorf((Yf - rs - Tl.gy0) * Tl.inv_gs));
    int iy1 = min(Tl.ny - 1, (int)floorf((Yf + rs - Tl.gy0) * Tl.inv_gs));
    for (int iy = iy0; iy <= iy1; ++iy)
        for (int ix = ix0; ix <= ix1; ++ix) {
            int cell = iy * Tl.nx + ix;
            int b = __ldg(Tl.cell_start + cell), e = __ldg(Tl.cell_start + cell + 1);
            for (int q = b; q < e; ++q) {
                float4 tp = __ldg(Tl.tel + __ldg(Tl.cell_tel + q));
                float sj = Num<float>::div(tp.z - A.h_obs, cz);
                float xr = p_f(o.X - (T)tp.x) + sj * cx;
                float yr = p_f(o.Y - (T)tp.y) + sj * cy;
                float wd = xr * cx + yr * cy;
                float d2 = fmaxf(xr * xr + yr * yr - wd * wd, 0.0f);
                float rw = tp.w + W;
                if (d2 < rw * rw) return true;
            }
        }
    return false;
}

}  // namespace clight
