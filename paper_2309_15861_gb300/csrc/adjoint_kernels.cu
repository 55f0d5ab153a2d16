// adjoint_kernels.cu -- gradients of the arrival positions and times of the
// hits, and of the soft-edged per-telescope yield, with respect to the
// atmosphere's layer scale heights c_i, its refractivity coefficient K and
// the extinction-length scale L0 (b_i, the layer edges and the random
// numbers held fixed; bunch counts frozen at the nominal parameters).
//
// Every ray is recomputed from its Philox counter; nothing is stored between
// the forward call and this one.  For each ray the primal is the forward's
// own computation (ray.cuh, FP32 pairs where the forward uses them), so the
// soft aperture sees exactly the forward's impact parameters.  The
// derivatives follow the same formulas in binary32 dual numbers carrying one
// tangent per parameter (n_layers + 2 of them): with so few parameters the
// tangent sweep costs about one extra ray in dual arithmetic and needs no
// tape.  Per-ray contributions, contracted with the upstream gradients, are
// summed per block in binary64 and then over blocks in a fixed order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "ray.cuh"

namespace clight {

// ------------------------------------------------------------------ duals
template <int NP> struct Dual {
    float v;
    float d[NP];
};

template <int NP> __device__ __forceinline__ Dual<NP> dc(float v)
{
    Dual<NP> r;
    r.v = v;
#pragma unroll
    for (int i = 0; i < NP; ++i) r.d[i] = 0.0f;
    return r;
}
template <int NP> __device__ __forceinline__ Dual<NP> operator+(const Dual<NP> &a, const Dual<NP> &b)
{
    Dual<NP> r;
    r.v = a.v + b.v;
#pragma unroll
    for (int i = 0; i < NP; ++i) r.d[i] = a.d[i] + b.d[i];
    return r;
}
template <int NP> __device__ __forceinline__ Dual<NP> operator-(const Dual<NP> &a, const Dual<NP> &b)
{
    Dual<NP> r;
    r.v = a.v - b.v;
#pragma unroll
    for (int i = 0; i < NP; ++i) r.d[i] = a.d[i] - b.d[i];
    return r;
}
template <int NP> __device__ __forceinline__ Dual<NP> operator-(const Dual<NP> &a)
{
    Dual<NP> r;
    r.v = -a.v;
#pragma unroll
    for (int i = 0; i < NP; ++i) r.d[i] = -a.d[i];
    return r;
}
template <int NP> __device__ __forceinline__ Dual<NP> operator+(const Dual<NP> &a, float b)
{
    Dual<NP> r = a;
    r.v = a.v + b;
    return r;
}
template <int NP> __device__ __forceinline__ Dual<NP> operator+(float b, const Dual<NP> &a) { return a + b; }
template <int NP> __device__ __forceinline__ Dual<NP> operator-(const Dual<NP> &a, float b) { return a + (-b); }
template <int NP> __device__ __forceinline__ Dual<NP> operator-(float b, const Dual<NP> &a) { return (-a) + b; }
template <int NP> __device__ __forceinline__ Dual<NP> operator*(const Dual<NP> &a, const Dual<NP> &b)
{
    Dual<NP> r;
    r.v = a.v * b.v;
#pragma unroll
    for (int i = 0; i < NP; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
    return r;
}
template <int NP> __device__ __forceinline__ Dual<NP> operator*(const Dual<NP> &a, float b)
{
    Dual<NP> r;
    r.v = a.v * b;
#pragma unroll
    for (int i = 0; i < NP; ++i) r.d[i] = a.d[i] * b;
    return r;
}
template <int NP> __device__ __forceinline__ Dual<NP> operator*(float b, const Dual<NP> &a) { return a * b; }
template <int NP> __device__ __forceinline__ Dual<NP> operator/(const Dual<NP> &a, const Dual<NP> &b)
{
    Dual<NP> r;
    float ib = 1.0f / b.v;
    r.v = a.v * ib;
#pragma unroll
    for (int i = 0; i < NP; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
    return r;
}
template <int NP> __device__ __forceinline__ Dual<NP> operator/(const Dual<NP> &a, float b) { return a * (1.0f / b); }
template <int NP> __device__ __forceinline__ Dual<NP> operator/(float a, const Dual<NP> &b) { return dc<NP>(a) / b; }
template <int NP> __device__ __forceinline__ Dual<NP> dsqrt(const Dual<NP> &a)
{
    Dual<NP> r;
    r.v = sqrtf(fmaxf(a.v, 0.0f));
    float h = r.v > 0.0f ? 0.5f / r.v : 0.0f;
#pragma unroll
    for (int i = 0; i < NP; ++i) r.d[i] = a.d[i] * h;
    return r;
}
template <int NP> __device__ __forceinline__ Dual<NP> dexp(const Dual<NP> &a)
{
    Dual<NP> r;
    r.v = expf(a.v);
#pragma unroll
    for (int i = 0; i < NP; ++i) r.d[i] = a.d[i] * r.v;
    return r;
}
template <int NP> __device__ __forceinline__ Dual<NP> with_value(Dual<NP> a, float v)
{
    a.v = v;
    return a;
}

// Parameters of the adjoint call.
struct AdjPar {
    float soft_s, soft_w;      // aperture softness and cut, m
    float K, L0;               // nominal refractivity coefficient and extinction length
    int n_layers;              // tangents 0..n_layers-1: c_i; n_layers: K; n_layers+1: L0
};

// delta = K b_i/(100 c_i) e^{-h/c_i} and rho/rho_ref at a fixed altitude:
// d/dc_i = value (h/c_i^2 - 1/c_i), d delta/dK = delta / K.
template <int NP>
__device__ __forceinline__ void atm_d(const DevAtm &A, const AdjPar &J, float h, Dual<NP> &dl, Dual<NP> &rr)
{
    dl = dc<NP>(0.0f);
    rr = dc<NP>(0.0f);
    if (h >= A.h_top) return;
    int i = 0;
#pragma unroll
    for (int j = 1; j < kMaxLayers; ++j)
        if (j < A.n_layers && h >= A.h_lo[j]) i = j;
    float ex = exp2f(h * A.nl2c[i]);
    float inv_c = -A.nl2c[i] * 0.6931471805599453f;          // 1/c_i
    float fc = inv_c * (h * inv_c - 1.0f);
    dl.v = A.kb[i] * ex;
    rr.v = A.rb[i] * ex;
    if (i < NP) {
        dl.d[i] = dl.v * fc;
        rr.d[i] = rr.v * fc;
    }
    if (J.n_layers < NP && J.K > 0.0f) dl.d[J.n_layers] = dl.v / J.K;
}

// the same at a quadrature node of cell c (the node lies in the cell's layer)
template <int NP>
__device__ __forceinline__ void atm_cell_d(const DevAtm &A, const AdjPar &J, int c, float h, Dual<NP> &dl,
                                           Dual<NP> &rr)
{
    const DevCell &C = A.cells[c];
    int i = (int)C.pad0;
    float ex = ex2_approx(h * C.nl2c);
    float inv_c = -C.nl2c * 0.6931471805599453f;
    float fc = inv_c * (h * inv_c - 1.0f);
    dl = dc<NP>(C.kb * ex);
    rr = dc<NP>(C.rb * ex);
    if (i < NP) {
        dl.d[i] = dl.v * fc;
        rr.d[i] = rr.v * fc;
    }
    if (J.n_layers < NP && J.K > 0.0f) dl.d[J.n_layers] = dl.v / J.K;
}

template <int NP> struct TanOut {
    Dual<NP> X, Y, t, cx, cy, cz, weight;
    Dual<NP> n_obs;
};

// Tangents of one ray, following trace_ray's formulas in binary32 duals.
template <int NP, bool SPH, bool REFR>
__device__ void tangent_ray(const Seg<float, df> &g, const clight_segment &s, int64_t seg_global, uint32_t k,
                            const DevAtm &A, const DevPar &Pp, const AdjPar &J, TanOut<NP> &T)
{
    using D = Dual<NP>;
    // ---- the step: delta at its midpoint drives theta_c and the yield
    D dmid, rmid;
    atm_d<NP>(A, J, g.h_mid, dmid, rmid);
    float eps = s.eps;
    D g1 = dmid * (1.0f - eps) - eps;                       // beta n - 1
    // its value from the step set-up (refractivity in FP32 pairs near the
    // threshold, where binary32 loses kappa/2 of its digits): the tangent of
    // sin(theta_c) goes like 1 / sqrt(beta n - 1)
    if (g.n_c > 0 && g.kappa > 0.0f) g1 = with_value(g1, g.kappa / (1.0f - g.kappa));
    D bn = g1 + 1.0f;
    D sin2 = g1 * (g1 + 2.0f) / (bn * bn);
    D sin_tc = dsqrt(sin2);
    D kappa = g1 / bn;
    float z2 = (float)s.charge * (float)s.charge;
    D Nc = sin2 * (Pp.band * z2 * s.L);
    // ---- the photon
    uint32_t proc = k < g.n_c ? 0u : 1u;
    uint32_t kk = proc ? k - g.n_c : k;
    uint4 x = philox4x32_10(make_uint4((uint32_t)(uint64_t)seg_global, (uint32_t)((uint64_t)seg_global >> 32), kk, proc),
                            Pp.seed, Pp.stream);
    float u0 = u01<float>(x.x), u1 = u01<float>(x.y), u2 = u01<float>(x.z), u3 = u01<float>(x.w);
    D dgx, dgy, dgz, w;
    float lam;
    if (proc == 0) {
        lam = 1.0f / (Pp.il1 - u0 * Pp.dil);
        float sc, cc;
        sincospif(2.0f * u2, &sc, &cc);
        dgx = (1.0f - kappa) * g.dx + sin_tc * (cc * g.e1x + sc * g.e2x);
        dgy = (1.0f - kappa) * g.dy + sin_tc * (cc * g.e1y + sc * g.e2y);
        dgz = (1.0f - kappa) * g.dz + sin_tc * (cc * g.e1z + sc * g.e2z);
        w = Nc / (float)g.n_c;
    } else {
        lam = Pp.fl1 + u0 * Pp.fdl;
        float sp, cp;
        sincospif(2.0f * u2, &sp, &cp);
        float fx, fy, fz;
        if (g.bomc > 0.0f) {
            cone_direction<float>(g.bux, g.buy, g.buz, u3 * g.bomc, sp, cp, fx, fy, fz);
        } else {
            fz = 2.0f * u3 - 1.0f;
            float sz = sqrtf((1.0f - fz) * (1.0f + fz));
            fx = sz * cp;
            fy = sz * sp;
        }
        // the emission geometry does not depend on the atmosphere
        dgx = dc<NP>(fx);
        dgy = dc<NP>(fy);
        dgz = dc<NP>(fz);
        w = dc<NP>(g.w_f);
    }
    float ell = u1 * g.L;
    float xe = p_f(g.x0 + ell * (g.dx + g.lx)), ye = p_f(g.y0 + ell * (g.dy + g.ly));
    float ze = p_f(g.z0 + ell * (g.dz + g.lz));
    const float RE = A.R_E, h_obs = A.h_obs;
    float he = altitude<float, SPH>(A, xe, ye, ze);
    D de, dummy;
    atm_d<NP>(A, J, he, de, dummy);
    D dob, rob;
    atm_d<NP>(A, J, h_obs, dob, rob);
    D ne = de + 1.0f, nob = dob + 1.0f;
    // ---- vacuum line and ray constants
    D s_v, pv2, bf2, b, so;
    if (SPH) {
        float Rz = ze + RE;
        b = -(dgx * xe + dgy * ye + dgz * Rz);
        float C = xe * xe + ye * ye + (ze - h_obs) * (ze + h_obs + 2.0f * RE);
        D xx = C / (b * b);
        D om = 1.0f - xx;
        so = dsqrt(om);
        D op = so + 1.0f;
        D gq = xx / (op * op * 2.0f);
        s_v = (C / b) * (gq + 0.5f);
        D c1 = dgy * Rz - dgz * ye, c2 = dgz * xe - dgx * Rz, c3 = dgx * ye - dgy * xe;
        pv2 = c1 * c1 + c2 * c2 + c3 * c3;
        bf2 = b * b;
    } else {
        s_v = (ze - h_obs) / (-dgz);
        pv2 = dgx * dgx + dgy * dgy;
        b = -dgz;
        bf2 = b * b;
        so = dc<NP>(1.0f);
    }
    // ---- quadrature (same cells and nodes as the forward)
    D I0 = dc<NP>(0.0f), I1 = dc<NP>(0.0f), I2 = dc<NP>(0.0f);
    float hcap = he < A.h_top ? he : A.h_top;
    for (int c = 0; c < A.n_cells; ++c) {
        const DevCell &C = A.cells[c];
        if (!(hcap > C.lo)) break;
        float hi = hcap < C.hi ? hcap : C.hi;
        float mid = 0.5f * (C.lo + hi), half = 0.5f * (hi - C.lo);
#pragma unroll
        for (int gi = 0; gi < kGLNodes; ++gi) {
            float h = mid + half * A.gl_x[gi];
            float wg = A.gl_w[gi] * half;
            D dl, rr;
            atm_cell_d<NP>(A, J, c, h, dl, rr);
            float r = SPH ? RE + h : 1.0f;
            D qv = SPH ? bf2 + (h - he) * (2.0f * RE + h + he) : bf2;
            if (REFR) {
                D n = dl + 1.0f;
                D n2 = n * n;
                D gg = (dl - de) * (dl + de + 2.0f);
                D q = n2 * qv + gg * pv2;
                D sq = dsqrt(q), sqv = dsqrt(qv);
                D cm = 1.0f / (sq * sqv);
                D a = dl * (dl + 2.0f);
                I0 = I0 + (-r * wg) * gg * cm / (ne * sqv + sq);
                I1 = I1 + (r * wg) * (n2 * a * qv - gg * pv2) * cm / (n2 * sqv + sq);
                I2 = I2 + (r * wg) * rr * n / sq;
            } else {
                D rqv = 1.0f / dsqrt(qv);
                I1 = I1 + (r * wg) * dl * rqv;
                I2 = I2 + (r * wg) * rr * rqv;
            }
        }
    }
    // ---- landing, arrival direction, crossing of z = h_obs, time, weight
    D X, Y, dLx, dLy, dLz, chord;
    if (SPH) {
        const float r_obs = A.r_obs, ir = 1.0f / r_obs;
        D Pvx = xe + s_v * dgx, Pvy = ye + s_v * dgy, Pvz = ze + s_v * dgz;
        D RLx = Pvx, RLy = Pvy, RLz = Pvz + RE;
        D sqf = b * so;
        D Tx = r_obs * dgx + sqf * ir * RLx, Ty = r_obs * dgy + sqf * ir * RLy, Tz = r_obs * dgz + sqf * ir * RLz;
        D Rhx = RLx * ir, Rhy = RLy * ir, Rhz = RLz * ir;
        D PLx = Pvx, PLy = Pvy, PLz = Pvz;
        if (REFR) {
            D pv = dsqrt(pv2);
            D dphi = I0 * pv;
            D sfac = I0 * r_obs;
            D c2 = dphi * dphi * (0.5f * r_obs);
            PLx = Pvx + sfac * Tx - c2 * Rhx;
            PLy = Pvy + sfac * Ty - c2 * Rhy;
            PLz = Pvz + sfac * Tz - c2 * Rhz;
            D gL = (dob - de) * (dob + de + 2.0f);
            D qL = nob * nob * sqf * sqf + gL * pv2;
            D inr = 1.0f / (nob * r_obs);
            D cpsi = dsqrt(qL) * inr;
            D spsi = ne * pv * inr;
            D at = ne * inr - cpsi * I0;
            D ar = cpsi + spsi * dphi;
            dLx = at * Tx - ar * Rhx;
            dLy = at * Ty - ar * Rhy;
            dLz = at * Tz - ar * Rhz;
        } else {
            dLx = dgx; dLy = dgy; dLz = dgz;
        }
        // zeta = h_obs - PLz is millimetres: its value from the horizontal
        // distance of the landing point on the observation sphere, its
        // tangent from PLz
        float rho2 = PLx.v * PLx.v + PLy.v * PLy.v;
        float zeta_v = rho2 / (r_obs + sqrtf(fmaxf(r_obs * r_obs - rho2, 0.0f)));
        D zeta = with_value(-PLz, zeta_v);
        chord = zeta / dLz;
        X = PLx + chord * dLx;
        Y = PLy + chord * dLy;
    } else {
        X = xe + s_v * dgx;
        Y = ye + s_v * dgy;
        if (REFR) {
            X = X + I0 * dgx;
            Y = Y + I0 * dgy;
            D qL = nob * nob * bf2 + (dob - de) * (dob + de + 2.0f) * pv2;
            D f = ne / nob;
            dLx = f * dgx;
            dLy = f * dgy;
            dLz = -(dsqrt(qL) / nob);
        } else {
            dLx = dgx; dLy = dgy; dLz = dgz;
        }
        chord = dc<NP>(0.0f);
    }
    T.t = (s_v + I1 + nob * chord) * 3.3356409519815204f;
    T.X = X;
    T.Y = Y;
    T.cx = dLx; T.cy = dLy; T.cz = dLz;
    T.n_obs = nob;
    D weight = w;
    if (A.absorption) {
        float lr = A.lambda_ref / lam;
        float lr4 = lr * lr * lr * lr;
        D L0 = dc<NP>(J.L0);
        if (J.n_layers + 1 < NP) L0.d[J.n_layers + 1] = 1.0f;
        D tau = I2 * lr4 / L0;
        weight = w * dexp(-tau);
    }
    T.weight = weight;
}

// d(perp) and the crossing of z = z_j relative to telescope j, with
// tangents; the values come from the primal (precise) quantities.
template <int NP>
__device__ __forceinline__ void tel_dual(const TanOut<NP> &T, float4 tp, float h_obs, float xr_p, float yr_p,
                                         float cxp, float cyp, float czp, Dual<NP> &xr, Dual<NP> &yr,
                                         Dual<NP> &tj, Dual<NP> &dperp)
{
    float dzj = tp.z - h_obs;
    Dual<NP> sj = dzj / T.cz;
    xr = with_value(T.X - tp.x + sj * T.cx, xr_p);
    yr = with_value(T.Y - tp.y + sj * T.cy, yr_p);
    tj = T.t + T.n_obs * sj * 3.3356409519815204f;
    Dual<NP> cx = with_value(T.cx, cxp), cy = with_value(T.cy, cyp);
    Dual<NP> wd = xr * cx + yr * cy;
    Dual<NP> d2 = xr * xr + yr * yr - wd * wd;
    dperp = dsqrt(d2);
    (void)czp;
}

template <int NP>
__device__ __forceinline__ void block_partials(double *acc, double *out)
{
    __shared__ double red[NP][128];
    for (int p = 0; p < NP; ++p) red[p][threadIdx.x] = acc[p];
    __syncthreads();
    for (int o = 64; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int p = 0; p < NP; ++p) red[p][threadIdx.x] += red[p][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int p = 0; p < NP; ++p) out[(size_t)blockIdx.x * NP + p] = red[p][0];
}

// Hit outputs: sum over hits of gx dx_rel + gy dy_rel + gt dt.
template <int NP, bool SPH, bool REFR>
__global__ void __launch_bounds__(128, 4)
k_adjoint_hits(const clight_segment *__restrict__ segs, const clight_hit *__restrict__ hits, int64_t n_hits,
               const float *__restrict__ gx, const float *__restrict__ gy, const float *__restrict__ gt,
               const __grid_constant__ DevAtm A, const __grid_constant__ DevTel Tl, const __grid_constant__ DevPar Pp,
               const __grid_constant__ AdjPar J, double *__restrict__ partial)
{
    double acc[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) acc[p] = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_hits; i += (int64_t)gridDim.x * blockDim.x) {
        clight_hit h = hits[i];
        int64_t sl = h.seg - Pp.seg_base;
        clight_segment s = segs[sl];
        Seg<float, df> g;
        load_segment_f<SPH>(s, h.seg, A, Pp, g);
        if (g.bad) continue;
        RayOut<float, df> o;
        trace_ray<float, df, false, SPH, REFR>(g, h.seg, h.k, true, A, Pp, o);
        if (o.status != 0) continue;
        TanOut<NP> T;
        tangent_ray<NP, SPH, REFR>(g, s, h.seg, h.k, A, Pp, J, T);
        float4 tp = __ldg(Tl.tel + h.tel);
        Dual<NP> xr, yr, tj, dp;
        tel_dual<NP>(T, tp, A.h_obs, h.x_rel, h.y_rel, h.cx, h.cy, (float)o.cz, xr, yr, tj, dp);
        float a = gx ? gx[i] : 0.0f, b = gy ? gy[i] : 0.0f, c = gt ? gt[i] : 0.0f;
#pragma unroll
        for (int p = 0; p < NP; ++p) acc[p] += (double)(a * xr.d[p] + b * yr.d[p] + c * tj.d[p]);
    }
    block_partials<NP>(acc, partial);
}

// Soft yield Y_g = sum over rays with d_perp < R + W of weight sigma((R - d_perp)/s):
// its value (optional) and sum_g gY_g dY_g, over the candidate rays the
// forward kernel's candidate pass compacted (local segment << 32 | bunch),
// so that every lane of a warp carries a ray that needs its tangents.
template <int NP, bool SPH, bool REFR>
__global__ void __launch_bounds__(128, 4)
k_adjoint_soft(const clight_segment *__restrict__ segs, const unsigned long long *__restrict__ cand, int64_t n_cand,
               const double *__restrict__ gY, unsigned long long *__restrict__ yfix, const __grid_constant__ DevAtm A,
               const __grid_constant__ DevTel Tl, const __grid_constant__ DevPar Pp, const __grid_constant__ AdjPar J,
               double *__restrict__ partial)
{
    double acc[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) acc[p] = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_cand; i += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long ck = cand[i];
        int64_t si = (int64_t)(ck >> Pp.k_bits);
        uint32_t k = (uint32_t)(ck & ((1ull << Pp.k_bits) - 1ull));
        clight_segment s = segs[si];
        Seg<float, df> g;
        load_segment_f<SPH>(s, Pp.seg_base + si, A, Pp, g);
        if (g.bad || k >= g.n_c + g.n_f) continue;
        int64_t seg_global = Pp.seg_base + si;
        RayOut<float, df> o;
        trace_ray<float, df, false, SPH, REFR>(g, seg_global, k, true, A, Pp, o);
        if (o.status != 0) continue;
        float Xf = p_f(o.X), Yf = p_f(o.Y), cz = (float)o.cz, cx = (float)o.cx, cy = (float)o.cy;
        if (!(finite_f(Xf) && finite_f(Yf) && cz < 0.0f)) continue;
        float acz = fabsf(cz);
        float reach = Tl.Rmax + J.soft_w;
        float dzmax = fmaxf(fabsf(Tl.zmax - A.h_obs), fabsf(Tl.zmin - A.h_obs));
        float rs = (reach + dzmax * sqrtf(fmaxf(0.0f, 1.0f - acz * acz))) / fmaxf(acz, 1e-6f) + 1e-3f;
        bool have_t = false;
        TanOut<NP> T;
        int ix0 = max(0, (int)floorf((Xf - rs - Tl.gx0) * Tl.inv_gs));
        int ix1 = min(Tl.nx - 1, (int)floorf((Xf + rs - Tl.gx0) * Tl.inv_gs));
        int iy0 = max(0, (int)floorf((Yf - rs - Tl.gy0) * Tl.inv_gs));
        int iy1 = min(Tl.ny - 1, (int)floorf((Yf + rs - Tl.gy0) * Tl.inv_gs));
        for (int iy = iy0; iy <= iy1; ++iy)
            for (int ix = ix0; ix <= ix1; ++ix) {
                int cell = iy * Tl.nx + ix;
                int cb = __ldg(Tl.cell_start + cell), ce = __ldg(Tl.cell_start + cell + 1);
                for (int q = cb; q < ce; ++q) {
                    int j = __ldg(Tl.cell_tel + q);
                    float4 tp = __ldg(Tl.tel + j);
                    float sj = (tp.z - A.h_obs) / cz;
                    float xr = p_f(o.X - tp.x) + sj * cx;
                    float yr = p_f(o.Y - tp.y) + sj * cy;
                    float wd = xr * cx + yr * cy;
                    float d2 = fmaxf(xr * xr + yr * yr - wd * wd, 0.0f);
                    float dperp = sqrtf(d2);
                    if (!(dperp < tp.w + J.soft_w)) continue;
                    float u = (tp.w - dperp) / J.soft_s;
                    float sg = 1.0f / (1.0f + expf(-u));
                    int64_t grp = (int64_t)g.shower * Tl.n_tel + j;
                    float val = (float)o.weight * sg;
                    // integer units of 2^-24 photons: the sum has the same bits in any order
                    if (yfix) atomicAdd(yfix + grp, __float2ull_rn(val * 16777216.0f));
                    if (gY) {
                        if (!have_t) {
                            tangent_ray<NP, SPH, REFR>(g, s, seg_global, k, A, Pp, J, T);
                            have_t = true;
                        }
                        Dual<NP> dxr, dyr, dtj, ddp;
                        tel_dual<NP>(T, tp, A.h_obs, xr, yr, cx, cy, cz, dxr, dyr, dtj, ddp);
                        float dsg = sg * (1.0f - sg) / J.soft_s;      // d sigma / d(R - d_perp)
                        double gy = gY[grp];
#pragma unroll
                        for (int p = 0; p < NP; ++p)
                            acc[p] += gy * (double)(T.weight.d[p] * sg - (float)o.weight * dsg * ddp.d[p]);
                    }
                }
            }
    }
    block_partials<NP>(acc, partial);
}

// Fixed-order sum of the block partials of both kernels.
template <int NP>
__global__ void k_adjoint_final(const double *__restrict__ partial, int n_blocks, double *__restrict__ out)
{
    int p = threadIdx.x;
    if (p >= NP) return;
    double s = 0.0;
    for (int b = 0; b < n_blocks; ++b) s += partial[(size_t)b * NP + p];
    out[p] = s;
}

// The soft yield from its fixed-point accumulators.
__global__ void k_yield_out(const unsigned long long *__restrict__ yfix, int64_t n, double *__restrict__ yield)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        yield[i] = (double)yfix[i] * 5.9604644775390625e-08;
}

template <int NP, bool SPH, bool REFR>
static cudaError_t adjoint_np(const clight_segment *segs, const unsigned long long *cand, int64_t n_cand,
                              const clight_hit *hits, int64_t n_hits,
                              const float *gx, const float *gy, const float *gt, const double *gY,
                              unsigned long long *yfix, const DevAtm &A, const DevTel &T, const DevPar &P,
                              const AdjPar &J, double *partial, int blocks, double *d_out, cudaStream_t s)
{
    k_adjoint_hits<NP, SPH, REFR><<<blocks, 128, 0, s>>>(segs, hits, n_hits, gx, gy, gt, A, T, P, J, partial);
    k_adjoint_soft<NP, SPH, REFR><<<blocks, 128, 0, s>>>(segs, cand, n_cand, gY, yfix, A, T, P, J,
                                                         partial + (size_t)blocks * NP);
    k_adjoint_final<NP><<<1, 32, 0, s>>>(partial, 2 * blocks, d_out);
    return cudaGetLastError();
}

template <int NP>
static cudaError_t adjoint_geo(const clight_segment *segs, const unsigned long long *cand, int64_t n_cand,
                               const clight_hit *hits, int64_t n_hits,
                               const float *gx, const float *gy, const float *gt, const double *gY,
                               unsigned long long *yfix, const DevAtm &A, const DevTel &T, const DevPar &P,
                               const AdjPar &J, double *partial, int blocks, double *d_out, cudaStream_t s)
{
    if (A.spherical && A.refraction)
        return adjoint_np<NP, true, true>(segs, cand, n_cand, hits, n_hits, gx, gy, gt, gY, yfix, A, T, P, J, partial, blocks, d_out, s);
    if (A.spherical)
        return adjoint_np<NP, true, false>(segs, cand, n_cand, hits, n_hits, gx, gy, gt, gY, yfix, A, T, P, J, partial, blocks, d_out, s);
    if (A.refraction)
        return adjoint_np<NP, false, true>(segs, cand, n_cand, hits, n_hits, gx, gy, gt, gY, yfix, A, T, P, J, partial, blocks, d_out, s);
    return adjoint_np<NP, false, false>(segs, cand, n_cand, hits, n_hits, gx, gy, gt, gY, yfix, A, T, P, J, partial, blocks, d_out, s);
}

int adjoint_params(int n_layers) { return n_layers <= 1 ? 3 : (n_layers <= 5 ? 7 : 10); }

cudaError_t launch_adjoint(const clight_segment *segs, const unsigned long long *cand, int64_t n_cand,
                           const clight_hit *hits, int64_t n_hits,
                           const float *gx, const float *gy, const float *gt, const double *gY,
                           unsigned long long *yfix, double *yield, int64_t n_groups,
                           const DevAtm &A, const DevTel &T, const DevPar &P, float soft_s, float soft_w, float K,
                           float L0, double *partial, int blocks, double *d_out, cudaStream_t s)
{
    AdjPar J;
    J.soft_s = soft_s;
    J.soft_w = soft_w;
    J.K = K;
    J.L0 = L0;
    J.n_layers = A.n_layers;
    int np = adjoint_params(A.n_layers);
    cudaError_t e;
    if (np == 3) e = adjoint_geo<3>(segs, cand, n_cand, hits, n_hits, gx, gy, gt, gY, yfix, A, T, P, J, partial, blocks, d_out, s);
    else if (np == 7) e = adjoint_geo<7>(segs, cand, n_cand, hits, n_hits, gx, gy, gt, gY, yfix, A, T, P, J, partial, blocks, d_out, s);
    else e = adjoint_geo<10>(segs, cand, n_cand, hits, n_hits, gx, gy, gt, gY, yfix, A, T, P, J, partial, blocks, d_out, s);
    if (e != cudaSuccess) return e;
    if (yield && yfix && n_groups > 0) {
        k_yield_out<<<(unsigned)std::min<int64_t>((n_groups + 255) / 256, 1024), 256, 0, s>>>(yfix, n_groups, yield);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace clight
