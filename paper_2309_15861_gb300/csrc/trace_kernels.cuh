// trace_kernels.cuh -- the forward kernels on sm_103a: the fused persistent
// generation + propagation + hit kernel (FP32 with FP32-pair or binary64
// precise steps), the classification and deferred-ray kernels of the
// two-pass path, and the plain binary64 kernel.  The per-ray device code is
// in ray.cuh (paper sections cited there).  Their launchers live in
// trace_twopass.cu, trace_inplace.cu and trace_noalloc.cu (three
// translation units, compiled in parallel).
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "ray.cuh"

namespace clight {

// ------------------------------------------------------------------ fused kernel
// Shared-memory record of a warp's 32 segments, one field per row so that
// lanes reading one field of different segments hit different banks.
enum SegField {
    // what the first pass of the deferred path (skip_ray) and the bunch loop read
    F_X0H, F_Y0H, F_Z0H, F_DX, F_DY, F_DZ, F_E1X, F_E1Y, F_E1Z, F_E2X, F_E2Y, F_E2Z,
    F_SIN, F_KAP, F_L, F_NC, F_NF, F_SEGI, F_INCL,
    F_DTH, F_GMX,                         // dispersion: cone-angle spread, largest g(lambda) (first pass)
    F_DEFER_END,
    // the rest of what a ray traced in the fused kernel needs
    F_X0L = F_DEFER_END, F_Y0L, F_Z0L, F_T0H, F_T0L, F_A0H, F_A0L, F_C0H, F_C0L, F_LX, F_LY, F_LZ,
    F_IBC, F_WC, F_WF, F_SHOWER,
    F_BUX, F_BUY, F_BUZ, F_BOMC,          // beamed fluorescence (kernels with FEAT_EXT only)
    F_COUNT
};
__host__ __device__ constexpr int fields_of(bool ext, bool defer = false)
{
    return ext ? F_COUNT : (defer ? F_DEFER_END : F_BUX);
}

// Segment records of the warps, then (kernels without FEAT_EXT) the
// clearance map; with FEAT_EXT the records are larger and the map is read
// from global memory, so that both stay under 48 KB.
inline int seg_smem_bytes(int block, bool ext, bool defer)
{
    return (block / 32) * fields_of(ext, defer) * 32 * (int)sizeof(float);
}
inline int fused_smem_bytes_f(int block, const DevTel &T, bool ext, bool defer = false)
{
    // the deferred first pass without FEAT_EXT also stages the next group's records
    return seg_smem_bytes(block, ext, defer) + (!ext && T.clr ? T.clr_bytes : 0) +
           (defer && !ext ? (block / 32) * 2048 : 0);
}
inline int fused_smem_bytes(int block, const DevTel &T) { return fused_smem_bytes_f(block, T, true); }

__device__ __forceinline__ void put_df(float *S, int fh, int fl, int l, df v)
{
    S[fh * 32 + l] = v.hi;
    S[fl * 32 + l] = v.lo;
}
__device__ __forceinline__ df get_df(const float *S, int fh, int fl, int l) { return {S[fh * 32 + l], S[fl * 32 + l]}; }

// Bitonic sort of one 32-bit key per lane across the warp (ascending).
__device__ __forceinline__ uint32_t warp_sort_u32(uint32_t key, int lane)
{
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            uint32_t other = __shfl_xor_sync(FULL_MASK, key, j);
            bool up = (lane & k) == 0;
            bool lower = (lane & j) == 0;
            uint32_t mn = min(key, other), mx = max(key, other);
            key = (lower == up) ? mn : mx;
        }
    }
    return key;
}

// Asynchronous 16-byte global -> shared copies (L2 only), for the next
// group's step records while the current group is worked on.
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// The 32 records (2 KB, contiguous) of the group starting at s_first, in
// 16-byte pieces spread over the warp; records at or past n_segs are not read.
__device__ __forceinline__ void prefetch_group(float4 *stage, const clight_segment *segs, int64_t n_segs,
                                               int64_t s_first, int lane)
{
    if (s_first >= n_segs) return;
    const float4 *src = reinterpret_cast<const float4 *>(segs + s_first);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int c = lane + 32 * j;
        if (s_first + (c >> 2) < n_segs) cp_async16(stage + c, src + c);
    }
    cp_async_commit();
}
constexpr int kStageBytes = 32 * (int)sizeof(clight_segment);   // per warp

// One atomic per warp and counter (the warp's lanes reduced by shuffles).
__device__ __forceinline__ void flush_stats(const uint32_t (&vals)[ST_N], unsigned status_bits, const DevOut &O,
                                            int lane)
{
#pragma unroll
    for (int i = 0; i < ST_N; ++i) {
        if (i == ST_STATUS) continue;
        uint32_t v = vals[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
        if (lane == 0 && v) atomicAdd(O.ctr + CTR_STATS + i, (unsigned long long)v);
    }
    unsigned sb = status_bits;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sb |= __shfl_xor_sync(FULL_MASK, sb, o);
    if (lane == 0 && sb) atomicOr(O.ctr + CTR_STATS + ST_STATUS, (unsigned long long)sb);
}

// A warp's entries for the deferred-ray queue, held in registers: each lane
// keeps at most one (the last it queued), `occ` marks the lanes that hold
// one.  When a lane would queue a second, the warp flushes: one atomic on the
// queue counter reserves a slot for every held entry and the holders write
// them to consecutive slots (one coalesced store).  One counter that every
// warp bumped for every round with a deferred ray limited the first pass to
// the rate at which one L2 slice serves atomics on one address; a flush
// carries ~7 entries on average.  Every member is called by all 32 lanes
// together.
struct WarpQueue {
    unsigned long long e = 0;
    unsigned occ = 0;                // warp-uniform

    __device__ __forceinline__ void flush(const DevOut &O, int lane, unsigned &status_bits)
    {
        const unsigned m = occ;
        unsigned long long b = 0;
        if (lane == 0) b = atomicAdd(O.ctr + CTR_DEFER, (unsigned long long)__popc(m));
        b = __shfl_sync(FULL_MASK, b, 0);
        if (m & (1u << lane)) {
            const unsigned long long qi = b + __popc(m & lanemask_lt());
            if ((int64_t)qi < O.defer_cap) O.defer[qi] = e;
            else status_bits |= 1u << kBitDeferFull;
        }
        occ = 0;
    }
    // Queues the entries of the lanes with p set.
    __device__ __forceinline__ void push(bool p, unsigned long long entry, const DevOut &O, int lane,
                                         unsigned &status_bits)
    {
        const unsigned m = __ballot_sync(FULL_MASK, p);
        if (!m) return;
        if (m & occ) flush(O, lane, status_bits);
        if (p) e = entry;
        occ |= m;
    }
    __device__ __forceinline__ void finish(const DevOut &O, int lane, unsigned &status_bits)
    {
        if (occ) flush(O, lane, status_bits);
    }
};

// Dispersion, first pass: a step's Cherenkov cone at the middle of its
// wavelength band (sine st, 1 - cos kap), the spread dth of the cone angle
// over the band (a bound on any photon's angle to that cone, widened) and
// the band's largest g(lambda).  (db, eps) come in the set-up's sin_tc and
// kappa.  A step without light in the band keeps st = kap = dth = 0, gmx = 1.
__device__ __forceinline__ void disp_band_cone(const DevAtm &A, const DevPar &Pp, const Seg<float, df> &g, float &st,
                                               float &kap, float &dth, float &gmx)
{
    st = 0.0f; kap = 0.0f; dth = 0.0f; gmx = 1.0f;
    float ulo, uhi;
    if (g.n_c > 0 && disp_band<float>(A, Pp, g.sin_tc, g.kappa, ulo, uhi)) {
        auto cone = [&](float u, float &s_, float &k_) {
            const float g1 = fmaxf(g.sin_tc * disp_gu<float>(A, u) - g.kappa, 0.0f);
            const float ib = 1.0f / (1.0f + g1);
            s_ = sqrtf(g1 * (2.0f + g1)) * ib;
            k_ = g1 * ib;
        };
        float s_lo, k_lo, s_hi, k_hi;
        cone(0.5f * (ulo + uhi), st, kap);
        cone(ulo, s_lo, k_lo);
        cone(uhi, s_hi, k_hi);
        dth = (asinf(fminf(s_hi, 1.0f)) - asinf(s_lo)) * 1.01f + 1.0e-6f;
        gmx = disp_gu<float>(A, uhi) * 1.000001f;
    }
}

// First pass of the deferred path: ray k of the step in record l, its
// direction and emission point in binary32 only, and what the full trace
// would conclude when that is already certain.  Returns 1 (escapes: points
// away from the Earth's centre by a wide margin), 2 (emitted below the
// observation level by more than 10 cm), 6 (reaches the observation level
// -- points down, emitted above it, cannot turn: the vacuum line meets the
// observation sphere at a zenith cosine above sqrt(2.1 delta_max) -- and
// clear_miss rules out every telescope), or 0 (trace it in full).  The
// direction and emission point are those of trace_ray without the low
// words of the pairs (millimetres at 10 km, inside the margins).
//
// With dispersion (DISP) a Cherenkov photon's cone angle follows its
// wavelength, drawn by rejection; the first pass takes the cone at the
// middle of the step's band instead, with derr >= the angle to any
// photon's true direction (the band's spread), and widens every margin by
// it; gl is then the band's largest g(lambda).
template <bool SPH, bool REFR, bool EXT, bool DISP>
__device__ __forceinline__ int skip_ray(const float *S, int l, uint32_t k, uint32_t n_c, int64_t seg_global,
                                        const DevAtm &A, const DevPar &Pp, const DevTel &Tl, const uint8_t *clr)
{
    const uint32_t proc = k < n_c ? 0u : 1u;
    const uint32_t kk = proc ? k - n_c : k;
    const uint4 x = philox4x32_10(make_uint4((uint32_t)(uint64_t)seg_global, (uint32_t)((uint64_t)seg_global >> 32),
                                             kk, proc),
                                  Pp.seed, Pp.stream);
    const float u1 = u01<float>(x.y), u2 = u01<float>(x.z), u3 = u01<float>(x.w);
    const float sdx = S[F_DX * 32 + l], sdy = S[F_DY * 32 + l], sdz = S[F_DZ * 32 + l];
    float dx, dy, dz;
    float derr = 0.0f, gl = 1.0f;
    if (DISP) {
        if (proc == 0) {
            derr = S[F_DTH * 32 + l];
            gl = S[F_GMX * 32 + l];
        } else {
            gl = disp_gu<float>(A, rcp_approx(Pp.fl1 + u01<float>(x.x) * Pp.fdl)) * 1.000001f;
        }
    }
    if (proc == 0) {
        float sc, cc;
        Num<float>::sincos2pi(u2, &sc, &cc);
        const float st = S[F_SIN * 32 + l], kap = S[F_KAP * 32 + l];
        dx = sdx + (-kap * sdx + st * (cc * S[F_E1X * 32 + l] + sc * S[F_E2X * 32 + l]));
        dy = sdy + (-kap * sdy + st * (cc * S[F_E1Y * 32 + l] + sc * S[F_E2Y * 32 + l]));
        dz = sdz + (-kap * sdz + st * (cc * S[F_E1Z * 32 + l] + sc * S[F_E2Z * 32 + l]));
    } else {
        float sp, cp;
        Num<float>::sincos2pi(u2, &sp, &cp);
        const float bomc = EXT ? S[F_BOMC * 32 + l] : 0.0f;
        if (EXT && bomc > 0.0f) {
            cone_direction<float>(S[F_BUX * 32 + l], S[F_BUY * 32 + l], S[F_BUZ * 32 + l], u3 * bomc, sp, cp, dx, dy,
                                  dz);
        } else {
            const float cz = 2.0f * u3 - 1.0f;
            const float sz = Num<float>::sqr((1.0f - cz) * (1.0f + cz));
            dx = sz * cp; dy = sz * sp; dz = cz;
        }
    }
    const float ell = u1 * S[F_L * 32 + l];
    const float xe = S[F_X0H * 32 + l] + ell * sdx;
    const float ye = S[F_Y0H * 32 + l] + ell * sdy;
    const float ze = S[F_Z0H * 32 + l] + ell * sdz;
    // the outward component (along the Earth radius; flat: d_z) decides escape
    const float Rz = ze + A.R_E;
    const float out = SPH ? dx * xe + dy * ye + dz * Rz : dz;
    const float mo = SPH ? (1.0e-3f + derr) * Rz : 1.0e-6f + derr;
    if (out > mo) return 1;
    if (!(out < -mo)) return 0;
    // altitude, cancellation-free (|r| + R_E in the denominator: the
    // approximate square root moves it by ~1e-7 relative)
    const float he = SPH ? (xe * xe + ye * ye + ze * (ze + 2.0f * A.R_E)) *
                               rcp_approx(sqrt_approx(xe * xe + ye * ye + Rz * Rz) + A.R_E)
                         : ze;
    if (he < A.h_obs - 0.1f) return 2;
    if (!(he > A.h_obs + 0.1f) || !(dz < -0.05f - derr)) return 0;
    float cos_obs = 0.0f;
    if (SPH) {
        // zenith sine at the landing point: p_v / r_obs, raised by the
        // direction's uncertainty (|R| derr / r_obs)
        const float c1 = dy * Rz - dz * ye, c2 = dz * xe - dx * Rz, c3 = dx * ye - dy * xe;
        float so = sqrt_approx(c1 * c1 + c2 * c2 + c3 * c3) * A.inv_r_obs;
        if (DISP) so += derr * (1.0f + (he - A.h_obs) * A.inv_r_obs) * 1.001f;
        const float co2 = 1.0f - so * so;
        if (!(so < 1.0f) || !(co2 > 2.1f * A.delta_max * gl + 2.6e-3f)) return 0;
        cos_obs = sqrt_approx(co2);
    }
    return clear_miss(xe, ye, ze, dx, dy, dz, he, cos_obs, gl, A, Tl, clr, SPH, REFR, 0.0f, derr) ? 6 : 0;
}

// DEFER (binary32 pairs): each ray only goes through skip_ray; the rays it
// cannot leave out are queued in O.defer and traced by k_trace_deferred in
// full warps, so that no warp integrates for one lane.  No launcher uses
// this form any more (k_classify is the first pass for every feature set);
// the in-place forms (DEFER = false) are unchanged by it.
// A ray that finds the queue full sets the kBitDeferFull status bit (the
// host then runs the call again).  Without the in-place path the kernel
// fits 4 CTAs of 256 threads per SM.
template <class P, bool SPH, bool REFR, bool NOALLOC = false, bool SOFT = false, int FEAT = FEAT_ALL,
          bool DEFER = false>
__global__ void __launch_bounds__(256, DEFER ? 4 : 3)
k_trace_fused(const clight_segment *__restrict__ segs, int64_t n_segs, const __grid_constant__ DevAtm A,
              const __grid_constant__ DevTel Tl, const __grid_constant__ DevPar Pp, const __grid_constant__ DevOut O)
{
    constexpr bool EXT = (FEAT & FEAT_EXT) != 0;
    constexpr int FC = fields_of(EXT, DEFER);
    extern __shared__ float smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float *S = smem + warp * (FC * 32);
    // the clearance map, staged once per CTA behind the segment records
    const uint8_t *clr = EXT ? Tl.clr : nullptr;
    if (!EXT && Tl.clr) {
        uint4 *dst = reinterpret_cast<uint4 *>(smem + (blockDim.x >> 5) * (FC * 32));
        const uint4 *src = reinterpret_cast<const uint4 *>(Tl.clr);
        for (int i = threadIdx.x; i < (Tl.clr_bytes >> 4); i += blockDim.x) dst[i] = __ldg(src + i);
        __syncthreads();
        clr = reinterpret_cast<const uint8_t *>(dst);
    }
    uint32_t c_rays = 0, c_esc = 0, c_under = 0, c_turn = 0, c_reach = 0, c_hits = 0, c_guard = 0, c_cells = 0;
    uint32_t c_cut = 0, c_skip = 0;
    unsigned status_bits = 0;
    WarpQueue dq;                    // deferred rays (DEFER)
    // the deferred first pass (without FEAT_EXT) loads each group's records
    // while the group before is worked on: the next group is claimed and its
    // records copied into the warp's stage (behind the map) asynchronously
    constexpr bool PREF = DEFER && !EXT;
    float4 *stage = nullptr;
    unsigned long long grp_next = 0;
    if (PREF) {
        stage = reinterpret_cast<float4 *>(reinterpret_cast<char *>(smem) + (blockDim.x >> 5) * (FC * 32) * 4 +
                                           (Tl.clr ? Tl.clr_bytes : 0) + warp * kStageBytes);
        if (lane == 0) grp_next = atomicAdd(O.ctr + CTR_WORK, 1ull);
        grp_next = __shfl_sync(FULL_MASK, grp_next, 0);
        prefetch_group(stage, segs, n_segs, (int64_t)grp_next * 32, lane);
    }
    for (;;) {
        unsigned long long grp = 0;
        if (PREF) {
            grp = grp_next;
            if (lane == 0) grp_next = atomicAdd(O.ctr + CTR_WORK, 1ull);
        } else {
            if (lane == 0) grp = atomicAdd(O.ctr + CTR_WORK, 1ull);
            grp = __shfl_sync(FULL_MASK, grp, 0);
        }
        int64_t s_first = (int64_t)grp * 32;
        if (s_first >= n_segs) break;
        int64_t si = s_first + lane;
        float4 w0 = make_float4(0.f, 0.f, 0.f, 0.f), w1 = w0, w2 = w0, w3 = w0;
        if (PREF) {
            cp_async_wait_all();
            __syncwarp();
            if (si < n_segs) {
                w0 = stage[lane * 4]; w1 = stage[lane * 4 + 1];
                w2 = stage[lane * 4 + 2]; w3 = stage[lane * 4 + 3];
            }
            __syncwarp();
            grp_next = __shfl_sync(FULL_MASK, grp_next, 0);
            prefetch_group(stage, segs, n_segs, (int64_t)grp_next * 32, lane);
        } else if (si < n_segs) {
            const float4 *src = reinterpret_cast<const float4 *>(segs + si);
            w0 = __ldg(src); w1 = __ldg(src + 1); w2 = __ldg(src + 2); w3 = __ldg(src + 3);
        }
        const clight_segment s = seg_from_words(w0, w1, w2, w3);
        // ---- per-segment set-up, one segment per lane
        Seg<float, df> g;
        uint32_t nb = 0;
        uint32_t key = 0xFFFFFFE0u | (uint32_t)lane;          // empty lanes sort last
        if (si < n_segs) {
            load_segment_f<SPH, EXT, (FEAT & FEAT_DISP) != 0>(s, Pp.seg_base + si, A, Pp, g);
            if (g.bad) status_bits |= 1u << g.bad;
            c_guard += g.guarded;
            c_cut += g.cut;
            nb = g.n_c + g.n_f;
            if (nb < g.n_c || nb > 0x7fffffffu) { status_bits |= 1u << CLIGHT_ERR_LIMIT; nb = 0; }
            // order the warp's segments by altitude (500 m bins), so that the
            // rays of one round need similar numbers of quadrature cells
            uint32_t bin = (uint32_t)fminf(fmaxf(g.h_mid * 2.0e-3f, 0.0f), 1.0e6f);
            key = (bin << 5) | (uint32_t)lane;
        } else {
            g.n_c = g.n_f = 0;
        }
        // (the deferred first pass integrates nothing: its steps keep their order)
        if (!DEFER) key = warp_sort_u32(key, lane);
        // the segment of source lane (key & 31) takes position `lane`; each
        // source lane learns its position through shared memory
        __syncwarp();
        S[F_INCL * 32 + (key & 31u)] = __uint_as_float((uint32_t)lane);
        __syncwarp();
        const int pos = (int)__float_as_uint(S[F_INCL * 32 + lane]);
        __syncwarp();
        // inclusive scan of the bunch counts in sorted order
        uint32_t incl = __shfl_sync(FULL_MASK, nb, (int)(key & 31u));
        uint32_t total;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t v = __shfl_up_sync(FULL_MASK, incl, o);
            if (lane >= o) incl += v;
        }
        total = __shfl_sync(FULL_MASK, incl, 31);
        if (si < n_segs) {
            S[F_X0H * 32 + pos] = g.x0.hi; S[F_Y0H * 32 + pos] = g.y0.hi; S[F_Z0H * 32 + pos] = g.z0.hi;
            S[F_DX * 32 + pos] = g.dx; S[F_DY * 32 + pos] = g.dy; S[F_DZ * 32 + pos] = g.dz;
            S[F_E1X * 32 + pos] = g.e1x; S[F_E1Y * 32 + pos] = g.e1y; S[F_E1Z * 32 + pos] = g.e1z;
            S[F_E2X * 32 + pos] = g.e2x; S[F_E2Y * 32 + pos] = g.e2y; S[F_E2Z * 32 + pos] = g.e2z;
            S[F_SIN * 32 + pos] = g.sin_tc; S[F_KAP * 32 + pos] = g.kappa; S[F_L * 32 + pos] = g.L;
            if (DEFER && (FEAT & FEAT_DISP)) {
                // (db, eps) -> the cone at the middle of the band, the spread
                // of the cone angle over the band, the band's largest g
                float st, kap, dth, gmx;
                disp_band_cone(A, Pp, g, st, kap, dth, gmx);
                S[F_SIN * 32 + pos] = st; S[F_KAP * 32 + pos] = kap;
                S[F_DTH * 32 + pos] = dth; S[F_GMX * 32 + pos] = gmx;
            }
            S[F_NC * 32 + pos] = __uint_as_float(g.n_c);
            S[F_NF * 32 + pos] = __uint_as_float(g.n_f);
            S[F_SEGI * 32 + pos] = __uint_as_float((uint32_t)lane);
            if (!DEFER) {
                S[F_X0L * 32 + pos] = g.x0.lo; S[F_Y0L * 32 + pos] = g.y0.lo; S[F_Z0L * 32 + pos] = g.z0.lo;
                put_df(S, F_T0H, F_T0L, pos, g.t0);
                put_df(S, F_A0H, F_A0L, pos, g.A0);
                put_df(S, F_C0H, F_C0L, pos, g.C0);
                S[F_LX * 32 + pos] = g.lx; S[F_LY * 32 + pos] = g.ly; S[F_LZ * 32 + pos] = g.lz;
                S[F_IBC * 32 + pos] = g.inv_bc;
                S[F_WC * 32 + pos] = g.w_c; S[F_WF * 32 + pos] = g.w_f;
                S[F_SHOWER * 32 + pos] = __uint_as_float(g.shower);
            }
            if (EXT) {
                S[F_BUX * 32 + pos] = g.bux; S[F_BUY * 32 + pos] = g.buy; S[F_BUZ * 32 + pos] = g.buz;
                S[F_BOMC * 32 + pos] = g.bomc;
            }
        } else {
            S[F_NC * 32 + pos] = __uint_as_float(0u);
            S[F_NF * 32 + pos] = __uint_as_float(0u);
        }
        S[F_INCL * 32 + lane] = __uint_as_float(incl);
        __syncwarp();
        // ---- flattened bunch loop: lane j takes ray j of the warp's segments
        uint32_t rounds = (total + 31) / 32;
        for (uint32_t r = 0; r < rounds; ++r) {
            uint32_t j = r * 32 + lane;
            bool active = j < total;
            uint32_t jj = active ? j : total - 1;
            int l = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1)
                if (__float_as_uint(S[F_INCL * 32 + l + step - 1]) <= jj) l += step;
            uint32_t nc_l = __float_as_uint(S[F_NC * 32 + l]);
            uint32_t nf_l = __float_as_uint(S[F_NF * 32 + l]);
            uint32_t excl = __float_as_uint(S[F_INCL * 32 + l]) - (nc_l + nf_l);
            uint32_t k = jj - excl;
            int64_t seg_local = s_first + (int64_t)__float_as_uint(S[F_SEGI * 32 + l]);
            int64_t seg_global = Pp.seg_base + seg_local;
            if (DEFER) {
                const int cls =
                    active ? skip_ray<SPH, REFR, EXT, (FEAT & FEAT_DISP) != 0>(S, l, k, nc_l, seg_global, A, Pp, Tl, clr)
                           : -1;
                const bool push = cls == 0;
                if (active) {
                    ++c_rays;
                    c_esc += cls == 1; c_under += cls == 2;
                    c_reach += cls == 6; c_skip += cls == 6;
                }
                dq.push(push, ((unsigned long long)seg_local << 32) | (unsigned long long)k, O, lane, status_bits);
                continue;
            }
            const bool act = active;
            Seg<float, df> q;
            q.x0 = get_df(S, F_X0H, F_X0L, l);
            q.y0 = get_df(S, F_Y0H, F_Y0L, l);
            q.z0 = get_df(S, F_Z0H, F_Z0L, l);
            q.t0 = get_df(S, F_T0H, F_T0L, l);
            q.A0 = get_df(S, F_A0H, F_A0L, l);
            q.C0 = get_df(S, F_C0H, F_C0L, l);
            q.rz0 = SPH ? q.z0 + df{A.re_hi, A.re_lo} : q.z0;  // fluorescence photons only
            q.dx = S[F_DX * 32 + l]; q.dy = S[F_DY * 32 + l]; q.dz = S[F_DZ * 32 + l];
            q.lx = S[F_LX * 32 + l]; q.ly = S[F_LY * 32 + l]; q.lz = S[F_LZ * 32 + l];
            q.e1x = S[F_E1X * 32 + l]; q.e1y = S[F_E1Y * 32 + l]; q.e1z = S[F_E1Z * 32 + l];
            q.e2x = S[F_E2X * 32 + l]; q.e2y = S[F_E2Y * 32 + l]; q.e2z = S[F_E2Z * 32 + l];
            q.sin_tc = S[F_SIN * 32 + l]; q.kappa = S[F_KAP * 32 + l];
            q.L = S[F_L * 32 + l]; q.inv_bc = S[F_IBC * 32 + l];
            q.w_c = S[F_WC * 32 + l]; q.w_f = S[F_WF * 32 + l];
            q.n_c = nc_l; q.n_f = nf_l;
            q.shower = __float_as_uint(S[F_SHOWER * 32 + l]);
            if (EXT) {
                q.bux = S[F_BUX * 32 + l]; q.buy = S[F_BUY * 32 + l]; q.buz = S[F_BUZ * 32 + l];
                q.bomc = S[F_BOMC * 32 + l];
            } else {
                q.bux = q.buy = q.buz = q.bomc = 0.0f;
            }
            int nh = 0;
            if (std::is_same<P, double>::value) {   // binary64 for the precise steps
                Seg<float, double> qd;
                widen_seg(q, qd);
                RayOut<float, double> o;
                trace_ray<float, double, true, SPH, REFR, FEAT>(qd, seg_global, k, active, A, Pp, o);
                nh = hit_test<float, double, true, NOALLOC>(o, Pp.key_off + seg_local, seg_global, k, q.shower, A, Tl, Pp, O, status_bits, clr);
                if (active) {
                    ++c_rays;
                    c_esc += o.status == 1; c_under += o.status == 2; c_turn += o.status == 3;
                    c_reach += o.status == 0 || o.status >= 5;
                    c_cells += o.status == 0 ? o.cells : 0;
                }
            } else if (SOFT) {
                // candidate pass of the soft-yield adjoint: compact the rays
                // near a telescope into O.keys
                // (rays that provably pass farther than R + W from every centre skip the quadrature)
                RayOut<float, df> o;
                trace_ray<float, df, true, SPH, REFR, FEAT, true>(q, seg_global, k, active, A, Pp, o, &Tl, clr, O.soft_w);
                bool cand = active && soft_candidate<float, df>(o, A, Tl, O.soft_w, clr);
                // key: local step << k_bits | bunch (sorted before the adjoint)
                if (cand && Pp.k_bits < 32 && k >= (1u << Pp.k_bits)) {
                    status_bits |= 1u << CLIGHT_ERR_LIMIT;
                    cand = false;
                }
                unsigned m = __ballot_sync(FULL_MASK, cand);
                if (m) {
                    unsigned long long base = 0;
                    if (lane == 0) base = atomicAdd(O.ctr + CTR_CURSOR, (unsigned long long)__popc(m));
                    base = __shfl_sync(FULL_MASK, base, 0);
                    unsigned long long idx = base + __popc(m & lanemask_lt());
                    if (cand && (int64_t)idx < O.capacity)
                        O.keys[idx] = ((unsigned long long)seg_local << Pp.k_bits) | (unsigned long long)k;
                }
                nh = cand ? 1 : 0;
                if (active) {
                    ++c_rays;
                    c_reach += o.status == 0 || o.status >= 5;
                    c_cells += o.status == 0 ? o.cells : 0;
                }
            } else {
                RayOut<float, df> o;
                trace_ray<float, df, true, SPH, REFR, FEAT, !DEFER>(q, seg_global, k, act, A, Pp, o, &Tl, clr);
                nh = hit_test<float, df, true, NOALLOC>(o, Pp.key_off + seg_local, seg_global, k, q.shower, A, Tl, Pp, O, status_bits, clr);
                if (act) {
                    ++c_rays;
                    c_esc += o.status == 1; c_under += o.status == 2; c_turn += o.status == 3;
                    c_reach += o.status == 0 || o.status >= 5;
                    c_skip += o.status == 6;
                    c_cells += o.status == 0 ? o.cells : 0;
                }
            }
            c_hits += nh;
        }
        __syncwarp();
    }
    if (DEFER) dq.finish(O, lane, status_bits);
    // ---- statistics: one atomic per warp and counter
    const uint32_t vals[ST_N] = {c_rays, c_esc, c_under, c_turn, c_reach, c_hits, c_guard, 0u, c_cells, c_cut, c_skip, 0u, 0u};
    flush_stats(vals, status_bits, O, lane);
}

// ------------------------------------------------------------------ classification pass
// First pass of the two-pass path for the default feature set (no angular
// cut, beaming or dispersion; either propagator).  It decides, for every
// ray, what the full trace would conclude wherever that is certain -- 1
// escapes, 2 emitted below the observation level, 6 reaches it and lands
// provably clear of every telescope -- and queues the rest for
// k_trace_deferred, as k_trace_fused<..., DEFER> does, with less work per
// ray:
//  - the Cherenkov bunches of a warp's 32 steps come first and the
//    fluorescence bunches after them, so that a round of 32 rays rarely
//    mixes the two code paths;
//  - each round finds the step of every lane from one OR-reduction over the
//    warp of the steps' start positions (no search per ray), and the step
//    records are read with 128-bit shared loads;
//  - for a Cherenkov step every photon direction lies on the cone of half-
//    angle theta_c about the flight direction d, so the quantities the
//    per-ray test bounds -- the smallest landing zenith cosine mu, the
//    refraction displacement coefficient and the hit search radius -- are
//    bounded once per step by their worst case over the cone (the landing
//    zenith angle is at most the emission zenith angle of d plus theta_c,
//    widened by the step length over the Earth radius).  Each bound is at
//    least the per-ray value clear_miss would use, so a ray skipped here
//    would be skipped by the per-ray test too.  A step whose cone comes
//    within about 87 degrees of the horizon (or turns rays before the
//    observation level) has no such bound and its rays take the per-ray
//    test;
//  - the emission altitude is linear along the step (h_mid + (l - L/2) dh/dl:
//    off by at most L^2 / (2 R_E), micrometres, against a 10 cm margin).
struct alignas(16) ClsRec {
    float x0, y0, z0, L;        // start of the step (binary32), length
    float dx, dy, dz, h_mid;    // unit direction, midpoint altitude
    float ax, ay, az, hd;       // cos(theta_c) d, dh/dl along the step
    float b1x, b1y, b1z, rsb;   // sin(theta_c) M_Rod x, search radius without the refraction term
    float b2x, b2y, b2z, cB;    // sin(theta_c) M_Rod y, refraction term per metre of height
    uint32_t nc;                // Cherenkov bunches
    float derr;                 // bound on a Cherenkov ray's direction error (rad)
    float gl;                   // largest g(lambda) of its refractivity (dispersion; else 1)
    float pad;
};
static_assert(sizeof(ClsRec) == 96, "ClsRec layout");
constexpr int kClsVmax = 64;                     // virtual steps per warp: 32 Cherenkov + 32 fluorescence
constexpr int kClsWarpBytes = 32 * (int)sizeof(ClsRec) + kClsVmax * 8;
constexpr uint32_t kVGated = 1u << 6;            // virtual-step flag: the step's Cherenkov bounds hold
// Bound on the error of (cos c, sin c) from the MUFU sine and cosine: each
// within 2^-21.41 = 3.6e-7 of the value at its argument (the vector moves by
// at most 5.1e-7), and the binary32 argument 2 pi (u - 1/2) within
// 2 pi |u - 1/2| 2^-23 <= 3.8e-7 of the exact angle: 8.9e-7, rounded up.
constexpr float kAzErr = 1.0e-6f;

constexpr int kClsBeamBytes = 32 * 16;         // EXT: each step's fluorescence beam cone (axis, 1 - cos)
inline int cls_smem_bytes(int block, const DevTel &, bool ext = false)
{
    return (block / 32) * (kClsWarpBytes + (ext ? kClsBeamBytes : 0) + kStageBytes);
}

// Per-ray part of the classification of a Cherenkov ray of a gated step:
// the per-step bounds stand in for the ray's own.
// The step's cB carries the direction error of its rays as well.
template <bool SPH>
__device__ __forceinline__ int classify_cherenkov_gated(const ClsRec &R, float ell, float dgx, float dgy, float dgz,
                                                        const DevAtm &A, const DevTel &Tl, const uint8_t *clr)
{
    // escape is impossible and every ray reaches the observation level (gate)
    const float he = R.h_mid + (ell - 0.5f * R.L) * R.hd;
    if (he < A.h_obs - 0.1f) return 2;
    if (!(he > A.h_obs + 0.1f)) return 0;
    const float xe = R.x0 + ell * R.dx, ye = R.y0 + ell * R.dy, ze = R.z0 + ell * R.dz;
    const float tp = (ze - A.h_obs) * rcp_approx(-dgz);
    const float Xv = xe + tp * dgx, Yv = ye + tp * dgy;
    const float zeta = SPH ? (Xv * Xv + Yv * Yv) * A.inv_r_obs : 0.0f;
    const float rs = R.rsb + R.cB * ((he - A.h_obs) + zeta);
    if (Xv + rs < Tl.xmin || Xv - rs > Tl.xmax || Yv + rs < Tl.ymin || Yv - rs > Tl.ymax) return 6;
    return clr_clear<true>(Tl, clr, Xv, Yv, rs) ? 6 : 0;
}

// The per-ray test (ray direction d, emission at l along the step), as in
// skip_ray: for fluorescence photons and the Cherenkov photons of steps
// without per-step bounds.  derr: a bound on the angle between (dx, dy, dz)
// and the direction the full trace forms (the azimuth's error here; under
// dispersion (DISP) the cone-angle spread over the band as well, which also
// widens the escape, steepness and landing-angle tests, as in skip_ray).  gl:
// the largest g(lambda) of the photon's refractivity (1 without dispersion).
template <bool SPH, bool REFR, bool DISP = false>
__device__ __forceinline__ int classify_ray(const ClsRec &R, float ell, float dx, float dy, float dz, float derr,
                                            float gl, const DevAtm &A, const DevTel &Tl, const uint8_t *clr)
{
    const float xe = R.x0 + ell * R.dx, ye = R.y0 + ell * R.dy, ze = R.z0 + ell * R.dz;
    const float Rz = ze + A.R_E;
    const float out = SPH ? dx * xe + dy * ye + dz * Rz : dz;
    const float dm = DISP ? derr : 0.0f;
    const float mo = SPH ? (1.0e-3f + dm) * Rz : 1.0e-6f + dm;
    if (out > mo) return 1;
    if (!(out < -mo)) return 0;
    const float he = R.h_mid + (ell - 0.5f * R.L) * R.hd;
    if (he < A.h_obs - 0.1f) return 2;
    if (!(he > A.h_obs + 0.1f) || !(dz < -0.05f - dm)) return 0;
    float cos_obs = 0.0f;
    if (SPH) {
        const float c1 = dy * Rz - dz * ye, c2 = dz * xe - dx * Rz, c3 = dx * ye - dy * xe;
        float so = sqrt_approx(c1 * c1 + c2 * c2 + c3 * c3) * A.inv_r_obs;
        if (DISP) so += dm * (1.0f + (he - A.h_obs) * A.inv_r_obs) * 1.001f;
        const float co2 = 1.0f - so * so;
        if (!(so < 1.0f) || !(co2 > 2.1f * A.delta_max * gl + 2.6e-3f)) return 0;
        cos_obs = sqrt_approx(co2);
    }
    return clear_miss<true>(xe, ye, ze, dx, dy, dz, he, cos_obs, gl, A, Tl, clr, SPH, REFR, 0.0f, derr) ? 6 : 0;
}

// Does every Cherenkov photon of a gated step land clear of the array?
// The photon directions are u(c) = ct d + st (cos c e1 + sin c e2); a ray
// from height dz above the plane z = h_obs crosses it at dz u_xy / (-u_z)
// from its emission point, and u_x / (-u_z) = (a0 + a . v) / (b0 + b . v)
// (v = (cos c, sin c)) ranges over the roots of
// (b0^2 - |b|^2) l^2 - 2 (a0 b0 - a . b) l + a0^2 - |a|^2 = 0 (the same for
// y).  The emission point moves linearly along the step, so the footprint
// of the whole step lies in the box spanned by its two ends.  The step's
// search radius (rsb + cB (height + zeta)) is taken at its largest over
// that box; the roots carry a rounding margin from the discriminant's
// binary32 error.  True when the box, widened by that radius, misses the
// array's bounding box (which holds every sphere) -- then every ray of the
// step would be skipped by classify_cherenkov_gated, and all are counted
// as skipped without being drawn.
__device__ __forceinline__ bool cone_lands_clear(const Seg<float, df> &g, const ClsRec &r, float ct, float st,
                                                 const DevAtm &A, const DevTel &Tl)
{
    const float dz0 = r.z0 - A.h_obs, dz1 = dz0 + r.L * g.dz;       // heights of both ends above the plane
    const float he_lo = r.h_mid - 0.5f * r.L * fabsf(r.hd), he_hi = r.h_mid + 0.5f * r.L * fabsf(r.hd);
    if (!(dz0 > 1.0f) || !(dz1 > 1.0f) || !(he_lo > A.h_obs + 0.2f)) return false;
    const float b0 = -ct * g.dz, b1 = -st * g.e1z, b2 = -st * g.e2z;
    const float A2 = b0 * b0 - (b1 * b1 + b2 * b2);                   // >= 0.05^2 (the gate)
    const float iA = rcp_approx(A2);
    auto roots = [&](float a0, float a1, float a2, float &lo, float &hi) {
        const float B1 = a0 * b0 - (a1 * b1 + a2 * b2);
        const float C0 = a0 * a0 - (a1 * a1 + a2 * a2);
        const float disc = fmaxf(B1 * B1 - A2 * C0, 0.0f);
        const float sq = sqrt_approx(disc);
        // the discriminant's binary32 error can reach ~4e-7 of its terms
        const float m = (sqrt_approx(4.0e-7f * (B1 * B1 + fabsf(A2 * C0))) + 4.0e-7f * (fabsf(B1) + sq)) * iA +
                        1.0e-6f;
        lo = (B1 - sq) * iA - m;
        hi = (B1 + sq) * iA + m;
    };
    float xl, xh, yl, yh;
    roots(ct * g.dx, st * g.e1x, st * g.e2x, xl, xh);
    roots(ct * g.dy, st * g.e1y, st * g.e2y, yl, yh);
    const float x1 = r.x0 + r.L * g.dx, y1 = r.y0 + r.L * g.dy;
    const float bx_lo = fminf(r.x0 + dz0 * xl, x1 + dz1 * xl), bx_hi = fmaxf(r.x0 + dz0 * xh, x1 + dz1 * xh);
    const float by_lo = fminf(r.y0 + dz0 * yl, y1 + dz1 * yl), by_hi = fmaxf(r.y0 + dz0 * yh, y1 + dz1 * yh);
    const float ax = fmaxf(fabsf(bx_lo), fabsf(bx_hi)), ay = fmaxf(fabsf(by_lo), fabsf(by_hi));
    const float zeta = (ax * ax + ay * ay) * A.inv_r_obs;
    const float rs = (r.rsb + r.cB * ((he_hi - A.h_obs) + zeta)) * 1.0001f + 0.5f;
    return bx_hi + rs < Tl.xmin || bx_lo - rs > Tl.xmax || by_hi + rs < Tl.ymin || by_lo - rs > Tl.ymax;
}

// EXT: the angular cut, fluorescence beaming and count rule 1 compiled in;
// DISP: dispersion (a Cherenkov ray's direction from the cone at the middle
// of its step's band, with the band's spread as a direction error and its
// largest g(lambda) in the refraction bounds).
template <bool SPH, bool REFR, bool EXT = false, bool DISP = false>
__global__ void __launch_bounds__(256, 4)
k_classify(const clight_segment *__restrict__ segs, int64_t n_segs, const __grid_constant__ DevAtm A,
           const __grid_constant__ DevTel Tl, const __grid_constant__ DevPar Pp, const __grid_constant__ DevOut O)
{
    extern __shared__ __align__(16) unsigned char smem_c[];
    constexpr int kWB = kClsWarpBytes + (EXT ? kClsBeamBytes : 0);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    ClsRec *rec = reinterpret_cast<ClsRec *>(smem_c + warp * kWB);
    uint2 *vl = reinterpret_cast<uint2 *>(smem_c + warp * kWB + 32 * sizeof(ClsRec));
    float4 *bc = reinterpret_cast<float4 *>(smem_c + warp * kWB + kClsWarpBytes);   // EXT only
    float4 *stage = reinterpret_cast<float4 *>(smem_c + nwarp * kWB + warp * kStageBytes);
    const uint8_t *clr = nullptr;                // the classification reads the fine map (Tl.fclr)
    // bound pieces that depend on the array and the atmosphere only
    const float dzmax = fmaxf(fabsf(Tl.zmax - A.h_obs), fabsf(Tl.zmin - A.h_obs));
    const float co2_min = 2.1f * A.delta_max + 2.6e-3f;
    // direction error of a Cherenkov ray from its azimuth: cos c e1 + sin c e2
    // moves by at most kAzErr, scaled by sin theta_c <= sqrt(2 delta_max (1 + delta_max))
    const float de_c = kAzErr * sqrtf(2.0f * A.delta_max * (1.0f + A.delta_max)) * 1.01f;
    uint32_t c_rays = 0, c_esc = 0, c_under = 0, c_skip = 0, c_guard = 0, c_whole = 0, c_cut = 0;
    unsigned status_bits = 0;
    WarpQueue dq;                    // the rays left to k_trace_deferred
    // work stealing: a claim is Pp.chunk consecutive groups of 32 steps; the
    // next claim's atomic is issued one group before it is needed, and each
    // group's records are copied in while the group before is worked on
    const unsigned long long chunk = (unsigned long long)Pp.chunk;
    unsigned long long cur = 0, end = 0;
    {
        unsigned long long c = 0;
        if (lane == 0) c = atomicAdd(O.ctr + CTR_WORK, 1ull);
        cur = __shfl_sync(FULL_MASK, c, 0) * chunk;
        end = cur + chunk;
    }
    prefetch_group(stage, segs, n_segs, (int64_t)cur * 32, lane);
    for (;;) {
        const unsigned long long grp = cur;
        const bool claim = cur + 1 == end;
        unsigned long long c = 0;
        if (claim && lane == 0) c = atomicAdd(O.ctr + CTR_WORK, 1ull);
        const int64_t s_first = (int64_t)grp * 32;
        if (s_first >= n_segs) break;
        const int64_t si = s_first + lane;
        float4 w0 = make_float4(0.f, 0.f, 0.f, 0.f), w1 = w0, w2 = w0, w3 = w0;
        cp_async_wait_all();
        __syncwarp();
        if (si < n_segs) {
            w0 = stage[lane * 4]; w1 = stage[lane * 4 + 1];
            w2 = stage[lane * 4 + 2]; w3 = stage[lane * 4 + 3];
        }
        __syncwarp();
        const clight_segment s = seg_from_words(w0, w1, w2, w3);
        if (claim) {
            cur = __shfl_sync(FULL_MASK, c, 0) * chunk;
            end = cur + chunk;
        } else {
            ++cur;
        }
        prefetch_group(stage, segs, n_segs, (int64_t)cur * 32, lane);

        // ---- per-step set-up: the counts exactly as the second pass forms them
        uint32_t nc = 0, nf = 0;
        ClsRec r;
        bool gated = false, whole = false;
        if (si < n_segs) {
            Seg<float, df> g;
            load_segment_f<SPH, EXT, DISP, false>(s, Pp.seg_base + si, A, Pp, g);
            if (g.bad) status_bits |= 1u << g.bad;
            c_guard += g.guarded;
            if (EXT) {
                c_cut += g.cut;
                bc[lane] = make_float4(g.bux, g.buy, g.buz, g.bomc);
            }
            nc = g.n_c;
            nf = g.n_f;
            if (nc > 0x7fffffffu || nf > 0x7fffffffu - nc) { status_bits |= 1u << CLIGHT_ERR_LIMIT; nc = nf = 0; }
            float ct = 1.0f - g.kappa, st = g.sin_tc, dth = 0.0f, glc = 1.0f;
            if (DISP && A.disp) {
                float kap;
                disp_band_cone(A, Pp, g, st, kap, dth, glc);
                ct = 1.0f - kap;
            }
            r.gl = glc;
            r.x0 = g.x0.hi; r.y0 = g.y0.hi; r.z0 = g.z0.hi; r.L = g.L;
            r.dx = g.dx; r.dy = g.dy; r.dz = g.dz; r.h_mid = g.h_mid;
            r.ax = ct * g.dx; r.ay = ct * g.dy; r.az = ct * g.dz;
            r.b1x = st * g.e1x; r.b1y = st * g.e1y; r.b1z = st * g.e1z;
            r.b2x = st * g.e2x; r.b2y = st * g.e2y; r.b2z = st * g.e2z;
            // dh/dl: the step direction's component along the local vertical
            // (approximate square roots and reciprocals: each bound below
            // carries margins far above their ~1e-7 relative error)
            float sdz = -g.dz;                                  // cos of the step's zenith angle (flat frame)
            float szd = sqrt_approx(g.dx * g.dx + g.dy * g.dy); // its sine
            float cps = sdz, sps = szd;                          // the same about the Earth radius at the start
            float r0 = 1.0f, ir0 = 1.0f;
            if (SPH) {
                const float Rz0 = r.z0 + A.R_E;
                ir0 = rsqrt_approx(r.x0 * r.x0 + r.y0 * r.y0 + Rz0 * Rz0);
                r0 = rcp_approx(ir0);
                const float c1 = g.dy * Rz0 - g.dz * r.y0, c2 = g.dz * r.x0 - g.dx * Rz0, c3 = g.dx * r.y0 - g.dy * r.x0;
                sps = sqrt_approx(c1 * c1 + c2 * c2 + c3 * c3) * ir0;
                cps = -(g.dx * r.x0 + g.dy * r.y0 + g.dz * Rz0) * ir0;
                r.hd = -cps;
            } else {
                r.hd = g.dz;
            }
            // Cherenkov bounds over the cone (half-angle theta_c: cos ct, sin st)
            r.rsb = 0.0f; r.cB = 0.0f; r.derr = 0.0f;
            if (nc > 0) {
                // a ray's direction error against the full trace's: the
                // azimuth's, and the cone's from a binary32 beta n - 1 g' (the
                // exact one within gerr of it).  theta_c ~ sqrt(2 g) is concave,
                // so the largest change is toward g' - gerr: sqrt(2 g') -
                // sqrt(2 (g' - gerr)) <= 2 gerr / theta_c'; cos theta_c moves by
                // at most gerr.  Margins 1.1.
                const float dstep = de_c + g.gerr * (2.2f * rcp_approx(st) + 1.1f) + dth;
                r.derr = dstep;
                // -d_gamma,z >= cos(zeta_d + theta_c)
                const float dzlo = sdz * ct - szd * st - 4.0e-6f - dstep;
                float cobs_lo = dzlo;
                bool ok = dzlo > 0.05f;
                if (SPH) {
                    // landing zenith sine: (r_e / r_obs) sin(psi_e), psi_e <= psi_d + theta_c + L / r0
                    const float csum = cps * ct - sps * st;
                    const float se = sps * ct + cps * st + (r.L + 1.0f) * ir0 + 4.0e-6f + dstep;
                    const float so = (r0 + r.L) * se * A.inv_r_obs * 1.000001f;
                    const float co2 = 1.0f - so * so;
                    ok = ok && csum > 0.0f && so < 1.0f && co2 > (DISP ? 2.1f * A.delta_max * glc + 2.6e-3f : co2_min);
                    cobs_lo = ok ? sqrt_approx(co2) * 0.999999f : 0.0f;
                }
                const float mu = fminf(cobs_lo, dzlo) - 1.0e-3f;
                ok = ok && mu > 0.05f;
                if (ok) {
                    const float im = rcp_approx(mu) * 1.000001f;
                    const float sd = REFR ? 1.25f * 1.000001f * sqrt_approx(1.0f - mu * mu) * A.delta_max * glc : 0.0f;
                    const float czb = dzlo - sd * im - 1.0e-5f;
                    ok = czb > 0.05f;
                    if (ok) {
                        // the refraction term per metre of height, plus the
                        // direction error's: the crossing moves by at most
                        // dstep tp (1 + 1/|d_z|), tp <= (h - h_obs) / dzlo
                        const float iz = rcp_approx(dzlo) * 1.000001f;
                        r.cB = sd * (im * im * im) * 1.0001f + 1.05f * dstep * iz * (1.0f + iz);
                        r.rsb = ((Tl.Rmax + dzmax * sqrt_approx(1.0f - czb * czb)) * rcp_approx(czb) + 2.0e-3f +
                                 0.05f) * 1.0001f + 1.0e-3f;
                    }
                }
                gated = ok;
                if (gated) whole = cone_lands_clear(g, r, ct, st, A, Tl);
            }
            r.nc = nc;
        }
        // a step whose every Cherenkov photon provably lands clear of the
        // array: its rays are counted here and never enumerated
        const uint32_t ncv = whole ? 0u : nc;
        if (whole) { c_rays += nc; c_skip += nc; c_whole += nc; }
        // ---- virtual steps: the Cherenkov steps with bunches, then the fluorescence ones
        const unsigned bC = __ballot_sync(FULL_MASK, ncv > 0), bF = __ballot_sync(FULL_MASK, nf > 0);
        const unsigned lt = lanemask_lt();
        uint32_t incC = ncv, incF = nf;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t vc = __shfl_up_sync(FULL_MASK, incC, o), vf = __shfl_up_sync(FULL_MASK, incF, o);
            if (lane >= o) { incC += vc; incF += vf; }
        }
        const uint32_t totC = __shfl_sync(FULL_MASK, incC, 31), totF = __shfl_sync(FULL_MASK, incF, 31);
        const uint32_t eC = incC - ncv, eF = totC + incF - nf;  // start positions in the group's ray sequence
        if (totF > 0x7fffffffu - totC) { status_bits |= 1u << CLIGHT_ERR_LIMIT; continue; }
        if (si < n_segs) rec[lane] = r;
        if (ncv > 0) vl[__popc(bC & lt)] = make_uint2(eC, (uint32_t)lane | (gated ? kVGated : 0u));
        if (nf > 0) vl[__popc(bC) + __popc(bF & lt)] = make_uint2(eF, (uint32_t)lane | 32u);
        __syncwarp();
        const uint32_t total = totC + totF;
        if (lane == 0) c_rays += total;
        // ---- the rays, 32 per round
        int carry = -1;
        for (uint32_t base = 0; base < total; base += 32) {
            uint32_t bits = 0;
            if (ncv > 0 && eC - base < 32u) bits |= 1u << (eC - base);
            if (nf > 0 && eF - base < 32u) bits |= 1u << (eF - base);
            const unsigned M = __reduce_or_sync(FULL_MASK, bits);
            const int idx = carry + __popc(M & (lt | (1u << lane)));
            carry += __popc(M);
            const uint32_t pos = base + (uint32_t)lane;
            const bool active = pos < total;
            int cls = -1;
            int64_t seg_local = 0;
            uint32_t kq = 0;
            if (active) {
                const uint2 v = vl[idx];
                const int l = (int)(v.y & 31u);
                const uint32_t proc = (v.y >> 5) & 1u;
                const uint32_t kk = pos - v.x;
                seg_local = s_first + l;
                const int64_t seg_global = Pp.seg_base + seg_local;
                const uint4 x = philox4x32_10(make_uint4((uint32_t)(uint64_t)seg_global,
                                                         (uint32_t)((uint64_t)seg_global >> 32), kk, proc),
                                              Pp.seed, Pp.stream);
                const float u1 = u01<float>(x.y), u2 = u01<float>(x.z);
                // the azimuth 2 pi u2 by the MUFU sine and cosine at
                // 2 pi (u2 - 1/2), inside [-pi, pi] where their absolute error
                // is at most 2^-21.41 (sin 2 pi u = -sin 2 pi (u - 1/2)); the
                // decisions below carry that error (kAzErr) as a direction
                // error, and the full trace forms the azimuth with sincospif
                float sn, cs;
                __sincosf(6.28318531f * (u2 - 0.5f), &sn, &cs);
                sn = -sn;
                cs = -cs;
                // the step's record in 128-bit shared loads, those of a
                // process issued together
                const float4 *rq = reinterpret_cast<const float4 *>(rec + l);
                ClsRec R;
                {
                    const float4 q0 = rq[0], q1 = rq[1], q2 = rq[2];
                    R.x0 = q0.x; R.y0 = q0.y; R.z0 = q0.z; R.L = q0.w;
                    R.dx = q1.x; R.dy = q1.y; R.dz = q1.z; R.h_mid = q1.w;
                    R.ax = q2.x; R.ay = q2.y; R.az = q2.z; R.hd = q2.w;
                }
                const float ell = u1 * R.L;
                if (proc == 0) {
                    kq = kk;
                    const float4 q3 = rq[3], q4 = rq[4];
                    R.b1x = q3.x; R.b1y = q3.y; R.b1z = q3.z; R.rsb = q3.w;
                    R.b2x = q4.x; R.b2y = q4.y; R.b2z = q4.z; R.cB = q4.w;
                    const float dgx = R.ax + (cs * R.b1x + sn * R.b2x);
                    const float dgy = R.ay + (cs * R.b1y + sn * R.b2y);
                    const float dgz = R.az + (cs * R.b1z + sn * R.b2z);
                    cls = (v.y & kVGated)
                              ? classify_cherenkov_gated<SPH>(R, ell, dgx, dgy, dgz, A, Tl, clr)
                              : classify_ray<SPH, REFR, DISP>(R, ell, dgx, dgy, dgz,
                                                              reinterpret_cast<const float4 *>(rq)[5].y,
                                                              reinterpret_cast<const float4 *>(rq)[5].z, A, Tl, clr);
                } else {
                    R.nc = reinterpret_cast<const uint4 *>(rq)[5].x;
                    kq = R.nc + kk;
                    const float u3 = u01<float>(x.w);
                    float fx, fy, fz;
                    const float4 b = EXT ? bc[l] : make_float4(0.f, 0.f, 0.f, 0.f);
                    if (EXT && b.w > 0.0f) {
                        // beamed: the full trace's cone direction, from the same azimuth
                        cone_direction<float>(b.x, b.y, b.z, u3 * b.w, sn, cs, fx, fy, fz);
                    } else {
                        fz = 2.0f * u3 - 1.0f;
                        const float sz = sqrt_approx((1.0f - fz) * (1.0f + fz));
                        fx = sz * cs;
                        fy = sz * sn;
                    }
                    // dispersion: this photon's refractivity is delta(h) g(lambda)
                    const float glf = (DISP && A.disp)
                                          ? disp_gu<float>(A, rcp_approx(Pp.fl1 + u01<float>(x.x) * Pp.fdl)) * 1.000001f
                                          : 1.0f;
                    cls = classify_ray<SPH, REFR, DISP>(R, ell, fx, fy, fz, kAzErr, glf, A, Tl, clr);
                }
                c_esc += cls == 1;
                c_under += cls == 2;
                c_skip += cls == 6;
            }
            dq.push(cls == 0, ((unsigned long long)seg_local << 32) | (unsigned long long)kq, O, lane, status_bits);
        }
        __syncwarp();
    }
    dq.finish(O, lane, status_bits);
    const uint32_t vals[ST_N] = {c_rays, c_esc, c_under, 0u, c_skip, 0u, c_guard, 0u, 0u, c_cut, c_skip, 0u, c_whole};
    flush_stats(vals, status_bits, O, lane);
}

// Second pass of the deferred path: the queued rays, 32 per warp, each from
// its step record in global memory (set up again exactly as in the first
// pass), traced and hit-tested in full.  Ray counts were taken in the first
// pass.  Persistent grid, each warp taking the next 32 entries from a counter.
template <bool SPH, bool REFR, int FEAT, class P = df, bool NOALLOC = false>
__global__ void __launch_bounds__(256, 3)
k_trace_deferred(const clight_segment *__restrict__ segs, const __grid_constant__ DevAtm A,
                 const __grid_constant__ DevTel Tl, const __grid_constant__ DevPar Pp,
                 const __grid_constant__ DevOut O)
{
    constexpr bool EXT = (FEAT & FEAT_EXT) != 0;
    extern __shared__ float smem[];
    const int lane = threadIdx.x & 31;
    const uint8_t *clr = EXT ? Tl.clr : nullptr;
    if (!EXT && Tl.clr) {
        uint4 *dst = reinterpret_cast<uint4 *>(smem);
        const uint4 *src = reinterpret_cast<const uint4 *>(Tl.clr);
        for (int i = threadIdx.x; i < (Tl.clr_bytes >> 4); i += blockDim.x) dst[i] = __ldg(src + i);
        __syncthreads();
        clr = reinterpret_cast<const uint8_t *>(dst);
    }
    const int64_t n = min((int64_t)O.ctr[CTR_DEFER], O.defer_cap);
    uint32_t c_esc = 0, c_under = 0, c_turn = 0, c_reach = 0, c_hits = 0, c_cells = 0, c_def = 0;
    unsigned status_bits = 0;
    for (;;) {
        unsigned long long grp = 0;
        if (lane == 0) grp = atomicAdd(O.ctr + CTR_DEFER_WORK, 1ull);
        const int64_t base = (int64_t)__shfl_sync(FULL_MASK, grp, 0) * 32;
        if (base >= n) break;
        const int64_t i = base + lane;
        const bool active = i < n;
        const unsigned long long e = O.defer[active ? i : base];
        const int64_t seg_local = (int64_t)(e >> 32);
        const uint32_t k = (uint32_t)e;
        const int64_t seg_global = Pp.seg_base + seg_local;
        const float4 *src = reinterpret_cast<const float4 *>(segs + seg_local);
        const clight_segment s = seg_from_words(__ldg(src), __ldg(src + 1), __ldg(src + 2), __ldg(src + 3));
        Seg<float, df> g;
        load_segment_f<SPH, EXT, (FEAT & FEAT_DISP) != 0>(s, seg_global, A, Pp, g);
        int st;
        uint32_t cells;
        if constexpr (std::is_same<P, double>::value) {
            // binary64 at the steps that otherwise carry FP32 pairs
            Seg<float, double> qd;
            widen_seg(g, qd);
            RayOut<float, double> o;
            trace_ray<float, double, true, SPH, REFR, FEAT>(qd, seg_global, k, active, A, Pp, o);
            c_hits += hit_test<float, double, true, NOALLOC>(o, Pp.key_off + seg_local, seg_global, k, g.shower, A,
                                                             Tl, Pp, O, status_bits, clr);
            st = o.status;
            cells = o.cells;
        } else {
            RayOut<float, df> o;
            trace_ray<float, df, true, SPH, REFR, FEAT>(g, seg_global, k, active, A, Pp, o);
            c_hits += hit_test<float, df, true, NOALLOC>(o, Pp.key_off + seg_local, seg_global, k, g.shower, A, Tl,
                                                         Pp, O, status_bits, clr);
            st = o.status;
            cells = o.cells;
        }
        if (active) {
            c_esc += st == 1; c_under += st == 2; c_turn += st == 3;
            c_reach += st == 0 || st == 5;
            c_cells += st == 0 ? cells : 0;
            ++c_def;
        }
    }
    const uint32_t vals[ST_N] = {0u, c_esc, c_under, c_turn, c_reach, c_hits, 0u, 0u, c_cells, 0u, 0u, c_def, 0u};
    flush_stats(vals, status_bits, O, lane);
}

// ------------------------------------------------------------------ plain FP64
// One thread per segment, binary64 throughout, every bunch of the segment in
// turn, one atomic per hit.
template <bool SPH, bool REFR>
__global__ void __launch_bounds__(128)
k_trace_fp64(const clight_segment *__restrict__ segs, int64_t n_segs, const __grid_constant__ DevAtm A,
             const __grid_constant__ DevTel Tl, const __grid_constant__ DevPar Pp, const __grid_constant__ DevOut O)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_segs) return;
    unsigned status_bits = 0;
    Seg<double, double> g;
    load_segment_d<SPH>(segs[i], Pp.seg_base + i, A, Pp, g);
    uint32_t c_rays = 0, c_esc = 0, c_under = 0, c_turn = 0, c_reach = 0, c_hits = 0, c_cells = 0;
    uint32_t c_cut = g.cut;
    if (g.bad) {
        status_bits |= 1u << g.bad;
    } else {
        uint32_t nb = g.n_c + g.n_f;
        if (nb < g.n_c || nb > 0x7fffffffu) { status_bits |= 1u << CLIGHT_ERR_LIMIT; nb = 0; }
        int64_t seg_global = Pp.seg_base + i;
        for (uint32_t k = 0; k < nb; ++k) {
            RayOut<double, double> o;
            trace_ray<double, double, false, SPH, REFR>(g, seg_global, k, true, A, Pp, o);
            ++c_rays;
            c_esc += o.status == 1; c_under += o.status == 2; c_turn += o.status == 3;
            c_reach += o.status == 0 || o.status >= 5;
            c_cells += o.status == 0 ? o.cells : 0;
            c_hits += hit_test<double, double, false>(o, i, seg_global, k, g.shower, A, Tl, Pp, O, status_bits);
        }
    }
    uint32_t vals[ST_N] = {c_rays, c_esc, c_under, c_turn, c_reach, c_hits, 0u, 0u, c_cells, c_cut, 0u, 0u, 0u};
    for (int q = 0; q < ST_N; ++q)
        if (vals[q] && q != ST_STATUS) atomicAdd(O.ctr + CTR_STATS + q, (unsigned long long)vals[q]);
    if (status_bits) atomicOr(O.ctr + CTR_STATS + ST_STATUS, (unsigned long long)status_bits);
}


// The two-pass launch (first pass, then the queued rays) of a feature set
// that has one (trace_twopass.cu); P = df or double (the precise steps).
template <class P>
void launch_two_pass(int feat, const clight_segment *segs, int64_t n_segs, const DevAtm &A, const DevTel &T,
                     const DevPar &Pp, const DevOut &O, int grid, int block, cudaStream_t s);
template <>
void launch_two_pass<df>(int feat, const clight_segment *segs, int64_t n_segs, const DevAtm &A, const DevTel &T,
                         const DevPar &Pp, const DevOut &O, int grid, int block, cudaStream_t s);
template <>
void launch_two_pass<double>(int feat, const clight_segment *segs, int64_t n_segs, const DevAtm &A,
                             const DevTel &T, const DevPar &Pp, const DevOut &O, int grid, int block, cudaStream_t s);

}  // namespace clight
