// trace_noalloc.cu -- the adjoint's candidate pass and the entry point
// without allocation (its scratch is a static array of this file).
#include <algorithm>

#include "trace_kernels.cuh"

namespace clight {

// ------------------------------------------------------------------ no allocation
// Scratch of clight_trace_noalloc: the work and hit counters and the ray
// statistics (CTR_N words), then one hit counter per (shower, telescope)
// group, then a copy of both taken before each chunk of the two-pass form;
// and that form's deferred-ray queue.  They live in the library image, so
// the entry point needs no cudaMalloc; every GPU that loads the library
// holds these 262,416 + 33,554,432 bytes until the process exits.
constexpr int kNoallocMaxGroups = 16384;
constexpr int64_t kNoallocWords = CTR_N + kNoallocMaxGroups;
constexpr int64_t kNoallocQueue = int64_t(1) << 22;     // deferred rays of one chunk
constexpr int64_t kNoallocChunk = int64_t(1) << 24;     // steps per chunk
static __device__ __align__(256) unsigned long long g_noalloc_scratch[2 * kNoallocWords];
static __device__ __align__(256) unsigned long long g_noalloc_queue[kNoallocQueue];

// The device addresses of the static arrays on the current device.  In host
// code their names are only stand-ins, so the addresses come from the
// runtime; they are looked up once per context (whose device is current
// here) and kept in the context, which a device reset invalidates as a whole.
static cudaError_t noalloc_arrays(clight_ctx *ctx, unsigned long long **scratch, unsigned long long **queue)
{
    void **slot = ctx_noalloc_slot(ctx);
    if (!slot) return cudaErrorInvalidValue;
    if (!slot[0] || !slot[1]) {
        void *p = nullptr, *q = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e == cudaSuccess) e = cudaGetSymbolAddress(&q, g_noalloc_queue);
        if (e != cudaSuccess) return e;
        slot[0] = p;
        slot[1] = q;
    }
    *scratch = static_cast<unsigned long long *>(slot[0]);
    *queue = static_cast<unsigned long long *>(slot[1]);
    return cudaSuccess;
}

template <int FEAT>
static void launch_soft_f(const clight_segment *segs, int64_t n_segs, const DevAtm &A, const DevTel &T,
                          const DevPar &Pp, const DevOut &O, int grid, int block, cudaStream_t s)
{
    const int smem = fused_smem_bytes_f(block, T, (FEAT & FEAT_EXT) != 0);
    if (A.spherical && A.refraction)
        k_trace_fused<df, true, true, false, true, FEAT><<<grid, block, smem, s>>>(segs, n_segs, A, T, Pp, O);
    else if (A.spherical)
        k_trace_fused<df, true, false, false, true, FEAT><<<grid, block, smem, s>>>(segs, n_segs, A, T, Pp, O);
    else if (A.refraction)
        k_trace_fused<df, false, true, false, true, FEAT><<<grid, block, smem, s>>>(segs, n_segs, A, T, Pp, O);
    else
        k_trace_fused<df, false, false, false, true, FEAT><<<grid, block, smem, s>>>(segs, n_segs, A, T, Pp, O);
}

// The adjoint's candidate pass (exact propagator, no dispersion: the
// adjoint refuses the others), with the angular cut and beaming compiled in
// only when on.
cudaError_t launch_soft_candidates(const clight_segment *segs, int64_t n_segs, const DevAtm &A, const DevTel &T,
                                   const DevPar &Pp, const DevOut &O, int grid, int block, cudaStream_t s)
{
    if (Pp.cut_mode != CLIGHT_CUT_OFF || Pp.beam || Pp.roulette)
        launch_soft_f<FEAT_EXT>(segs, n_segs, A, T, Pp, O, grid, block, s);
    else
        launch_soft_f<0>(segs, n_segs, A, T, Pp, O, grid, block, s);
    return cudaGetLastError();
}

template <class P, bool SPH, bool REFR>
static void launch_noalloc(const clight_segment *segs, int64_t n_segs, const DevAtm &A, const DevTel &T,
                           const DevPar &Pp, const DevOut &O, int grid, int block, cudaStream_t s)
{
    k_trace_fused<P, SPH, REFR, true><<<grid, block, fused_smem_bytes(block, T), s>>>(segs, n_segs, A, T, Pp, O);
}

// The default feature set on a spherical, refracting atmosphere in FP32
// pairs takes the two passes of clight_trace: the classification queues the
// rays that may land near a telescope and k_trace_deferred traces them, one
// chunk of steps at a time so that the static queue holds a chunk's rays.  A
// chunk whose rays overflow it (its first pass sets the status bit) is
// traced again by the in-place kernel from the counters saved before it.
static cudaError_t noalloc_two_pass(const clight_segment *segs, int64_t n_segs, const DevAtm &A, const DevTel &T,
                                    DevPar P, DevOut O, unsigned long long *queue, unsigned long long *backup,
                                    int64_t words, int n_sm, int block, cudaStream_t s)
{
    const int smem1 = cls_smem_bytes(block, T), smem2 = T.clr ? T.clr_bytes : 0;
    cudaError_t e = cudaFuncSetAttribute(k_classify<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem1);
    if (e != cudaSuccess) return e;
    int per_sm1 = 1, per_sm2 = 1;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm1, k_classify<true, true>, block, smem1)) !=
            cudaSuccess ||
        (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, k_trace_deferred<true, true, 0, df, true>,
                                                           block, smem2)) != cudaSuccess)
        return e;
    const int64_t seg_base = P.seg_base;
    for (int64_t start = 0; start < n_segs; start += kNoallocChunk) {
        const int64_t m = std::min(kNoallocChunk, n_segs - start);
        P.seg_base = seg_base + start;
        O.defer = queue;
        O.defer_cap = kNoallocQueue;
        const int64_t groups32 = (m + 31) / 32;
        const int grid1 = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)n_sm * std::max(per_sm1, 1), groups32));
        const int grid2 = std::max(1, n_sm * std::max(per_sm2, 1));
        if ((e = cudaMemcpyAsync(backup, O.ctr, sizeof(unsigned long long) * (size_t)words, cudaMemcpyDeviceToDevice,
                                 s)) != cudaSuccess ||
            (e = cudaMemsetAsync(O.ctr + CTR_WORK, 0, sizeof(unsigned long long), s)) != cudaSuccess ||
            (e = cudaMemsetAsync(O.ctr + CTR_DEFER, 0, 2 * sizeof(unsigned long long), s)) != cudaSuccess)
            return e;
        k_classify<true, true><<<grid1, block, smem1, s>>>(segs + start, m, A, T, P, O);
        k_trace_deferred<true, true, 0, df, true><<<grid2, block, smem2, s>>>(segs + start, A, T, P, O);
        unsigned long long status = 0;
        if ((e = cudaMemcpyAsync(&status, O.ctr + CTR_STATS + ST_STATUS, sizeof(status), cudaMemcpyDeviceToHost,
                                 s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess)
            return e;
        if (status & (1ull << kBitDeferFull)) {
            if ((e = cudaMemcpyAsync(O.ctr, backup, sizeof(unsigned long long) * (size_t)words,
                                     cudaMemcpyDeviceToDevice, s)) != cudaSuccess ||
                (e = cudaMemsetAsync(O.ctr + CTR_WORK, 0, sizeof(unsigned long long), s)) != cudaSuccess)
                return e;
            O.defer = nullptr;
            const int grid0 = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)n_sm * 3, (m + block - 1) / block));
            launch_noalloc<df, true, true>(segs + start, m, A, T, P, O, grid0, block, s);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace clight

extern "C" clight_status clight_trace_noalloc(clight_ctx *ctx, const clight_segment *d_segs, int64_t n_segs,
                                              int32_t n_showers, clight_hit *d_hits, int64_t hit_capacity,
                                              int64_t *d_counts, clight_stats *h_stats, int64_t *h_n_hits,
                                              void *stream)
{
    using namespace clight;
    CtxView v;
    if (!ctx_view(ctx, &v)) return CLIGHT_ERR_ARG;
    if (n_segs < 0 || n_showers < 1 || hit_capacity < 0 || !h_n_hits || (n_segs > 0 && !d_segs) ||
        (hit_capacity > 0 && !d_hits) || (reinterpret_cast<uintptr_t>(d_segs) & 15u))
        return CLIGHT_ERR_ARG;
    if (n_segs > (int64_t(1) << 31)) return CLIGHT_ERR_LIMIT;
    int64_t groups = (int64_t)n_showers * v.tel.n_tel;
    if (groups > kNoallocMaxGroups) return CLIGHT_ERR_LIMIT;     // n_showers x n_tel above 16384
    DeviceGuard dg(v.device);                                    // the caller's device comes back on return
    if (!dg.ok) return CLIGHT_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    // the call reads its counters back and synchronises its stream, which a
    // stream capture does not allow: refuse one, leaving the capture intact
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return CLIGHT_ERR_CUDA;
    if (cs != cudaStreamCaptureStatusNone) return CLIGHT_ERR_ARG;
    unsigned long long *scr = nullptr, *queue = nullptr;
    if (noalloc_arrays(ctx, &scr, &queue) != cudaSuccess) return CLIGHT_ERR_CUDA;
    // counters and group counts left by the previous call start again at zero
    if (cudaMemsetAsync(scr, 0, sizeof(unsigned long long) * (size_t)(CTR_N + groups), s) != cudaSuccess)
        return CLIGHT_ERR_CUDA;
    if (n_segs > 0) {
        DevPar P = v.par;
        P.n_showers = n_showers;
        DevOut O{};
        O.rec = d_hits;
        O.keys = scr + CTR_N;        // per-group hit counters
        O.vals = nullptr;
        O.capacity = hit_capacity;
        O.ctr = scr;
        int block = v.block;
        int64_t grid = std::min<int64_t>((int64_t)v.n_sm * v.ctas_per_sm, (n_segs + block - 1) / block);
        grid = std::max<int64_t>(grid, 1);
        const DevAtm &A = v.atm;
        bool fp64 = v.precision == CLIGHT_PREC_FP64_GUARD;
        const bool plain = !fp64 && A.spherical && A.refraction && !A.disp && P.cut_mode == CLIGHT_CUT_OFF && !P.beam &&
                           !P.roulette && P.prop == CLIGHT_PROP_EXACT;
        auto go = [&](auto tag) {
            using PP = decltype(tag);
            if (A.spherical && A.refraction) launch_noalloc<PP, true, true>(d_segs, n_segs, A, v.tel, P, O, (int)grid, block, s);
            else if (A.spherical) launch_noalloc<PP, true, false>(d_segs, n_segs, A, v.tel, P, O, (int)grid, block, s);
            else if (A.refraction) launch_noalloc<PP, false, true>(d_segs, n_segs, A, v.tel, P, O, (int)grid, block, s);
            else launch_noalloc<PP, false, false>(d_segs, n_segs, A, v.tel, P, O, (int)grid, block, s);
        };
        if (plain) {
            if (noalloc_two_pass(d_segs, n_segs, A, v.tel, P, O, queue, scr + kNoallocWords, CTR_N + groups, v.n_sm,
                                 block, s) != cudaSuccess)
                return CLIGHT_ERR_CUDA;
        } else if (fp64) {
            go(double{});
        } else {
            go(df{});
        }
        if (cudaGetLastError() != cudaSuccess) return CLIGHT_ERR_CUDA;
    }
    unsigned long long h[CTR_N];
    if (cudaMemcpyAsync(h, scr, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess) return CLIGHT_ERR_CUDA;
    if (d_counts && cudaMemcpyAsync(d_counts, scr + CTR_N, sizeof(int64_t) * (size_t)groups,
                                    cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return CLIGHT_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return CLIGHT_ERR_CUDA;
    *h_n_hits = (int64_t)h[CTR_CURSOR];
    unsigned long long bits = h[CTR_STATS + ST_STATUS];
    if (h_stats) {
        h_stats->rays = (int64_t)h[CTR_STATS + ST_RAYS];
        h_stats->escaped = (int64_t)h[CTR_STATS + ST_ESCAPED];
        h_stats->under = (int64_t)h[CTR_STATS + ST_UNDER];
        h_stats->turned = (int64_t)h[CTR_STATS + ST_TURNED];
        h_stats->reached = (int64_t)h[CTR_STATS + ST_REACHED];
        h_stats->hits = (int64_t)h[CTR_STATS + ST_HITS];
        h_stats->guarded = (int64_t)h[CTR_STATS + ST_GUARDED];
        h_stats->status = (int64_t)bits;
        h_stats->cells = (int64_t)h[CTR_STATS + ST_CELLS];
        h_stats->cut = (int64_t)h[CTR_STATS + ST_CUT];
        h_stats->skipped = (int64_t)h[CTR_STATS + ST_SKIPPED];
        h_stats->deferred = (int64_t)h[CTR_STATS + ST_DEFERRED];
        h_stats->step_skipped = (int64_t)h[CTR_STATS + ST_STEP_SKIPPED];
    }
    if ((int64_t)h[CTR_CURSOR] > hit_capacity) return CLIGHT_ERR_HIT_CAPACITY;
    if (bits & (1ull << CLIGHT_ERR_BAD_SEGMENT)) return CLIGHT_ERR_BAD_SEGMENT;
    if (bits & (1ull << CLIGHT_ERR_LIMIT)) return CLIGHT_ERR_LIMIT;
    return CLIGHT_OK;
}
