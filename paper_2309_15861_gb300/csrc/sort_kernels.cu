// sort_kernels.cu -- ordering the hits and reducing them per telescope.
//
// Hits leave the fused kernel in arbitrary order (one atomic per warp and
// round).  The per-telescope photon lists the paper's pipeline hands
// downstream (Sec. 1, "common memory block"; Sec. 2) are made deterministic
// here: a stable LSD radix sort of the 64-bit keys
// (shower * n_tel + telescope, segment, bunch), a gather of the 48-byte
// records into that order, and per-(shower, telescope) counts and binary64
// photon sums taken in that fixed order.
//
// Every kernel reads the number of hits from the device counter, so the
// whole sequence can run inside a CUDA graph; when the hits overflowed the
// caller's capacity the count is taken as zero and nothing is written.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "internal.h"

namespace clight {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kTile = kSortThreads * kSortItems;        // 2048 keys per tile
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanChunk = kScanThreads * kScanItems;   // 4096 entries per block

int sort_tile_items() { return kTile; }

static int device_sms()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        n = 0;
    return n > 0 ? n : 1;
}
int64_t scan_block_sums_needed(int64_t n) { return (n + kScanChunk - 1) / kScanChunk; }

__device__ __forceinline__ int64_t valid_hits(const unsigned long long *ctr, int64_t capacity)
{
    unsigned long long c = ctr[CTR_CURSOR];
    return (int64_t)c <= capacity ? (int64_t)c : 0;
}

__device__ __forceinline__ unsigned lane_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ int64_t live_tiles(int64_t n) { return (n + kTile - 1) / kTile; }

// Per-tile digit histograms of the live tiles (those holding hits), stored
// digit-major with the live tile count as stride: hist[d * nt + tile].  A
// bounded grid walks the tiles, so the work follows the hit count, not the
// buffer's capacity.
__global__ void __launch_bounds__(kSortThreads)
k_radix_hist(const unsigned long long *__restrict__ keys, const unsigned long long *ctr, int64_t capacity,
             int shift, uint32_t *__restrict__ hist)
{
    __shared__ uint32_t cnt[256];
    const int64_t n = valid_hits(ctr, capacity);
    const int64_t nt = live_tiles(n);
    for (int64_t tile = blockIdx.x; tile < nt; tile += gridDim.x) {
        cnt[threadIdx.x] = 0;
        __syncthreads();
        const int64_t base = tile * kTile;
#pragma unroll 4
        for (int i = 0; i < kSortItems; ++i) {
            int64_t idx = base + (int64_t)i * kSortThreads + threadIdx.x;
            if (idx < n) atomicAdd(&cnt[(keys[idx] >> shift) & 0xFF], 1u);
        }
        __syncthreads();
        hist[(int64_t)threadIdx.x * nt + tile] = cnt[threadIdx.x];
        __syncthreads();
    }
}

// ---- exclusive scan of a uint32 array (three kernels) ---------------------
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *warp_tot, uint32_t *total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t t = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
        uint32_t s = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < (int)(blockDim.x >> 5)) warp_tot[lane] = s - t;
        if (lane == 31) *total = s;
    }
    __syncthreads();
    uint32_t r = x - v + warp_tot[w];
    __syncthreads();
    return r;
}

// The histograms' live length: 256 digits x the live tiles.
__device__ __forceinline__ int64_t live_hist(const unsigned long long *ctr, int64_t capacity)
{
    return 256 * live_tiles(valid_hits(ctr, capacity));
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_reduce(const uint32_t *__restrict__ a, const unsigned long long *ctr, int64_t capacity,
              uint32_t *__restrict__ sums)
{
    __shared__ uint32_t red[kScanThreads / 32];
    const int64_t n = live_hist(ctr, capacity);
    const int64_t nb = (n + kScanChunk - 1) / kScanChunk;
    for (int64_t blk = blockIdx.x; blk < nb; blk += gridDim.x) {
        const int64_t base = blk * kScanChunk;
        uint32_t s = 0;
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            int64_t idx = base + (int64_t)threadIdx.x * kScanItems + i;
            if (idx < n) s += a[idx];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x < 32) {
            uint32_t t = red[threadIdx.x];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (threadIdx.x == 0) sums[blk] = t;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_top(uint32_t *__restrict__ sums, const unsigned long long *ctr, int64_t capacity)
{
    __shared__ uint32_t wt[32];
    __shared__ uint32_t tot;
    const int64_t n = (live_hist(ctr, capacity) + kScanChunk - 1) / kScanChunk;
    uint32_t carry = 0;
    for (int64_t base = 0; base < n; base += kScanThreads) {
        int64_t idx = base + threadIdx.x;
        uint32_t v = idx < n ? sums[idx] : 0;
        uint32_t e = block_exclusive_scan(v, wt, &tot);
        if (idx < n) sums[idx] = e + carry;
        carry += tot;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_apply(uint32_t *__restrict__ a, const unsigned long long *ctr, int64_t capacity,
             const uint32_t *__restrict__ sums)
{
    __shared__ uint32_t wt[32];
    __shared__ uint32_t tot;
    const int64_t n = live_hist(ctr, capacity);
    const int64_t nb = (n + kScanChunk - 1) / kScanChunk;
    for (int64_t blk = blockIdx.x; blk < nb; blk += gridDim.x) {
        const int64_t base = blk * kScanChunk + (int64_t)threadIdx.x * kScanItems;
        uint32_t v[kScanItems];
        uint32_t s = 0;
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            v[i] = base + i < n ? a[base + i] : 0;
            s += v[i];
        }
        uint32_t e = block_exclusive_scan(s, wt, &tot) + sums[blk];
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            if (base + i < n) a[base + i] = e;
            e += v[i];
        }
    }
}

// In-place exclusive scan of the live histograms; grid: blocks for at most
// `max_n` entries, capped at `cap_blocks`.
static cudaError_t exclusive_scan(uint32_t *a, int64_t max_n, const unsigned long long *ctr, int64_t capacity,
                                  uint32_t *sums, int cap_blocks, cudaStream_t s)
{
    const int64_t nb = std::max<int64_t>(1, std::min<int64_t>(scan_block_sums_needed(max_n), cap_blocks));
    k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, s>>>(a, ctr, capacity, sums);
    k_scan_top<<<1, kScanThreads, 0, s>>>(sums, ctr, capacity);
    k_scan_apply<<<(unsigned)nb, kScanThreads, 0, s>>>(a, ctr, capacity, sums);
    return cudaGetLastError();
}

// Stable scatter of one 8-bit digit.  Warp w of a tile owns items
// [w*256, (w+1)*256) and walks them in 8 rounds of 32 consecutive keys;
// __match_any_sync groups equal digits inside a round, a per-warp counter
// per digit carries ranks across rounds, and a prefix over the warps per
// digit places each warp after the ones before it.  The tile is first
// ordered by digit in shared memory, then written out in that order, so each
// digit's run leaves as consecutive addresses (coalesced stores).
__global__ void __launch_bounds__(kSortThreads, 3)
k_radix_scatter(const unsigned long long *__restrict__ kin, const uint32_t *__restrict__ vin,
                unsigned long long *__restrict__ kout, uint32_t *__restrict__ vout,
                const unsigned long long *ctr, int64_t capacity, int shift,
                const uint32_t *__restrict__ hist)
{
    __shared__ uint32_t wcount[kSortThreads / 32][256];
    __shared__ uint32_t gbase[256];
    __shared__ uint32_t tdo[256];                 // the tile's first position of each digit
    __shared__ uint32_t wt[32], tot;
    __shared__ unsigned long long skey[kTile];
    __shared__ uint32_t sval[kTile];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t n = valid_hits(ctr, capacity);
    const int64_t nt = live_tiles(n);
    for (int64_t tile = blockIdx.x; tile < nt; tile += gridDim.x) {
        const int64_t tile0 = tile * kTile;
        const int tile_n = (int)min((int64_t)kTile, n - tile0);
        for (int d = lane; d < 256; d += 32) wcount[w][d] = 0;
        gbase[threadIdx.x] = hist[(int64_t)threadIdx.x * nt + tile];
        __syncwarp();
        unsigned long long key[kSortItems];
        uint32_t val[kSortItems];
        uint32_t loc[kSortItems];
        int dig[kSortItems];
        const int64_t wbase = tile0 + (int64_t)w * (kSortItems * 32);
#pragma unroll
        for (int r = 0; r < kSortItems; ++r) {
            const int64_t idx = wbase + r * 32 + lane;
            const bool ok = idx < n;
            key[r] = ok ? kin[idx] : 0ull;
            val[r] = ok ? vin[idx] : 0u;
            const int d = ok ? (int)((key[r] >> shift) & 0xFF) : 256;
            dig[r] = d;
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            const uint32_t before = ok ? wcount[w][d] : 0;
            loc[r] = before + __popc(peers & lane_lt());
            __syncwarp();
            const int leader = __ffs(peers) - 1;
            if (ok && lane == leader) wcount[w][d] = before + __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        uint32_t run = 0;
        {   // exclusive prefix over warps, per digit
            const int d = threadIdx.x;
#pragma unroll
            for (int q = 0; q < kSortThreads / 32; ++q) {
                const uint32_t t = wcount[q][d];
                wcount[q][d] = run;
                run += t;
            }
        }
        // and over digits: where each digit's run starts in the tile
        tdo[threadIdx.x] = block_exclusive_scan(run, wt, &tot);
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kSortItems; ++r) {
            const int d = dig[r];
            if (d < 256) {
                const uint32_t p = tdo[d] + wcount[w][d] + loc[r];
                skey[p] = key[r];
                sval[p] = val[r];
            }
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            const int i = j * kSortThreads + threadIdx.x;
            if (i < tile_n) {
                const unsigned long long k = skey[i];
                const int d = (int)((k >> shift) & 0xFF);
                const uint32_t pos = gbase[d] + (uint32_t)i - tdo[d];
                if ((int64_t)pos < n) {          // always true for a consistent histogram
                    kout[pos] = k;
                    vout[pos] = sval[i];
                }
            }
        }
        __syncthreads();                 // the shared arrays are reset for the next tile
    }
}

// out[i] = rec[perm[i]] (48-byte records as three 16-byte words).
__global__ void k_gather(const clight_hit *__restrict__ rec, const uint32_t *__restrict__ perm,
                         const unsigned long long *ctr, int64_t capacity, clight_hit *__restrict__ out)
{
    int64_t n = valid_hits(ctr, capacity);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t pi = perm[i];
        if ((int64_t)pi >= n) continue;      // always false for a consistent permutation
        const float4 *s = reinterpret_cast<const float4 *>(rec + pi);
        float4 *d = reinterpret_cast<float4 *>(out + i);
        float4 a = s[0], b = s[1], c = s[2];
        d[0] = a; d[1] = b; d[2] = c;
    }
}

__global__ void k_group_bounds(const unsigned long long *__restrict__ keys, const unsigned long long *ctr,
                               int64_t capacity, int group_shift, int64_t n_groups,
                               int64_t *__restrict__ gstart, int64_t *__restrict__ gend)
{
    int64_t n = valid_hits(ctr, capacity);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long g = keys[i] >> group_shift;
        if (g >= (unsigned long long)n_groups) continue;
        if (i == 0 || (keys[i - 1] >> group_shift) != g) gstart[g] = i;
        if (i == n - 1 || (keys[i + 1] >> group_shift) != g) gend[g] = i + 1;
    }
}

// Counts and binary64 photon sums per group, in a fixed order: thread t adds
// items t, t+256, ... in sequence, then a fixed tree joins the threads.
__global__ void __launch_bounds__(256)
k_group_sums(const clight_hit *__restrict__ hits, const int64_t *__restrict__ gstart,
             const int64_t *__restrict__ gend, int64_t n_groups, int64_t *__restrict__ counts,
             double *__restrict__ sums)
{
    __shared__ double red[256];
    for (int64_t g = blockIdx.x; g < n_groups; g += gridDim.x) {
        int64_t b = gstart[g], e = gend[g];
        double s = 0.0;
        for (int64_t i = b + threadIdx.x; i < e; i += 256) s += (double)hits[i].weight;
        red[threadIdx.x] = s;
        __syncthreads();
        for (int o = 128; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            if (counts) counts[g] = e - b;
            if (sums) sums[g] = red[0];
        }
        __syncthreads();
    }
}

cudaError_t radix_sort_pairs(unsigned long long **kin, uint32_t **vin, unsigned long long **kout, uint32_t **vout,
                             const unsigned long long *ctr, int64_t capacity, int key_bits, uint32_t *hist,
                             uint32_t *block_sums, int64_t tiles, cudaStream_t s)
{
    // grids bounded by the SM count: the kernels walk the live tiles
    const int n_sm = device_sms();
    int oh = 0, os = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&oh, k_radix_hist, kSortThreads, 0) != cudaSuccess) oh = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&os, k_radix_scatter, kSortThreads, 0) != cudaSuccess) os = 1;
    const unsigned gh = (unsigned)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)n_sm * std::max(oh, 1)));
    const unsigned gs = (unsigned)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)n_sm * std::max(os, 1)));
    for (int shift = 0; shift < key_bits; shift += 8) {
        k_radix_hist<<<gh, kSortThreads, 0, s>>>(*kin, ctr, capacity, shift, hist);
        cudaError_t e = exclusive_scan(hist, 256 * tiles, ctr, capacity, block_sums, 2 * n_sm, s);
        if (e != cudaSuccess) return e;
        k_radix_scatter<<<gs, kSortThreads, 0, s>>>(*kin, *vin, *kout, *vout, ctr, capacity, shift, hist);
        unsigned long long *tk = *kin; *kin = *kout; *kout = tk;
        uint32_t *tv = *vin; *vin = *vout; *vout = tv;
    }
    return cudaGetLastError();
}

cudaError_t launch_sort_and_finalize(const DevOut &O, const SortScratch &S, int key_bits, int group_shift,
                                     int64_t n_groups, clight_hit *out, int64_t *counts, double *sums,
                                     cudaStream_t s)
{
    const int64_t tiles = S.max_tiles;
    unsigned long long *kin = O.keys, *kout = S.keys_alt;
    uint32_t *vin = O.vals, *vout = S.vals_alt;
    cudaError_t e = radix_sort_pairs(&kin, &vin, &kout, &vout, O.ctr, O.capacity, key_bits, S.hist, S.block_sums,
                                     tiles, s);
    if (e != cudaSuccess) return e;
    const int gg = 4 * device_sms();
    k_gather<<<gg, 256, 0, s>>>(O.rec, vin, O.ctr, O.capacity, out);
    cudaMemsetAsync(S.gstart, 0, sizeof(int64_t) * n_groups, s);
    cudaMemsetAsync(S.gend, 0, sizeof(int64_t) * n_groups, s);
    k_group_bounds<<<gg, 256, 0, s>>>(kin, O.ctr, O.capacity, group_shift, n_groups, S.gstart, S.gend);
    if (counts || sums) {
        int64_t gb = n_groups < 65535 ? n_groups : 65535;
        k_group_sums<<<(unsigned)gb, 256, 0, s>>>(out, S.gstart, S.gend, n_groups, counts, sums);
    }
    return cudaGetLastError();
}

}  // namespace clight
