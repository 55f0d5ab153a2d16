// internal.h -- structures shared by the host side and the kernels of the
// clight library (not part of the public ABI).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/clight.h"

namespace clight {

constexpr int kMaxLayers = 8;
constexpr int kMaxCells = 64;
constexpr int kGLNodes = 3;

// One altitude cell of the ray quadrature: inside it the density is
// rho = B exp(-h/c) of a single layer, so delta = kb 2^(h nl2c) and
// rho/rho_ref = rb 2^(h nl2c).
struct DevCell {
    float lo, hi, kb, rb, nl2c, pad0, pad1, pad2;
};

// Atmosphere as the kernels see it (passed by value as a kernel parameter,
// so every access is a uniform constant-bank read).
struct DevAtm {
    int n_layers, n_cells, spherical, refraction, absorption, pad;
    float h_lo[kMaxLayers], kb[kMaxLayers], rb[kMaxLayers], nl2c[kMaxLayers];
    float kb_lo[kMaxLayers], nl2c_lo[kMaxLayers];   // low words: kb, nl2c as FP32 pairs
    double h_lo_d[kMaxLayers], kb_d[kMaxLayers], rb_d[kMaxLayers], inv_c_d[kMaxLayers];
    float h_top, h_obs, R_E, r_obs, inv_r_obs;  // binary32 copies
    double inv_r_obs_d;
    double h_top_d, h_obs_d, R_E_d, r_obs_d;  // binary64 copies
    float delta_obs, n_obs;                   // n(h_obs) - 1 and n(h_obs)
    double delta_obs_d;
    float delta_max;                          // largest n - 1 between h_obs and h_top
    float inv_L0, lambda_ref;                 // tau = I * (lambda_ref/lambda)^4 * inv_L0
    double inv_L0_d, lambda_ref_d;
    // the same constants as FP32 pairs (hi, lo), so that no ray converts binary64
    float hobs_hi, hobs_lo, re_hi, re_lo, k2_hi, k2_lo, invc_hi, invc_lo;  // h_obs, R_E, h_obs + 2 R_E, 1/c
    double k2_d;                              // h_obs + 2 R_E
    float gl_x[kGLNodes], gl_w[kGLNodes];     // Gauss-Legendre on [-1, 1]
    double gl_x_d[kGLNodes], gl_w_d[kGLNodes];
    // straight-line propagator: per layer c_i and the constants E_i, F_i of
    // int_h^top delta = c_i delta(h) + E_i, int_h^top rho/rho_ref = c_i rho(h)/rho_ref + F_i,
    // and both integrals from h_obs
    float lay_c[kMaxLayers], lay_E[kMaxLayers], lay_F[kMaxLayers];
    float D_obs, R_obs;
    // dispersion: n - 1 = delta(h) (1 + B/lambda^2) inv_g0
    int disp;
    float disp_B, disp_ig0;
    double disp_B_d, disp_ig0_d;
    DevCell cells[kMaxCells];
    double cell_lo_d[kMaxCells], cell_hi_d[kMaxCells], cell_kb_d[kMaxCells], cell_rb_d[kMaxCells],
        cell_ic_d[kMaxCells];                 // binary64 copies; ic = 1/c
};

// Telescopes and their uniform grid (device pointers owned by the context).
struct DevTel {
    const float4 *tel;          // x, y, z, R
    const int *cell_start;      // nx*ny + 1
    const int *cell_tel;        // telescope indices, grouped by cell
    int n_tel, nx, ny, pad;
    float gx0, gy0, gs, inv_gs; // grid origin and cell size
    float xmin, xmax, ymin, ymax, Rmax, zmin, zmax, pad2;
    // clearance map: per square cell of side cgs, a lower bound on the
    // distance from any point of the cell to the nearest telescope centre,
    // in units of kClrQuantum (255 = at least 255 units); nullptr if none
    const uint8_t *clr;
    int cnx, cny, clr_bytes, pad3;  // cells, bytes (a multiple of 16)
    float cx0, cy0, inv_cgs, pad4;
    float mx, my, mz, mr;           // mean centre, largest distance of a centre from it (rounded up)
    float cabs;                     // largest |x| + |y| + |z| of a centre
    // the same map at a finer cell (read from global memory by the classification)
    const uint8_t *fclr;
    int fcnx, fcny;
    float fcx0, fcy0, finv_cgs;
};
constexpr float kClrQuantum = 0.25f;     // metres per unit of the clearance map
constexpr int kClrMaxCells = 10240;      // 10 KB of shared memory per CTA
constexpr int kClrFineMaxCells = 524288; // 512 KB in global memory

struct DevPar {
    float band, inv_bunch;       // 2 pi alpha (1/l1 - 1/l2) [1/m], 1/B
    float fta;                   // 2 pi alpha 1e9 (the yield per unit of u = 1/lambda in 1/nm)
    double fta_d;
    double band_d, bunch_d;
    float il1, dil;              // 1/lambda1, 1/lambda1 - 1/lambda2 (1/nm)
    double il1_d, dil_d;
    float fl1, fdl;              // fluorescence band start and width (nm)
    double fl1_d, fdl_d;
    float fyield;                // photons per MeV
    double fyield_d;
    uint32_t seed, stream;
    int64_t seg_base;
    int64_t key_off;             // added to the launch-local step index in the sort keys (chunked launches)
    int n_showers, seg_bits, k_bits, pad;
    float bunch;
    // angular segment cut (CLIGHT_CUT_*): cos of the angle, the centre, and
    // for the per-telescope mode the telescope centres
    int cut_mode, cut_n_tel;
    float cut_cos;
    double cut_cos_d;
    float cut_cx, cut_cy, cut_cz;
    double cut_cx_d, cut_cy_d, cut_cz_d;
    const float4 *cut_tel;
    // per-telescope mode: the array's mean centre and the largest distance of
    // a telescope centre from it (rounded up), and the cut angle in radians
    float cut_tx, cut_ty, cut_tz, cut_tr, cut_rad;
    float cut_cabs;              // bound of |c|_1 over the cut's target centres
    // and the telescope grid (CSR), to try the telescopes near the point
    // where the step's line meets the array plane first
    const int *cut_cell_start, *cut_cell_tel;
    int cut_nx, cut_ny;
    float cut_gx0, cut_gy0, cut_inv_gs;
    int prop;                    // CLIGHT_PROP_*
    int cull;                    // 1: rays provably clear of every telescope skip the quadrature
    int chunk;                   // groups of 32 steps per work claim (two-pass first kernel)
    // fluorescence beaming: on/off, cone centre and radius
    int beam, roulette;
    float beam_cx, beam_cy, beam_cz, beam_r;
    double beam_cx_d, beam_cy_d, beam_cz_d, beam_r_d;
};

struct DevOut {
    clight_hit *rec;             // unsorted hit records (scratch)
    unsigned long long *keys;    // sort keys, parallel to rec
    uint32_t *vals;              // 0..n-1
    int64_t capacity;
    unsigned long long *ctr;     // [0] work counter, [1] hit cursor, [CTR_STATS..] statistics, [CTR_DEFER]
                                 // deferred rays, [CTR_DEFER_WORK] the deferred kernel's work counter
    float soft_w;                // candidate pass of the adjoint: aperture widening (m)
    // rays the fused kernel leaves to k_trace_deferred: (step << 32) | bunch,
    // the step counted from the launch's first; nullptr = trace every ray in place
    unsigned long long *defer;
    int64_t defer_cap;
};

// Offsets inside DevOut::ctr.
enum { ST_RAYS = 0, ST_ESCAPED, ST_UNDER, ST_TURNED, ST_REACHED, ST_HITS, ST_GUARDED, ST_STATUS, ST_CELLS, ST_CUT,
       ST_SKIPPED, ST_DEFERRED, ST_STEP_SKIPPED, ST_N };
enum { CTR_WORK = 0, CTR_CURSOR = 1, CTR_STATS = 2, CTR_DEFER = CTR_STATS + ST_N, CTR_DEFER_WORK = CTR_DEFER + 1,
       CTR_N = CTR_DEFER + 2 };
// Status bit (above the CLIGHT_ERR_* codes) of a launch whose deferred-ray
// queue filled; the host runs such a call again.
constexpr int kBitDeferFull = 30;

// Makes a device current for the life of an entry point and gives the
// caller's current device back when it returns.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            prev = -1;
            cudaGetLastError();
        }
        ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
    DeviceGuard(const DeviceGuard &) = delete;
    DeviceGuard &operator=(const DeviceGuard &) = delete;
};

// What the no-allocation entry point reads from a context (clight_api.cu).
struct CtxView {
    DevAtm atm;
    DevTel tel;
    DevPar par;
    int device, n_sm, block, ctas_per_sm, precision;
};
bool ctx_view(clight_ctx *c, CtxView *v);
// Per-context slots holding the device addresses of the no-allocation entry
// point's static arrays, [0] the scratch and [1] the deferred-ray queue
// (looked up on the context's first such call).
void **ctx_noalloc_slot(clight_ctx *c);

// kernel launchers (trace_twopass.cu, trace_inplace.cu, trace_noalloc.cu)
cudaError_t launch_trace_fused(const clight_segment *segs, int64_t n_segs, const DevAtm &A,
                               const DevTel &T, const DevPar &P, const DevOut &O, int precision,
                               int grid, int block, cudaStream_t s);
// Candidate pass of the soft-yield adjoint: every ray whose arrival line
// passes within R + O.soft_w of a telescope centre appends
// (local segment << 32 | bunch) to O.keys (capacity O.capacity, cursor
// O.ctr[CTR_CURSOR]).
cudaError_t launch_soft_candidates(const clight_segment *segs, int64_t n_segs, const DevAtm &A, const DevTel &T,
                                   const DevPar &Pp, const DevOut &O, int grid, int block, cudaStream_t s);
cudaError_t launch_trace_fp64(const clight_segment *segs, int64_t n_segs, const DevAtm &A,
                              const DevTel &T, const DevPar &P, const DevOut &O, cudaStream_t s);
int fused_smem_bytes(int block, const DevTel &T);

// tangent-linear adjoint (adjoint_kernels.cu)
int adjoint_params(int n_layers);   // tangents carried: >= n_layers + 2
// cand: the candidate rays (local step << P.k_bits | bunch), sorted; yfix:
// n_groups accumulators of the soft yield in units of 2^-24 photons, zeroed
// by the caller (integer sums: the same bits in any order), converted into
// yield when that is not NULL.
cudaError_t launch_adjoint(const clight_segment *segs, const unsigned long long *cand, int64_t n_cand,
                           const clight_hit *hits, int64_t n_hits,
                           const float *gx, const float *gy, const float *gt, const double *gY,
                           unsigned long long *yfix, double *yield, int64_t n_groups,
                           const DevAtm &A, const DevTel &T, const DevPar &P, float soft_s, float soft_w, float K,
                           float L0, double *partial, int blocks, double *d_out, cudaStream_t s);

// sort and finalize (sort_kernels.cu)
struct SortScratch {
    unsigned long long *keys_alt;
    uint32_t *vals_alt;
    uint32_t *hist;              // 256 * max_tiles
    uint32_t *block_sums;        // scan partials
    int64_t max_tiles;
    int64_t *gstart, *gend;      // per group
};
int sort_tile_items();
int64_t scan_block_sums_needed(int64_t n);
// Stable LSD radix sort of the first ctr[CTR_CURSOR] (key, value) pairs by
// the low key_bits bits of the key (nothing when that count exceeds
// capacity); the sorted pairs end in (*kin, *vin), the pointers swapped.
cudaError_t radix_sort_pairs(unsigned long long **kin, uint32_t **vin, unsigned long long **kout, uint32_t **vout,
                             const unsigned long long *ctr, int64_t capacity, int key_bits, uint32_t *hist,
                             uint32_t *block_sums, int64_t tiles, cudaStream_t s);
cudaError_t launch_sort_and_finalize(const DevOut &O, const SortScratch &S, int key_bits,
                                     int group_shift, int64_t n_groups, clight_hit *out,
                                     int64_t *counts, double *sums, cudaStream_t s);

}  // namespace clight
