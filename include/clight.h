/*
 * clight.h -- C ABI of the GB300 (sm_103a) library for Cherenkov and
 * fluorescence light generation and atmospheric propagation to telescopes.
 *
 * The calls follow the paper's statement of the problem (Baack &
 * Alameddine, "Comparison and efficiency of GPU accelerated optical light
 * propagation in CORSIKA 8", ICRC 2023): charged-particle track steps go in
 * (Sec. 1.2), together with the atmosphere the light crosses (Sec. 1.2,
 * Sec. 2) and the telescope array it lands on; photon bunches come out as
 * per-telescope hit lists, counts and photon sums (Sec. 1, "common memory
 * block" of photon data; Sec. 2, propagation to ground).
 *
 * Conventions
 *  - Pointers named d_* are device pointers owned by the caller; h_* are host
 *    pointers owned by the caller.  The library owns its context: the
 *    atmosphere tables, the telescope grid, scratch buffers and CUDA graphs.
 *  - Every call is ordered on the CUDA stream passed as `stream`
 *    (a cudaStream_t; NULL = legacy default stream).  Calls that return host
 *    results synchronise that stream once before returning.
 *  - Errors are return codes; nothing aborts, throws or faults the GPU to
 *    signal an error.  clight_status_string() names each code.
 *  - A context is used by one host thread and one stream at a time.
 *  - Every call makes the context's device current while it runs and makes
 *    the caller's current device current again before it returns.
 *  - Units: metres, nanoseconds, nanometres, g/cm^3, MeV.
 *
 * Limits: at most 8 atmosphere layers, 64 quadrature cells, 2^31 segments
 * per call, 2^24 telescopes x showers, and a sort key of 64 bits holding
 * (shower*n_tel + tel, segment, bunch).  A bunch index that does not fit
 * the key returns CLIGHT_ERR_LIMIT.
 */
#ifndef CLIGHT_H
#define CLIGHT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CLIGHT_OK = 0,
    CLIGHT_ERR_ARG = 1,           /* invalid argument (null, negative size, bad table) */
    CLIGHT_ERR_CUDA = 2,          /* a CUDA runtime call failed */
    CLIGHT_ERR_HIT_CAPACITY = 3,  /* more hits than hit_capacity; *h_n_hits = required */
    CLIGHT_ERR_BAD_SEGMENT = 4,   /* NaN/inf field, L < 0, zero direction, shower >= n_showers */
    CLIGHT_ERR_LIMIT = 5,         /* a size or index exceeds a documented limit */
    CLIGHT_ERR_NO_DEVICE = 6      /* no usable CUDA device */
} clight_status;

/* Charged-particle track step (64 bytes, little endian).  Sec. 1.2: steps of
 * "a couple of meters" over which the atmosphere is taken as homogeneous. */
typedef struct {
    double x, y, z;     /* start of the step, local frame (z up, origin at sea
                           level below the array centre), m */
    double t0;          /* time at the start of the step, ns */
    float dx, dy, dz;   /* direction of flight; normalised by the library */
    float L;            /* step length, m (>= 0) */
    float eps;          /* 1 - beta of the particle */
    float dE;           /* energy deposited over the step, MeV (fluorescence) */
    int32_t charge;     /* charge number z */
    uint32_t shower;    /* shower index, < n_showers */
} clight_segment;

/* Telescope sphere (16 bytes). */
typedef struct {
    float x, y, z, R;   /* centre (m) and radius (m) */
} clight_telescope;

/* Layered exponential atmosphere: on [h_lo[i], h_lo[i+1]) the density is
 * rho_i(h) = b_i / (100 c_i) exp(-h / c_i) g/cm^3 (b_i in g/cm^2, c_i in m),
 * zero at and above h_top; n - 1 = K rho.  Extinction length
 * L_ext(lambda) = L0 (lambda / lambda_ref)^4; optical depth
 * tau = int rho / rho_ref ds / L_ext. */
typedef struct {
    int32_t n_layers;               /* 1..8, h_lo increasing */
    int32_t spherical;              /* 0 = flat Earth, 1 = spherical Earth of radius R_E */
    double h_lo[8], b[8], c[8];
    double h_top;                   /* top of the atmosphere, m */
    double K;                       /* refractivity per density, cm^3/g */
    double rho_ref;                 /* density normalising tau, g/cm^3 */
    double L0;                      /* extinction length at lambda_ref, m */
    double lambda_ref;              /* nm */
    double R_E;                     /* Earth radius, m */
    double h_obs;                   /* observation level, m */
    int32_t refraction;             /* 1 = refracted rays, 0 = straight lines */
    int32_t absorption;             /* 1 = weight photons by exp(-tau) */
    /* Dispersion (Sec. 1.2 keeps n(lambda) inside the Frank-Tamm integral;
     * the form is a stated reading): n(lambda, h) - 1 = delta(h) g(lambda),
     * g = (1 + disp_B / lambda^2) / (1 + disp_B / disp_lref^2), delta(h) the
     * refractivity of the layers at disp_lref.  The yield integrates over
     * the band above threshold, each photon takes its own wavelength and
     * Cherenkov angle, and its ray sees delta(h) g(lambda).  disp_B = 0:
     * no dispersion.  Not supported by clight_trace_adjoint. */
    double disp_B;                  /* nm^2, >= 0 */
    double disp_lref;               /* nm, > 0 when disp_B > 0 */
} clight_atmosphere;

/* Precision of the fused FP32 path's few extended-precision steps. */
enum {
    CLIGHT_PREC_FLOAT_PAIR = 0,     /* FP32 pairs (double-float) -- default */
    CLIGHT_PREC_FP64_GUARD = 1      /* native FP64 for the same steps */
};

/* Cherenkov angular segment cut (Sec. 1.2.1, optimisation): a step emits
 * no Cherenkov light when its flight direction makes more than cut_deg with
 * the direction from its midpoint to the array centre (CENTRE) or to every
 * telescope centre (TELESCOPES).  Fluorescence is not affected. */
enum {
    CLIGHT_CUT_OFF = 0,
    CLIGHT_CUT_CENTRE = 1,
    CLIGHT_CUT_TELESCOPES = 2
};

typedef struct {
    double lambda1, lambda2;        /* Cherenkov band, nm */
    double bunch;                   /* maximum photons per bunch (> 0) */
    uint32_t seed, stream;          /* Philox-4x32-10 key words */
    double fluor_yield;             /* photons per MeV deposited; 0 = no fluorescence */
    double fl_lambda1, fl_lambda2;  /* fluorescence band, nm */
    int64_t seg_base;               /* global index of d_segs[0] (keys the random numbers) */
    int32_t precision;              /* CLIGHT_PREC_* */
    int32_t block;                  /* threads per block of the fused kernel (0 = default) */
    int32_t ctas_per_sm;            /* persistent CTAs per SM (0 = default) */
    int32_t use_graph;              /* capture the whole pipeline in a CUDA graph and replay */
    float cell_width;               /* quadrature cell width in scale heights (0 = 1.5) */
    int32_t key_bunch_bits;         /* bits of the bunch index in the sort key (0 = 16) */
    int32_t cut_mode;               /* CLIGHT_CUT_* */
    int32_t cut_pad;
    double cut_deg;                 /* cut angle in degrees, (0, 180) (0 = 6) */
    double cut_centre[3];           /* array centre for CLIGHT_CUT_CENTRE, m, local frame */
    /* Fluorescence beaming (Sec. 1.1.1, optimisation): when on, a step whose
     * midpoint m lies at D = |C - m| >= 2 beam_radius from beam_centre C emits
     * its fluorescence only into the cone about C - m of half-angle
     * alpha = asin(beam_radius / D) + 5e-3 + L / D, uniformly in solid angle,
     * and its photon number is scaled by the cone's share sin^2(alpha / 2).
     * beam_radius must hold every telescope sphere (centre distance + R). */
    int32_t fl_beaming;             /* 0 off, 1 on */
    /* Propagator (Sec. 2): CLIGHT_PROP_EXACT integrates the refracted ray's
     * deviation from the vacuum line; CLIGHT_PROP_STRAIGHT keeps the vacuum
     * line and applies first-order corrections in n - 1 (closed forms per
     * exponential layer, evaluated with the zenith angle at emission): the
     * paper's straight line plus refraction corrections, approximate. */
    int32_t propagator;
    double beam_centre[3];          /* m, local frame */
    double beam_radius;             /* m */
    /* Count rule of the fluorescence bunches: 0 = ceil(N / B) bunches of
     * weight N / n_b (every step with N > 0 emits at least one); 1 = a step
     * with N < B emits one bunch of weight B with probability N / B (its own
     * Philox draw, counter (step, 0xFFFFFFFF, 1)), else none; N >= B as for 0.
     * The expected photon number is the same; with beaming it is what turns
     * the smaller photon numbers into fewer rays. */
    int32_t fl_roulette;
    int32_t roulette_pad;
    /* Entries of the deferred-ray queue.  The fused kernel first decides,
     * from each ray's vacuum line, whether it can land near a telescope;
     * rays that can are queued and traced in full by a second kernel in
     * full warps.  0 = 2 per step (at least 2^20, at most 2^28, 8 bytes
     * each), launches of at most half as many steps; a call that fills it
     * runs again with twice the queue (remembered by the context, at most
     * 2^31 entries), then without it.  > 0 = that many entries (<= 2^31); a
     * call that fills them runs again without the queue.  < 0 = no queue:
     * every ray is traced in the fused kernel.  The hits are the same in
     * every case.  Without device memory for the queue the call runs
     * without it. */
    int64_t defer_cap;
    /* 1 = every ray traced in full in the fused kernel: no first pass and no
     * skip of the rays that provably land clear of every telescope -- the
     * same algorithm as clight_trace_fp64, for measurements.  The hits are
     * the same.  0 = default. */
    int32_t trace_all;
    /* Work stealing of the two-pass path's first kernel: a warp claims
     * work_chunk groups of 32 steps per atomic (0 = 1; at most 64). */
    int32_t work_chunk;
} clight_params;

enum {
    CLIGHT_PROP_EXACT = 0,
    CLIGHT_PROP_STRAIGHT = 1
};

/* One telescope hit (48 bytes). */
typedef struct {
    int64_t seg;                    /* global segment index (seg_base + i) */
    uint32_t k;                     /* bunch index within the segment (Cherenkov first) */
    uint32_t tel;                   /* telescope index */
    float x_rel, y_rel;             /* crossing of the plane z = z_tel, relative to the centre, m */
    float cx, cy;                   /* direction cosines at arrival */
    float lambda;                   /* wavelength, nm */
    float weight;                   /* photons in the bunch times exp(-tau) */
    double t;                       /* arrival time at that crossing, ns */
} clight_hit;

typedef struct {
    int64_t rays;       /* bunches generated and traced */
    int64_t escaped;    /* pointing away from the Earth */
    int64_t under;      /* emitted at or below the observation level */
    int64_t turned;     /* never reach the observation level */
    int64_t reached;    /* arrived at the observation level */
    int64_t hits;       /* ray-telescope hits (a ray may hit several) */
    int64_t guarded;    /* segments whose bunch count was recomputed in FP64 */
    int64_t status;     /* OR of CLIGHT_ERR_* bits seen in the kernels (1 << code) */
    int64_t cells;      /* altitude cells integrated, summed over arrived rays */
    int64_t cut;        /* steps whose Cherenkov light the angular cut removed */
    int64_t skipped;    /* arrived rays that provably land clear of every telescope,
                           decided from their vacuum line (no quadrature, no landing) */
    int64_t deferred;   /* rays the second pass of the two-pass path traced in full
                           (0 for a call traced in place) */
    int64_t step_skipped; /* of `skipped`, the rays of steps whose whole Cherenkov cone
                             the first pass showed to land clear of the array (decided
                             per step; these rays are never drawn) */
} clight_stats;

typedef struct clight_ctx clight_ctx;

/* Create a context on CUDA device `device`.  Allocates nothing large yet.
 * Returns CLIGHT_ERR_NO_DEVICE if the device cannot be used. */
clight_status clight_create(clight_ctx **out, int device);

/* Destroy a context and free everything it owns.  NULL is accepted. */
void clight_destroy(clight_ctx *ctx);

/* Copy the atmosphere model (host struct) into the context and build the
 * altitude cells of the ray quadrature.  ERR_ARG on an invalid table. */
clight_status clight_set_atmosphere(clight_ctx *ctx, const clight_atmosphere *atm);

/* Copy n telescopes (host array) into the context and build their uniform
 * grid.  ERR_ARG if n < 1 or a radius is not positive. */
clight_status clight_set_telescopes(clight_ctx *ctx, const clight_telescope *h_tels, int32_t n);

/* Set generation and launch parameters.  ERR_ARG on an invalid value. */
clight_status clight_set_params(clight_ctx *ctx, const clight_params *par);

/* Generate, propagate and hit-test every photon bunch of n_segs segments
 * (Sec. 1.1, 1.2, 2) on the fused FP32 path: one persistent work-stealing
 * launch over the segments, then a sort of the hits by
 * (shower, telescope, segment, bunch) and per-(shower, telescope) counts and
 * FP64 photon sums.
 *   d_segs        n_segs segments (device, read only, 16-byte aligned: a
 *                 misaligned array is refused with CLIGHT_ERR_ARG; this holds
 *                 for every entry point that takes d_segs)
 *   d_hits        hit_capacity records (device); the first *h_n_hits are
 *                 written, sorted
 *   d_counts      n_showers * n_tel int64 (device) or NULL
 *   d_sums        n_showers * n_tel double (device) or NULL
 *   h_stats       statistics (host) or NULL
 *   h_n_hits      number of hits (host); on CLIGHT_ERR_HIT_CAPACITY the
 *                 required capacity, and nothing beyond hit_capacity is
 *                 written, counts and sums are left zero.
 * Synchronises `stream` once.  Kernel-detected input errors are returned as
 * CLIGHT_ERR_BAD_SEGMENT / CLIGHT_ERR_LIMIT after the run. */
clight_status clight_trace(clight_ctx *ctx, const clight_segment *d_segs, int64_t n_segs,
                           int32_t n_showers, clight_hit *d_hits, int64_t hit_capacity,
                           int64_t *d_counts, double *d_sums, clight_stats *h_stats,
                           int64_t *h_n_hits, void *stream);

/* The same computation with FP64 arithmetic throughout: one thread per
 * segment, no work stealing, no graph (the plain double-precision path the
 * fused one is measured against).  Same arguments and outputs. */
clight_status clight_trace_fp64(clight_ctx *ctx, const clight_segment *d_segs, int64_t n_segs,
                                int32_t n_showers, clight_hit *d_hits, int64_t hit_capacity,
                                int64_t *d_counts, double *d_sums, clight_stats *h_stats,
                                int64_t *h_n_hits, void *stream);

/* clight_trace on HOST buffers, results copied back to h_hits / h_counts /
 * h_sums (the last two may be NULL).  How the steps reach the GPU:
 *   - at least 2 x 2^22 steps: copied in chunks of 2^22 steps on a second
 *     stream while earlier chunks are traced (from page-locked memory the
 *     copies run at the link's DMA rate, about 210 GB/s on GB300);
 *   - otherwise one copy, then the trace.
 * Device staging buffers are owned by the context.  Same results in every
 * case.  Synchronises `stream`. */
clight_status clight_trace_host(clight_ctx *ctx, const clight_segment *h_segs, int64_t n_segs,
                                int32_t n_showers, clight_hit *h_hits, int64_t hit_capacity,
                                int64_t *h_counts, double *h_sums, clight_stats *h_stats,
                                int64_t *h_n_hits, void *stream);

/* Gradient of a scalar loss with respect to the atmosphere parameters
 * theta = (c_1 .. c_L, K, L0): the layer scale heights, the refractivity
 * coefficient and the extinction length (b_i, layer edges, the random
 * numbers and the bunch counts held at their values of the forward call).
 *   loss = sum_hits (gx x_rel + gy y_rel + gt t)
 *        + sum_(shower, tel) gY Y,
 *   Y = sum over rays with d_perp < R + soft_w of
 *       weight exp(-tau) sigma((R - d_perp) / soft_s), sigma logistic,
 * the soft-edged absorption-weighted yield of each telescope.
 *   d_hits        the hits of clight_trace at the same parameters (device)
 *   d_gx/gy/gt    per-hit upstream gradients (device float, NULL = zero)
 *   d_gyield      per-(shower, tel) upstream gradients of Y (device double,
 *                 NULL = zero)
 *   d_yield       if not NULL receives Y (device double, n_showers * n_tel)
 *   h_grad        n_layers + 2 doubles (host): d loss / d theta
 * Each ray is recomputed from its random-number counter; derivatives are
 * carried as binary32 tangents and summed per block in binary64, then over
 * blocks in a fixed order.  The rays near a telescope (those within
 * R + soft_w of a centre) are listed by a candidate pass and sorted before
 * the tangent kernels run, so every thread sees the same rays in the same
 * order on every call, and Y is summed in integer units of 2^-24 photons
 * (at most 2^39 photons per shower and telescope): h_grad and d_yield are
 * bitwise reproducible.  Synchronises `stream` once or twice.  The tangents
 * are those of the exact propagator without dispersion: with dispersion on
 * or CLIGHT_PROP_STRAIGHT set it returns CLIGHT_ERR_ARG.  A bunch index
 * beyond 2^16 (the key_bunch_bits of clight_params) returns
 * CLIGHT_ERR_LIMIT. */
clight_status clight_trace_adjoint(clight_ctx *ctx, const clight_segment *d_segs, int64_t n_segs,
                                   int32_t n_showers, const clight_hit *d_hits, int64_t n_hits,
                                   const float *d_gx, const float *d_gy, const float *d_gt,
                                   const double *d_gyield, float soft_s, float soft_w, double *d_yield,
                                   double *h_grad, void *stream);

/* clight_trace without any allocation, for callers that cannot call
 * cudaMalloc while they run: code that must not touch the CUDA allocator
 * (an embedding framework that owns all device memory through its own
 * pool, a host process that reserves everything at start-up, a pipeline
 * whose memory budget must not move between events).  The paper has no
 * counterpart; it exists for such callers.
 *
 * It keeps no sort keys: the hit records go straight into d_hits in
 * arbitrary order (not sorted, no photon sums), and d_counts (optional,
 * n_showers * n_tel int64, device) receives the per-(shower, telescope)
 * hit counts.  With the default feature set (spherical, refracting
 * atmosphere, exact propagator, float-pair precision, no cut, beaming or
 * dispersion) it runs clight_trace's two passes, 2^24 steps at a time, with
 * a static queue of 2^22 rays; a chunk whose rays overflow the queue is
 * traced again by the in-place kernel.  Otherwise it runs the in-place
 * kernel (every ray traced where it is generated).  Its scratch --
 * counters, ray statistics, one hit counter per group and a copy of these
 * taken before each chunk -- and the queue are static arrays in the
 * library image (262,416 + 33,554,432 bytes, held on every GPU that loads
 * the library until the process exits).
 *   - n_showers * n_tel above 16384 returns CLIGHT_ERR_LIMIT before any
 *     launch; other errors as clight_trace.
 *   - The first call with a context looks up the arrays' device addresses
 *     (with the context's device current) and keeps them in the context.
 *   - The call reads its counters back to the host and synchronises
 *     `stream`, so it cannot run inside a stream capture: on a capturing
 *     stream it returns CLIGHT_ERR_ARG before doing anything, and the
 *     caller's capture is left intact.
 *   - Calls share the one array, which keeps the last call's contents; each
 *     call clears what must start at zero.  Calls that overlap on the GPU
 *     (different streams or threads) race on it: order them.
 *   - The context must already hold its atmosphere and telescopes (their
 *     tables were allocated by clight_set_*); this call allocates nothing.
 * Synchronises `stream` once, and once more per chunk of the two passes. */
clight_status clight_trace_noalloc(clight_ctx *ctx, const clight_segment *d_segs, int64_t n_segs,
                                   int32_t n_showers, clight_hit *d_hits, int64_t hit_capacity,
                                   int64_t *d_counts, clight_stats *h_stats, int64_t *h_n_hits, void *stream);

/* Result of clight_autotune. */
typedef struct clight_tune {
    int32_t block;          /* chosen threads per CTA */
    int32_t ctas_per_sm;    /* chosen persistent CTAs per SM (0 = the path's default) */
    float cell_width;       /* chosen quadrature cell width (scale heights) */
    int32_t work_chunk;     /* chosen groups of 32 steps per work claim */
    double bunch;           /* chosen bunch size (<= the caller's maximum) */
    double best_ms;         /* median step time of the chosen settings on the sample */
    double default_ms;      /* the same for the library defaults at the caller's bunch size */
    int32_t n_tried;        /* settings timed */
    int32_t pad;
    int64_t n_sample;       /* steps in the sample */
} clight_tune;

/* Pick the bunch size, launch shape, work-stealing granularity and
 * quadrature cell width for a batch (the batching pattern of the forward
 * path: one persistent launch over many showers).  Paper: no counterpart;
 * the paper's GPU code has fixed launch parameters.
 *   - The sample: n_sample steps in 64 blocks spread evenly over all n_segs
 *     steps of d_segs (so every shower of a batch contributes in proportion
 *     to its size), copied into context memory; all of d_segs when
 *     n_sample >= n_segs.
 *   - Each setting is timed as the median of `reps` (>= 1; 5 or more
 *     recommended) calls of the whole step (trace, sort, per-telescope
 *     reduction; no graph) after one warm-up call.
 *   - The library defaults (at the caller's bunch size, capped at
 *     bunch_max) are the first incumbent.  Then one knob at a time: bunch
 *     size in {1, 2, 5, bunch_max} (<= bunch_max), block x CTAs per SM in
 *     {256x4, 256x3, 128x8, 128x6, 64x16}, work chunk in {2, 4}, cell width
 *     1.0 (never wider than the default 1.5, whose accuracy the tests
 *     establish).  A candidate replaces the incumbent only when its median
 *     is lower by more than the incumbent's spread (interquartile range for
 *     5 or more calls, else the range) and by more than 1%.  So best_ms <=
 *     default_ms.  The photon count of a batch does not depend on the
 *     bunch size, so the fastest setting carries the most photons per
 *     second.
 *   - d_hits / hit_capacity: scratch for the sample's hits (the caller's
 *     buffer; overflow only truncates the sample's list and is ignored).
 *   - On success the context keeps the chosen settings (as if set by
 *     clight_set_params with the other fields unchanged) and *out holds
 *     them.  ERR_ARG for a bad argument (bunch_max <= 0, n_sample < 1,
 *     n_segs < 1, reps < 1, NULL out); the context's settings are unchanged
 *     on error.
 * Synchronises `stream`. */
clight_status clight_autotune(clight_ctx *ctx, const clight_segment *d_segs, int64_t n_segs, int64_t n_sample,
                              int32_t n_showers, clight_hit *d_hits, int64_t hit_capacity, double bunch_max,
                              int32_t reps, clight_tune *out, void *stream);

/* Measured instruction throughput of the GPU (operations per second, all
 * SMs), and the mean SM clock during each probe (MHz, from clock64() against
 * the global timer on the device).  The tracing path is bound by arithmetic
 * issue, so these -- not a copy bandwidth or a GEMM rate -- are its roofline
 * denominators.  The paper has no counterpart. */
typedef struct {
    double ffma_per_s;      /* FP32 fused multiply-add (one operation each) */
    double mufu_ex2_per_s;  /* MUFU ex2.approx (the special-function unit) */
    double dfma_per_s;      /* FP64 fused multiply-add */
    double imad_per_s;      /* 32-bit integer multiply-add */
    double lop3_per_s;      /* 3-input logic operation */
    double ffma_mhz, mufu_mhz, dfma_mhz, imad_mhz, lop3_mhz;
    int32_t n_sm;
    int32_t pad;
} clight_pipe_rates;

/* Run the throughput probes on `device` (each: 8 independent chains of one
 * instruction per thread in a grid that fills every SM; best of 3 timed
 * launches after a warm-up, CUDA events; a few milliseconds each).  Changes
 * no GPU setting.  Allocates and frees a small scratch buffer.
 * CLIGHT_ERR_NO_DEVICE without the device, CLIGHT_ERR_CUDA on a runtime
 * error. */
clight_status clight_measure_pipes(int device, clight_pipe_rates *out);

/* Device time of the last clight_trace / clight_trace_fp64 call, measured
 * with CUDA events recorded on the launch stream around its phases:
 * ms[0] = generation + propagation + hit kernel, ms[1] = sort and per-
 * telescope reduction.  ERR_ARG if ms is NULL or no call has run. */
clight_status clight_last_timing(clight_ctx *ctx, float ms[2]);

/* The last clight_trace_adjoint call of the context: the candidate rays of
 * the soft-yield term (rays whose arrival line passes within R + soft_w of a
 * centre; 0 without d_gyield / d_yield), the hits it was given, and the
 * device time of its phases from CUDA events on its stream: ms[0] candidate
 * pass, ms[1] candidate sort, ms[2] tangent kernels and the fixed-order
 * sums.  Any pointer may be NULL.  ERR_ARG if no adjoint call has completed
 * on the context. */
clight_status clight_last_adjoint(clight_ctx *ctx, int64_t *h_candidates, int64_t *h_hits, float ms[3]);

/* Human-readable name of a status code (static string). */
const char *clight_status_string(clight_status s);

/* Version of this ABI (major * 10000 + minor * 100 + patch). */
int clight_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CLIGHT_H */
