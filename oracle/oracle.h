/*
 * oracle.h -- plain FP64 CPU oracle for Cherenkov / fluorescence photon
 * generation and atmospheric propagation to telescope spheres.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link
 * or call this code; only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark do.  It shares no code with the CUDA
 * library: the record layouts below are restated here as formats.
 *
 * What it computes (paper: Baack & Alameddine, "Comparison and efficiency of
 * GPU accelerated optical light propagation in CORSIKA 8", ICRC 2023):
 *   - Cherenkov yield of a track step by the Frank-Tamm formula with its
 *     threshold, n taken constant over the step (Sec. 1.2);
 *   - fluorescence yield N = Y * dE (Eq. 1, Sec. 1.1), isotropic emission;
 *   - photon generation: cone vector p rotated by M_Rod (Sec. 1.2.1, Fig. 1)
 *     and moved to a uniformly drawn emission point (Sec. 1.1, 1.2);
 *   - propagation to the observation level (Sec. 2) through a layered
 *     exponential atmosphere, written out as the exact refracted ray of a
 *     stratified medium (Snell / Bouguer invariant) by adaptive quadrature;
 *   - the telescope-sphere hit test and sorted per-telescope lists.
 *
 * Units: metres, nanoseconds, nanometres, g/cm^3, MeV.
 */
#ifndef CLIGHT_ORACLE_H
#define CLIGHT_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {            /* 64 bytes, same byte layout as the inputs */
    double x, y, z, t0;
    float dx, dy, dz, L, eps, dE;
    int32_t charge;
    uint32_t shower;
} or_segment;

typedef struct {            /* 16 bytes */
    float x, y, z, R;
} or_telescope;

typedef struct {
    int n_layers;                 /* 1..8 */
    double h_lo[8], b[8], c[8];   /* rho = b/(100 c) exp(-h/c) on [h_lo[i], h_lo[i+1]) */
    double h_top;                 /* rho = 0 above */
    double K;                     /* n - 1 = K rho */
    double rho_ref;               /* density normalising the optical depth */
    double L0, lambda_ref;        /* extinction length L0 (lambda/lambda_ref)^4 */
    double R_E, h_obs;
    int spherical, refraction, absorption;
    /* dispersion (reading): n(lambda, h) - 1 = delta(h) g(lambda),
     * g = (1 + B/lambda^2) / (1 + B/lambda_d^2); B = 0: none */
    double disp_B, disp_lref;     /* nm^2, nm */
} or_atmosphere;

typedef struct {
    double lambda1, lambda2;      /* Cherenkov band, nm */
    double bunch;                 /* maximum photons per bunch */
    uint32_t seed, stream;        /* Philox key */
    double fluor_yield;           /* photons per MeV deposited (0 = off) */
    double fl_lambda1, fl_lambda2;
    int64_t seg_base;             /* global index of segs[0] (Philox counter) */
    /* Cherenkov angular segment cut (Sec. 1.2.1, optimisation):
     * 0 off, 1 array centre, 2 each telescope */
    int32_t cut_mode;
    double cut_deg;               /* degrees (0 = 6) */
    double cut_centre[3];         /* mode 1 */
    const or_telescope *cut_tels; /* mode 2 */
    int32_t cut_n_tel;
    /* fluorescence beaming (Sec. 1.1.1, optimisation) */
    int32_t fl_beaming;
    double beam_centre[3];
    double beam_radius;
    /* fluorescence count rule: 0 ceil(N/B); 1 N < B -> one bunch of weight B
     * with probability N/B (Philox counter (step, 0xFFFFFFFF, 1)) */
    int32_t fl_roulette;
} or_params;

typedef struct {            /* oracle output record, all FP64 */
    int64_t seg;
    uint32_t k, tel;
    double x_rel, y_rel, cx, cy, lambda, weight, t, dperp;
} or_hit;

enum { OR_TRACED = 0, OR_ESCAPED = 1, OR_UNDER = 2, OR_TURNED = 3 };

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11). */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double or_u01(uint32_t x);

/* out: n_c, w_c, n_f, w_f, cos_tc, sin_tc, Nbar_c, Nbar_f, delta_mid, h_mid */
void or_yield(const or_segment *s, const or_atmosphere *a, const or_params *p, double out[10]);
/* The same for the step of global index seg_index (the fluorescence count
 * rule 1 draws a number keyed by it; or_yield uses p->seg_base). */
void or_yield_at(const or_segment *s, int64_t seg_index, const or_atmosphere *a, const or_params *p,
                 double out[10]);

/* Rotation M_Rod for track direction d (normalised inside), row-major. */
void or_rotation(const double d[3], double M[9]);

/* Photon of bunch k: out = r_e[3], d[3], t_e, lambda, weight, process. */
void or_photon(const or_segment *s, int64_t seg_index, uint32_t k,
               const or_atmosphere *a, const or_params *p, double out[10]);

/* out: status, P[3], dL[3], t_L, tau, n_obs */
void or_propagate(const or_atmosphere *a, const double r_e[3], const double d[3],
                  double t_e, double lambda, double out[10]);

/* Refractive-index excess and density at altitude h. */
double or_delta(const or_atmosphere *a, double h);
/* The dispersion factor g(lambda) (1 without dispersion). */
double or_disp_g(const or_atmosphere *a, double lambda);
double or_density(const or_atmosphere *a, double h);

/* Full trace.  Writes at most `capacity` hits, sorted by
 * (shower, telescope, segment, bunch); returns the number of hits (may exceed
 * capacity, in which case nothing beyond capacity is written).
 * stats[0..4] = rays, escaped, under, turned, reached.
 * counts/sums (n_showers * n_tel) may be NULL.  threads <= 0: default. */
int64_t or_trace(const or_segment *segs, int64_t n_segs,
                 const or_atmosphere *a, const or_telescope *tels, int n_tel,
                 const or_params *p, int n_showers,
                 or_hit *hits, int64_t capacity,
                 int64_t *counts, double *sums, int64_t *stats, int threads);

/* Soft-edged yield of every (shower, telescope) with the given aperture
 * softness s (m) and cut W (m): sum over rays with d_perp < R + W of
 * w e^{-tau} sigma((R - d_perp)/s).  Bunch counts are supplied (frozen). */
void or_soft_yield(const or_segment *segs, int64_t n_segs, const uint32_t *n_bunch_c,
                   const uint32_t *n_bunch_f, const or_atmosphere *a,
                   const or_telescope *tels, int n_tel, const or_params *p,
                   int n_showers, double s, double W, double *yield, int threads);

/* Re-evaluate listed rays (seg, k, tel) with frozen bunch counts: out per
 * ray = x_rel, y_rel, t, weight*e^{-tau}, dperp. */
void or_eval_rays(const or_segment *segs, const int64_t *seg_idx, const uint32_t *k,
                  const uint32_t *tel, const uint32_t *n_bunch_c, const uint32_t *n_bunch_f,
                  int64_t n, const or_atmosphere *a, const or_telescope *tels,
                  const or_params *p, double *out, int threads);

#ifdef __cplusplus
}
#endif
/* FP64 reference gradient by forward-mode dual numbers (parameters
 * c_1..c_L, K, L0; grad has n_layers + 2 entries).  or_grad_rays: of
 * sum gx x_rel + gy y_rel + gt t + gw weight over the given hits (gx, gy,
 * gt, gw may be NULL); or_grad_soft: of sum gY_g Y_g for the soft yield. */
void or_grad_rays(const or_segment *segs, const int64_t *seg_idx, const uint32_t *k, const uint32_t *tel,
                  const uint32_t *n_bunch_c, const uint32_t *n_bunch_f, int64_t n, const or_atmosphere *a,
                  const or_telescope *tels, const or_params *p, const double *gx, const double *gy,
                  const double *gt, const double *gw, double *grad, int threads);
void or_grad_soft(const or_segment *segs, int64_t n_segs, const uint32_t *n_bunch_c, const uint32_t *n_bunch_f,
                  const or_atmosphere *a, const or_telescope *tels, int n_tel, const or_params *p, int n_showers,
                  double s, double W, const double *gY, double *grad, int threads);

#endif
