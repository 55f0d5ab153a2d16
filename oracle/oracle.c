/*
 * oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY; see oracle.h).
 *
 * Every function states the passage of Baack & Alameddine (ICRC 2023) it
 * follows.  Where the paper is silent the reading used is stated in place.
 * Nothing here is blocked, fused or reordered for speed: each ray is built,
 * propagated and tested against every telescope in turn.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static const double OR_PI = 3.14159265358979323846;
static const double OR_ALPHA = 7.2973525643e-3;   /* fine-structure constant */
static const double OR_C = 0.299792458;           /* speed of light, m/ns */

/* ------------------------------------------------------------------------
 * Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64 bit
 * multiplications (constants 0xD2511F53, 0xCD9E8D57) with a Weyl key
 * schedule (0x9E3779B9, 0xBB67AE85).
 * ---------------------------------------------------------------------- */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)p1;
        uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)p0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Top 23 bits, centred in their cell: (m + 1/2) 2^-23 needs 24 significand
 * bits, so the same uniform is exactly representable in binary32 and
 * binary64 and both precisions see the same number. */
double or_u01(uint32_t x)
{
    return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0);
}

/* ------------------------------------------------------------------------
 * Atmosphere: rho_i(h) = b_i / c_i exp(-h / c_i) per layer, n - 1 = K rho.
 * The paper states only that the medium is inhomogeneous and treated as
 * homogeneous over one track step (Sec. 1.2); the layered exponential form is
 * the workload's model.
 * ---------------------------------------------------------------------- */
static int layer_of(const or_atmosphere *a, double h)
{
    int i = 0;
    for (int j = 1; j < a->n_layers; j++)
        if (h >= a->h_lo[j]) i = j;
    return i;
}

double or_density(const or_atmosphere *a, double h)
{
    if (h >= a->h_top) return 0.0;
    int i = layer_of(a, h);
    return a->b[i] / (100.0 * a->c[i]) * exp(-h / a->c[i]);
}

double or_delta(const or_atmosphere *a, double h)
{
    return a->K * or_density(a, h);
}

/* h = |r + R_E z| - R_E, written as (x^2 + y^2 + z (z + 2 R_E)) /
   (|r + R_E z| + R_E): the same quantity without subtracting two numbers of
   6.4e6 m (which would lose ~1e-9 m, and near the Cherenkov threshold the
   yield's relative error is the refractivity's times (delta + eps) /
   (beta n - 1)). */
static double altitude(const or_atmosphere *a, const double r[3])
{
    if (!a->spherical) return r[2];
    double zc = r[2] + a->R_E;
    double num = r[0] * r[0] + r[1] * r[1] + r[2] * (r[2] + 2.0 * a->R_E);
    return num / (sqrt(r[0] * r[0] + r[1] * r[1] + zc * zc) + a->R_E);
}

static void unit3(const float d[3], double u[3])
{
    double n = sqrt((double)d[0] * d[0] + (double)d[1] * d[1] + (double)d[2] * d[2]);
    u[0] = d[0] / n; u[1] = d[1] / n; u[2] = d[2] / n;
}

/* ------------------------------------------------------------------------
 * Yield of one track step.
 * Cherenkov (Sec. 1.2, Frank-Tamm formula): with n independent of lambda and
 * constant along the step, the double integral reduces to
 *   N = mu_r pi z^2 e^2/(h eps0 c0) (1/lambda1 - 1/lambda2)
 *       (1 - 1/(beta n)^2) Theta(beta - 1/n) L,
 * and mu_r pi e^2/(h eps0 c0) = 2 pi alpha for mu_r = 1.  n is evaluated at
 * the midpoint of the step (reading of "homogeneous" over the step).
 * Fluorescence (Eq. 1, Sec. 1.1): N = Y dE with a constant yield Y.
 * Bunching (reading): n_b = ceil(N / B) bunches of weight N / n_b.
 * ---------------------------------------------------------------------- */
/* ------------------------------------------------------------------------
 * Angular segment cut (Sec. 1.2.1, optimisation): a step keeps its
 * Cherenkov light when its flight direction d lies within the cut angle of
 * the vector v from the step midpoint m to the array centre (mode 1) or to
 * some telescope centre (mode 2): d . v >= |v| cos(cut).
 * ---------------------------------------------------------------------- */
static int cut_one(const double d[3], const double m[3], const double c[3], double cosc)
{
    double v0 = c[0] - m[0], v1 = c[1] - m[1], v2 = c[2] - m[2];
    double dot = d[0] * v0 + d[1] * v1 + d[2] * v2;
    double nv = sqrt(v0 * v0 + v1 * v1 + v2 * v2);
    return dot - nv * cosc >= 0.0;
}

static int cut_keeps(const double d[3], const double m[3], const or_params *p)
{
    double deg = p->cut_deg > 0 ? p->cut_deg : 6.0;
    double cosc = cos(deg * (OR_PI / 180.0));
    if (p->cut_mode == 1) return cut_one(d, m, p->cut_centre, cosc);
    for (int j = 0; j < p->cut_n_tel; j++) {
        double c[3] = {p->cut_tels[j].x, p->cut_tels[j].y, p->cut_tels[j].z};
        if (cut_one(d, m, c, cosc)) return 1;
    }
    return 0;
}

/* ------------------------------------------------------------------------
 * Fluorescence beaming (Sec. 1.1.1, optimisation): instead of isotropic
 * emission, a step emits into the cone from its midpoint m towards the
 * array centre C that holds every telescope (radius R_b about C), and its
 * photon number is scaled by the cone's solid-angle share.  Reading of the
 * cone: beaming only when D = |C - m| >= 2 R_b; half-angle
 * alpha = asin(R_b / D) + 5e-3 (refraction) + L / D (emission anywhere on
 * the step); share (1 - cos alpha) / 2 = sin^2(alpha / 2).
 * Returns 1 and the axis u and 1 - cos(alpha) when the step is beamed.
 * ---------------------------------------------------------------------- */
static int beam_cone(const or_segment *s, const double d[3], const or_params *p, double u[3], double *omc)
{
    if (!p->fl_beaming) return 0;
    double m[3] = {s->x + 0.5 * s->L * d[0], s->y + 0.5 * s->L * d[1], s->z + 0.5 * s->L * d[2]};
    double v[3] = {p->beam_centre[0] - m[0], p->beam_centre[1] - m[1], p->beam_centre[2] - m[2]};
    double D2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    double R = p->beam_radius;
    if (!(D2 >= 4.0 * R * R)) return 0;
    double D = sqrt(D2);
    double alpha = asin(R / D) + 5e-3 + (double)s->L / D;
    double sh = sin(0.5 * alpha);
    *omc = 2.0 * sh * sh;
    u[0] = v[0] / D; u[1] = v[1] / D; u[2] = v[2] / D;
    return 1;
}

/* ------------------------------------------------------------------------
 * Dispersion.  Sec. 1.2 keeps n(lambda, l) inside the Frank-Tamm double
 * integral but gives no formula for it.  Reading: n - 1 = delta(h) g(lambda)
 * with the Cauchy form g = (1 + B/lambda^2) / (1 + B/lambda_d^2), delta(h)
 * being the refractivity at lambda_d; B is a stated parameter.  In
 * u = 1/lambda the yield is 2 pi alpha z^2 L int (1 - 1/(beta n(u))^2) du
 * over the band where beta n > 1, and the emitted u has that integrand as
 * its density; cos(theta_c) = 1/(beta n(u)) per photon.
 * ---------------------------------------------------------------------- */
double or_disp_g(const or_atmosphere *a, double lambda)
{
    if (!(a->disp_B > 0)) return 1.0;
    return (1.0 + a->disp_B / (lambda * lambda)) / (1.0 + a->disp_B / (a->disp_lref * a->disp_lref));
}

/* beta n(u) - 1 = delta g(u) (1 - eps) - eps, u in 1/nm */
static double disp_g1(const or_atmosphere *a, double delta, double eps, double u)
{
    double g = (1.0 + a->disp_B * u * u) / (1.0 + a->disp_B / (a->disp_lref * a->disp_lref));
    double dg = delta * g;
    return dg - eps - eps * dg;
}

static double disp_f(const or_atmosphere *a, double delta, double eps, double u)
{
    double g1 = disp_g1(a, delta, eps, u);
    if (!(g1 > 0)) return 0.0;
    return g1 * (2.0 + g1) / ((1.0 + g1) * (1.0 + g1));
}

/* the band of u = 1/lambda above threshold: [u_lo, u_hi], 0 if empty */
static int disp_band(const or_atmosphere *a, const or_params *p, double delta, double eps, double *u_lo,
                     double *u_hi)
{
    double u1 = 1.0 / p->lambda1, u2 = 1.0 / p->lambda2;
    if (!(delta > 0)) return 0;
    double G = eps / (delta * (1.0 - eps));
    double g0 = 1.0 + a->disp_B / (a->disp_lref * a->disp_lref);
    double t = (G * g0 - 1.0) / a->disp_B;
    double ut = t > 0 ? sqrt(t) : 0.0;
    *u_lo = ut > u2 ? ut : u2;
    *u_hi = u1;
    return *u_lo < *u_hi;
}

static double disp_integral(const or_atmosphere *a, double delta, double eps, double u_lo, double u_hi);

void or_yield(const or_segment *s, const or_atmosphere *a, const or_params *p, double out[10])
{
    or_yield_at(s, p->seg_base, a, p, out);
}

void or_yield_at(const or_segment *s, int64_t seg_index, const or_atmosphere *a, const or_params *p,
                 double out[10])
{
    double d[3];
    float df[3] = {s->dx, s->dy, s->dz};
    unit3(df, d);
    double rm[3] = {s->x + 0.5 * s->L * d[0], s->y + 0.5 * s->L * d[1], s->z + 0.5 * s->L * d[2]};
    double h_mid = altitude(a, rm);
    double delta = or_delta(a, h_mid);
    double eps_d = (double)s->eps;
    double g1 = delta - eps_d - eps_d * delta;          /* beta n - 1 */
    double z2 = (double)s->charge * (double)s->charge;
    if (p->cut_mode != 0 && z2 > 0 && !cut_keeps(d, rm, p)) z2 = 0;
    double n_c = 0, w_c = 0, cos_tc = 1, sin_tc = 0, Nc = 0;
    double u_lo, u_hi;
    if (a->disp_B > 0) {
        /* the full wavelength integral; cos_tc / sin_tc are then per photon */
        if (z2 > 0 && s->L > 0 && disp_band(a, p, delta, (double)s->eps, &u_lo, &u_hi)) {
            Nc = 2.0 * OR_PI * OR_ALPHA * z2 * 1e9 * disp_integral(a, delta, (double)s->eps, u_lo, u_hi) *
                 (double)s->L;
            n_c = ceil(Nc / p->bunch);
            w_c = n_c > 0 ? Nc / n_c : 0.0;
        }
    } else if (z2 > 0 && g1 > 0.0 && s->L > 0) {
        /* beta n > 1 and 1 - 1/(beta n)^2 = (beta n - 1)(beta n + 1)/(beta n)^2,
           with beta n - 1 = (1 - eps)(1 + delta) - 1 = delta - eps - eps delta:
           the same quantities without the cancellation of 1 - 1/(beta n)^2
           (which keeps only ~16 + log10(beta n - 1) digits near threshold) */
        double bn = 1.0 + g1;
        cos_tc = 1.0 / bn;
        double sin2 = g1 * (2.0 + g1) / (bn * bn);
        sin_tc = sqrt(sin2);
        double band = (1.0 / p->lambda1 - 1.0 / p->lambda2) * 1e9;   /* 1/m */
        Nc = 2.0 * OR_PI * OR_ALPHA * z2 * band * sin2 * (double)s->L;
        n_c = ceil(Nc / p->bunch);
        w_c = n_c > 0 ? Nc / n_c : 0.0;
    }
    double n_f = 0, w_f = 0, Nf = 0;
    if (p->fluor_yield > 0 && s->dE > 0 && s->L > 0) {
        Nf = p->fluor_yield * (double)s->dE;
        double u[3], omc;
        if (beam_cone(s, d, p, u, &omc)) Nf *= 0.5 * omc;
        double x = Nf / p->bunch;
        if (p->fl_roulette && x < 1.0) {
            /* reading of an unbiased count for steps with fewer photons than a
             * bunch: one full bunch with probability N/B */
            uint32_t ctr[4] = {(uint32_t)(uint64_t)seg_index, (uint32_t)((uint64_t)seg_index >> 32), 0xFFFFFFFFu, 1u};
            uint32_t key[2] = {p->seed, p->stream}, r[4];
            or_philox4x32_10(ctr, key, r);
            n_f = or_u01(r[0]) < x ? 1 : 0;
            w_f = n_f > 0 ? p->bunch : 0.0;
        } else {
            n_f = ceil(x);
            w_f = n_f > 0 ? Nf / n_f : 0.0;
        }
    }
    out[0] = n_c; out[1] = w_c; out[2] = n_f; out[3] = w_f;
    out[4] = cos_tc; out[5] = sin_tc; out[6] = Nc; out[7] = Nf;
    out[8] = delta; out[9] = h_mid;
}

/* ------------------------------------------------------------------------
 * M_Rod = 1 + 2 R_Rod^2 (Sec. 1.2.1), written entry by entry as printed,
 * with A the unit bisector of the flight direction and the downward normal.
 * Reading: for a flight direction exactly +z the bisector is undefined and
 * A = x is used.
 * ---------------------------------------------------------------------- */
void or_rotation(const double din[3], double M[9])
{
    double n = sqrt(din[0] * din[0] + din[1] * din[1] + din[2] * din[2]);
    double d[3] = {din[0] / n, din[1] / n, din[2] / n};
    double A[3] = {d[0], d[1], d[2] - 1.0};
    double na = sqrt(A[0] * A[0] + A[1] * A[1] + A[2] * A[2]);
    if (na > 0) { A[0] /= na; A[1] /= na; A[2] /= na; }
    else { A[0] = 1; A[1] = 0; A[2] = 0; }
    double ax = A[0], ay = A[1], az = A[2];
    M[0] = -2 * ay * ay - 2 * az * az + 1; M[1] = 2 * ax * ay;                  M[2] = 2 * ax * az;
    M[3] = 2 * ax * ay;                  M[4] = -2 * ax * ax - 2 * az * az + 1; M[5] = 2 * ay * az;
    M[6] = 2 * ax * az;                  M[7] = 2 * ay * az;                  M[8] = -2 * ax * ax - 2 * ay * ay + 1;
}

typedef struct {
    double n_c, w_c, n_f, w_f, cos_tc, sin_tc;
    double delta;                 /* refractivity at the midpoint (dispersion: per photon theta_c) */
} seg_yield;

/* Photon of bunch k (Sec. 1.2 and Fig. 1: created at the origin pointing
 * down at the Cherenkov angle with azimuth c_rng, rotated by M_Rod, moved to
 * the emission point; Sec. 1.1: fluorescence isotropic, emission points
 * uniform along the track).  Random numbers: Philox counter
 * (segment lo, segment hi, bunch index within its process, process),
 * key (seed, stream); u0 -> wavelength, u1 -> emission point,
 * u2 -> azimuth, u3 -> cos(theta) of fluorescence. */
static void photon_of(const or_segment *s, int64_t seg_index, uint32_t k, const seg_yield *y,
                      const or_atmosphere *a, const or_params *p, double out[10])
{
    double d[3];
    float df[3] = {s->dx, s->dy, s->dz};
    unit3(df, d);
    int process = (double)k < y->n_c ? 0 : 1;
    uint32_t kk = process == 0 ? k : (uint32_t)(k - (uint32_t)y->n_c);
    uint32_t ctr[4] = {(uint32_t)(uint64_t)seg_index, (uint32_t)((uint64_t)seg_index >> 32), kk,
                       (uint32_t)process};
    uint32_t key[2] = {p->seed, p->stream};
    uint32_t x[4];
    or_philox4x32_10(ctr, key, x);
    double u0 = or_u01(x[0]), u1 = or_u01(x[1]), u2 = or_u01(x[2]), u3 = or_u01(x[3]);
    double lambda, dg[3], w;
    if (process == 0) {
        double cos_tc = y->cos_tc, sin_tc = y->sin_tc;
        if (a->disp_B > 0) {
            /* u = 1/lambda with density (1 - 1/(beta n(u))^2) on the band above
             * threshold, by rejection: proposal 0 uses (u0, u3), proposal m >= 1
             * word pair (m - 1) % 2 of Philox with counter word 3 = 2 + (m - 1) / 2;
             * after 64 proposals the last one stands (reading) */
            double eps = (double)s->eps, ulo, uhi;
            disp_band(a, p, y->delta, eps, &ulo, &uhi);
            double fmax = disp_f(a, y->delta, eps, uhi);
            double v = u0, w = u3, u = ulo;
            uint32_t xr[4];
            for (int m = 0;; m++) {
                u = ulo + v * (uhi - ulo);
                if (w * fmax < disp_f(a, y->delta, eps, u) || m == 64) break;
                if (m % 2 == 0) {
                    uint32_t c2[4] = {ctr[0], ctr[1], ctr[2], 2u + (uint32_t)(m / 2)};
                    or_philox4x32_10(c2, key, xr);
                    v = or_u01(xr[0]); w = or_u01(xr[1]);
                } else {
                    v = or_u01(xr[2]); w = or_u01(xr[3]);
                }
            }
            lambda = 1.0 / u;
            double g1 = disp_g1(a, y->delta, eps, u);
            cos_tc = 1.0 / (1.0 + g1);
            sin_tc = sqrt(g1 * (2.0 + g1)) / (1.0 + g1);
        } else {
            /* wavelength density proportional to 1/lambda^2 (Frank-Tamm) */
            double inv = 1.0 / p->lambda1 - u0 * (1.0 / p->lambda1 - 1.0 / p->lambda2);
            lambda = 1.0 / inv;
        }
        double c = 2.0 * OR_PI * u2;
        double pv[3] = {cos(c) * sin_tc, sin(c) * sin_tc, -cos_tc};
        double M[9];
        or_rotation(d, M);
        for (int i = 0; i < 3; i++) dg[i] = M[3 * i] * pv[0] + M[3 * i + 1] * pv[1] + M[3 * i + 2] * pv[2];
        w = y->w_c;
    } else {
        lambda = p->fl_lambda1 + u0 * (p->fl_lambda2 - p->fl_lambda1);
        double u[3], omc;
        if (beam_cone(s, d, p, u, &omc)) {
            /* uniform in solid angle inside the cone about u, rotated like the
             * Cherenkov cone (M_Rod of the axis, Sec. 1.2.1) */
            double ct = 1.0 - u3 * omc;
            double st = sqrt((1.0 - ct) * (1.0 + ct));
            double ph = 2.0 * OR_PI * u2;
            double pv[3] = {cos(ph) * st, sin(ph) * st, -ct};
            double M[9];
            or_rotation(u, M);
            for (int i = 0; i < 3; i++) dg[i] = M[3 * i] * pv[0] + M[3 * i + 1] * pv[1] + M[3 * i + 2] * pv[2];
        } else {
            double ct = 2.0 * u3 - 1.0;
            double st = sqrt((1.0 - ct) * (1.0 + ct));
            double ph = 2.0 * OR_PI * u2;
            dg[0] = st * cos(ph); dg[1] = st * sin(ph); dg[2] = ct;
        }
        w = y->w_f;
    }
    double ell = u1 * (double)s->L;
    double beta = 1.0 - (double)s->eps;
    out[0] = s->x + ell * d[0];
    out[1] = s->y + ell * d[1];
    out[2] = s->z + ell * d[2];
    out[3] = dg[0]; out[4] = dg[1]; out[5] = dg[2];
    out[6] = s->t0 + ell / (beta * OR_C);
    out[7] = lambda;
    out[8] = w;
    out[9] = process;
}

static void yield_struct(const or_segment *s, int64_t seg_index, const or_atmosphere *a, const or_params *p,
                         seg_yield *y)
{
    double o[10];
    or_yield_at(s, seg_index, a, p, o);
    y->n_c = o[0]; y->w_c = o[1]; y->n_f = o[2]; y->w_f = o[3];
    y->cos_tc = o[4]; y->sin_tc = o[5];
    y->delta = o[8];
}

void or_photon(const or_segment *s, int64_t seg_index, uint32_t k,
               const or_atmosphere *a, const or_params *p, double out[10])
{
    seg_yield y;
    yield_struct(s, seg_index, a, p, &y);
    photon_of(s, seg_index, k, &y, a, p, out);
}

/* ------------------------------------------------------------------------
 * Quadrature: adaptive Gauss-Legendre (10 nodes, nodes from Newton's method
 * on the Legendre recurrence), bisecting until the halves agree with the
 * whole to 1e-12 of the integral.
 * ---------------------------------------------------------------------- */
#define GLN 10
static double gl_x[GLN], gl_w[GLN];
static int gl_ready = 0;

static void gl_init(void)
{
    if (gl_ready) return;
    for (int i = 0; i < GLN; i++) {
        double x = cos(OR_PI * (i + 0.75) / (GLN + 0.5)), dp = 1;
        for (int it = 0; it < 100; it++) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= GLN; k++) {
                double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1; p1 = p2;
            }
            dp = GLN * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-17) break;
        }
        gl_x[i] = x;
        gl_w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
    gl_ready = 1;
}

__attribute__((constructor)) static void or_init(void) { gl_init(); }

/* int_{u_lo}^{u_hi} (1 - 1/(beta n(u))^2) du by Gauss-Legendre on 8 panels
 * (the integrand is a smooth rational function of u^2). */
static double disp_integral(const or_atmosphere *a, double delta, double eps, double u_lo, double u_hi)
{
    gl_init();
    const int panels = 8;
    double h = (u_hi - u_lo) / panels, sum = 0;
    for (int q = 0; q < panels; q++) {
        double lo = u_lo + q * h, mid = lo + 0.5 * h;
        for (int i = 0; i < GLN; i++) sum += 0.5 * h * gl_w[i] * disp_f(a, delta, eps, mid + 0.5 * h * gl_x[i]);
    }
    return sum;
}

typedef struct {
    const or_atmosphere *a;
    int refr;
    double p;          /* ray invariant: n r sin(psi) (spherical) or n sin(theta) (flat) */
} ray_ctx;

/* Integrands over altitude h of: angle around the Earth centre (spherical)
 * or horizontal distance (flat); optical path n ds; density-weighted path. */
static void integrand(const ray_ctx *c, double h, double f[3])
{
    const or_atmosphere *a = c->a;
    double rho = or_density(a, h);
    double n = 1.0 + a->K * rho;
    double rr = a->spherical ? (a->R_E + h) : 1.0;
    if (c->refr) {
        double q = n * n * rr * rr - c->p * c->p;
        double sq = sqrt(q);
        f[0] = c->p / (rr * sq);
        f[1] = n * n * rr / sq;
        f[2] = rho / a->rho_ref * n * rr / sq;
    } else {
        double q = rr * rr - c->p * c->p;
        double sq = sqrt(q);
        f[0] = c->p / (rr * sq);
        f[1] = n * rr / sq;
        f[2] = rho / a->rho_ref * rr / sq;
    }
}

static void gl_apply(const ray_ctx *c, double lo, double hi, double out[3])
{
    double m = 0.5 * (lo + hi), r = 0.5 * (hi - lo);
    out[0] = out[1] = out[2] = 0;
    for (int i = 0; i < GLN; i++) {
        double f[3];
        integrand(c, m + r * gl_x[i], f);
        for (int k = 0; k < 3; k++) out[k] += gl_w[i] * f[k];
    }
    for (int k = 0; k < 3; k++) out[k] *= r;
}

/* Bisect until each half-pair agrees with its parent to the interval's share
 * (width / total width) of an absolute tolerance tol[k]; stop at 0.1 mm
 * intervals, where near-grazing integrands reach their rounding floor. */
static void adapt(const ray_ctx *c, double lo, double hi, const double whole[3], const double tol[3],
                  double total_w, int depth, double acc[3])
{
    double mid = 0.5 * (lo + hi), L[3], R[3];
    gl_apply(c, lo, mid, L);
    gl_apply(c, mid, hi, R);
    int ok = 1;
    double share = (hi - lo) / total_w;
    for (int k = 0; k < 3; k++) {
        double s = L[k] + R[k];
        if (!(fabs(s - whole[k]) <= tol[k] * share)) ok = 0;
    }
    if (ok || depth >= 60 || hi - lo < 1e-4) {
        for (int k = 0; k < 3; k++) acc[k] += L[k] + R[k];
        return;
    }
    adapt(c, lo, mid, L, tol, total_w, depth + 1, acc);
    adapt(c, mid, hi, R, tol, total_w, depth + 1, acc);
}

/* Integral over [h_obs, h_e], split where the density has kinks; the
 * tolerance is 1e-12 of each integral's first estimate over the path. */
static void integrate_path(const ray_ctx *c, double h0, double h1, double out[3])
{
    const or_atmosphere *a = c->a;
    double br[12];
    int nb = 0;
    br[nb++] = h0;
    for (int i = 1; i < a->n_layers; i++)
        if (a->h_lo[i] > h0 && a->h_lo[i] < h1) br[nb++] = a->h_lo[i];
    if (a->h_top > h0 && a->h_top < h1) br[nb++] = a->h_top;
    br[nb++] = h1;
    double whole[12][3], est[3] = {0, 0, 0};
    for (int i = 0; i + 1 < nb; i++) {
        gl_apply(c, br[i], br[i + 1], whole[i]);
        for (int k = 0; k < 3; k++) est[k] += fabs(whole[i][k]);
    }
    double tol[3];
    for (int k = 0; k < 3; k++) tol[k] = 1e-12 * est[k] + 1e-300;
    out[0] = out[1] = out[2] = 0;
    double total_w = h1 - h0;
    for (int i = 0; i + 1 < nb; i++) adapt(c, br[i], br[i + 1], whole[i], tol, total_w, 0, out);
}

/* ------------------------------------------------------------------------
 * Propagation to the observation level (Sec. 2).  The paper propagates on a
 * straight line and corrects for refraction; the quantity those corrections
 * approximate is the refracted ray itself, written out here exactly: in a
 * horizontally stratified medium n sin(theta) is constant along the ray, in
 * a spherically stratified one n r sin(psi) is (Bouguer), so position,
 * optical path and optical depth follow as integrals over altitude.
 * With refraction switched off the ray is the straight line but the time
 * still uses the optical path (1/c) int n ds.
 * Readings: the arrival time is the optical path over c (phase index, no
 * dispersion); the optical depth is int rho/rho_ref ds / L_ext(lambda) with
 * L_ext = L0 (lambda/lambda_ref)^4; a photon pointing up (away from the
 * Earth centre) escapes; a ray that turns before the observation level is
 * dropped.
 * out: status, P[3], dL[3], t_L, tau, n_obs.
 * ---------------------------------------------------------------------- */
void or_propagate(const or_atmosphere *a, const double r_e[3], const double din[3],
                  double t_e, double lambda, double out[10])
{
    or_atmosphere ad;
    if (a->disp_B > 0) {          /* n - 1 = delta(h) g(lambda): K scaled for this photon */
        ad = *a;
        ad.K = a->K * or_disp_g(a, lambda);
        a = &ad;
    }
    double nd = sqrt(din[0] * din[0] + din[1] * din[1] + din[2] * din[2]);
    double d[3] = {din[0] / nd, din[1] / nd, din[2] / nd};
    for (int i = 0; i < 10; i++) out[i] = 0;
    double h_e = altitude(a, r_e);
    double n_e = 1.0 + or_delta(a, h_e);
    double n_obs = 1.0 + or_delta(a, a->h_obs);
    out[9] = n_obs;
    ray_ctx c;
    c.a = a;
    c.refr = a->refraction;
    double I[3];
    if (!a->spherical) {
        double cos_e = -d[2];
        if (cos_e <= 0) { out[0] = OR_ESCAPED; return; }
        if (h_e <= a->h_obs) { out[0] = OR_UNDER; return; }
        double sin_e = hypot(d[0], d[1]);
        c.p = a->refraction ? n_e * sin_e : sin_e;
        integrate_path(&c, a->h_obs, h_e, I);
        double ux = sin_e > 0 ? d[0] / sin_e : 1.0, uy = sin_e > 0 ? d[1] / sin_e : 0.0;
        out[1] = r_e[0] + I[0] * ux;
        out[2] = r_e[1] + I[0] * uy;
        out[3] = a->h_obs;
        double sL, cL;
        if (a->refraction) {
            sL = c.p / n_obs;
            cL = sqrt(n_obs * n_obs - c.p * c.p) / n_obs;
        } else {
            sL = sin_e;
            cL = cos_e;
        }
        out[4] = sL * ux; out[5] = sL * uy; out[6] = -cL;
    } else {
        double R[3] = {r_e[0], r_e[1], r_e[2] + a->R_E};
        double r = sqrt(R[0] * R[0] + R[1] * R[1] + R[2] * R[2]);
        double rh[3] = {R[0] / r, R[1] / r, R[2] / r};
        double cos_psi = -(d[0] * rh[0] + d[1] * rh[1] + d[2] * rh[2]);
        if (cos_psi <= 0) { out[0] = OR_ESCAPED; return; }
        if (h_e <= a->h_obs) { out[0] = OR_UNDER; return; }
        double cr[3] = {d[1] * rh[2] - d[2] * rh[1], d[2] * rh[0] - d[0] * rh[2], d[0] * rh[1] - d[1] * rh[0]};
        double sin_psi = sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
        double r_obs = a->R_E + a->h_obs;
        c.p = a->refraction ? n_e * r * sin_psi : r * sin_psi;
        double q_obs = a->refraction ? n_obs * n_obs * r_obs * r_obs - c.p * c.p
                                     : r_obs * r_obs - c.p * c.p;
        if (q_obs <= 0) { out[0] = OR_TURNED; return; }
        integrate_path(&c, a->h_obs, h_e, I);
        double et[3];
        if (sin_psi > 0) {
            for (int i = 0; i < 3; i++) et[i] = (d[i] + cos_psi * rh[i]) / sin_psi;
        } else {  /* vertical ray: any horizontal direction, the angle is 0 */
            double t0[3] = {1, 0, 0};
            double dd = t0[0] * rh[0] + t0[1] * rh[1] + t0[2] * rh[2];
            for (int i = 0; i < 3; i++) et[i] = t0[i] - dd * rh[i];
            double ne = sqrt(et[0] * et[0] + et[1] * et[1] + et[2] * et[2]);
            for (int i = 0; i < 3; i++) et[i] /= ne;
        }
        double phi = I[0], cp = cos(phi), sp = sin(phi);
        double rL[3], eL[3];
        for (int i = 0; i < 3; i++) {
            rL[i] = cp * rh[i] + sp * et[i];
            eL[i] = -sp * rh[i] + cp * et[i];
        }
        out[1] = r_obs * rL[0];
        out[2] = r_obs * rL[1];
        out[3] = r_obs * rL[2] - a->R_E;
        double sL, cL;
        if (a->refraction) {
            sL = c.p / (n_obs * r_obs);
            cL = sqrt(q_obs) / (n_obs * r_obs);
        } else {
            sL = c.p / r_obs;
            cL = sqrt(q_obs) / r_obs;
        }
        for (int i = 0; i < 3; i++) out[4 + i] = sL * eL[i] - cL * rL[i];
    }
    out[0] = OR_TRACED;
    out[7] = t_e + I[1] / OR_C;
    double Lext = a->L0 * pow(lambda / a->lambda_ref, 4.0);
    out[8] = a->absorption ? I[2] / Lext : 0.0;
}

/* ------------------------------------------------------------------------
 * Hit test: the straight line through the landing point along the arrival
 * direction against the sphere (x_j, y_j, z_j; R_j) of every telescope; a
 * hit when the line passes closer than R_j to the centre.  Position and time
 * are taken where the line crosses the plane z = z_j, the time advanced at
 * c / n(h_obs) along the line.
 * ---------------------------------------------------------------------- */
typedef struct {
    or_hit *v;
    int64_t n, cap;
} hitvec;

static void hv_push(hitvec *h, const or_hit *x)
{
    if (h->n == h->cap) {
        h->cap = h->cap ? 2 * h->cap : 1024;
        h->v = (or_hit *)realloc(h->v, (size_t)h->cap * sizeof(or_hit));
    }
    h->v[h->n++] = *x;
}

static void line_to_tel(const double P[3], const double dL[3], double t_L, double n_obs,
                        const or_telescope *T, double *dperp, double *x_rel, double *y_rel, double *t)
{
    double w[3] = {T->x - P[0], T->y - P[1], T->z - P[2]};
    double wd = w[0] * dL[0] + w[1] * dL[1] + w[2] * dL[2];
    double d2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2] - wd * wd;
    *dperp = sqrt(d2 > 0 ? d2 : 0);
    double s = (T->z - P[2]) / dL[2];
    *x_rel = P[0] + s * dL[0] - T->x;
    *y_rel = P[1] + s * dL[1] - T->y;
    *t = t_L + n_obs * s / OR_C;
}

static int cmp_hit(const void *pa, const void *pb, void *ctx);
static int g_ntel_for_sort;
static const or_segment *g_segs_for_sort;
static int64_t g_base_for_sort;

static int cmp_hit_plain(const void *pa, const void *pb)
{
    const or_hit *a = (const or_hit *)pa, *b = (const or_hit *)pb;
    uint32_t sa = g_segs_for_sort[a->seg - g_base_for_sort].shower;
    uint32_t sb = g_segs_for_sort[b->seg - g_base_for_sort].shower;
    if (sa != sb) return sa < sb ? -1 : 1;
    if (a->tel != b->tel) return a->tel < b->tel ? -1 : 1;
    if (a->seg != b->seg) return a->seg < b->seg ? -1 : 1;
    if (a->k != b->k) return a->k < b->k ? -1 : 1;
    return 0;
}
static int cmp_hit(const void *pa, const void *pb, void *ctx) { (void)ctx; return cmp_hit_plain(pa, pb); }

int64_t or_trace(const or_segment *segs, int64_t n_segs,
                 const or_atmosphere *a, const or_telescope *tels, int n_tel,
                 const or_params *p, int n_showers,
                 or_hit *hits, int64_t capacity,
                 int64_t *counts, double *sums, int64_t *stats, int threads)
{
    gl_init();
    int nt = 1;
#ifdef _OPENMP
    nt = threads > 0 ? threads : omp_get_max_threads();
#endif
    hitvec *hv = (hitvec *)calloc((size_t)nt, sizeof(hitvec));
    int64_t *st = (int64_t *)calloc((size_t)nt * 5, sizeof(int64_t));
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
    for (int64_t i = 0; i < n_segs; i++) {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        const or_segment *s = &segs[i];
        seg_yield y;
        yield_struct(s, p->seg_base + i, a, p, &y);
        uint32_t nb = (uint32_t)(y.n_c + y.n_f);
        for (uint32_t k = 0; k < nb; k++) {
            double ph[10], pr[10];
            photon_of(s, p->seg_base + i, k, &y, a, p, ph);
            or_propagate(a, ph, ph + 3, ph[6], ph[7], pr);
            st[tid * 5 + 0]++;
            int status = (int)pr[0];
            if (status != OR_TRACED) { st[tid * 5 + status]++; continue; }
            st[tid * 5 + 4]++;
            double w = ph[8] * exp(-pr[8]);
            for (int j = 0; j < n_tel; j++) {
                double dperp, xr, yr, t;
                line_to_tel(pr + 1, pr + 4, pr[7], pr[9], &tels[j], &dperp, &xr, &yr, &t);
                if (dperp < tels[j].R) {
                    or_hit hrec;
                    hrec.seg = p->seg_base + i; hrec.k = k; hrec.tel = (uint32_t)j;
                    hrec.x_rel = xr; hrec.y_rel = yr; hrec.cx = pr[4]; hrec.cy = pr[5];
                    hrec.lambda = ph[7]; hrec.weight = w; hrec.t = t; hrec.dperp = dperp;
                    hv_push(&hv[tid], &hrec);
                }
            }
        }
    }
    int64_t total = 0;
    for (int t = 0; t < nt; t++) total += hv[t].n;
    or_hit *all = (or_hit *)malloc((size_t)(total > 0 ? total : 1) * sizeof(or_hit));
    int64_t off = 0;
    for (int t = 0; t < nt; t++) {
        if (hv[t].n) memcpy(all + off, hv[t].v, (size_t)hv[t].n * sizeof(or_hit));
        off += hv[t].n;
        free(hv[t].v);
    }
    g_segs_for_sort = segs;
    g_base_for_sort = p->seg_base;
    g_ntel_for_sort = n_tel;
    qsort(all, (size_t)total, sizeof(or_hit), cmp_hit_plain);
    (void)cmp_hit;
    if (counts) memset(counts, 0, sizeof(int64_t) * (size_t)n_showers * (size_t)n_tel);
    if (sums) memset(sums, 0, sizeof(double) * (size_t)n_showers * (size_t)n_tel);
    for (int64_t i = 0; i < total; i++) {
        int64_t g = (int64_t)segs[all[i].seg - p->seg_base].shower * n_tel + all[i].tel;
        if (counts) counts[g] += 1;
        if (sums) sums[g] += all[i].weight;
    }
    if (hits) {
        int64_t m = total < capacity ? total : capacity;
        if (m > 0) memcpy(hits, all, (size_t)m * sizeof(or_hit));
    }
    if (stats) {
        for (int k = 0; k < 5; k++) {
            stats[k] = 0;
            for (int t = 0; t < nt; t++) stats[k] += st[t * 5 + k];
        }
    }
    free(all);
    free(hv);
    free(st);
    return total;
}

/* ------------------------------------------------------------------------
 * Frozen-bunch evaluations used to differentiate by finite differences:
 * the bunch counts are held at their nominal values, so the weight of a
 * bunch becomes N(theta) / n_b.
 * ---------------------------------------------------------------------- */
static void frozen_yield(const or_segment *s, const or_atmosphere *a, const or_params *p,
                         uint32_t nbc, uint32_t nbf, seg_yield *y)
{
    double o[10];
    or_yield(s, a, p, o);
    y->n_c = nbc;
    y->n_f = nbf;
    y->w_c = nbc > 0 ? o[6] / nbc : 0;
    y->w_f = nbf > 0 ? (p->fl_roulette && o[7] < p->bunch ? p->bunch : o[7] / nbf) : 0;
    y->cos_tc = o[4];
    y->sin_tc = o[5];
    y->delta = o[8];
}

static double logistic(double x) { return 1.0 / (1.0 + exp(-x)); }

void or_soft_yield(const or_segment *segs, int64_t n_segs, const uint32_t *n_bunch_c,
                   const uint32_t *n_bunch_f, const or_atmosphere *a,
                   const or_telescope *tels, int n_tel, const or_params *p,
                   int n_showers, double s, double W, double *yield, int threads)
{
    gl_init();
    int nt = 1;
#ifdef _OPENMP
    nt = threads > 0 ? threads : omp_get_max_threads();
#endif
    size_t ng = (size_t)n_showers * (size_t)n_tel;
    double *part = (double *)calloc((size_t)nt * ng, sizeof(double));
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
    for (int64_t i = 0; i < n_segs; i++) {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        seg_yield y;
        frozen_yield(&segs[i], a, p, n_bunch_c[i], n_bunch_f[i], &y);
        uint32_t nb = n_bunch_c[i] + n_bunch_f[i];
        for (uint32_t k = 0; k < nb; k++) {
            double ph[10], pr[10];
            photon_of(&segs[i], p->seg_base + i, k, &y, a, p, ph);
            or_propagate(a, ph, ph + 3, ph[6], ph[7], pr);
            if ((int)pr[0] != OR_TRACED) continue;
            double w = ph[8] * exp(-pr[8]);
            for (int j = 0; j < n_tel; j++) {
                double dperp, xr, yr, t;
                line_to_tel(pr + 1, pr + 4, pr[7], pr[9], &tels[j], &dperp, &xr, &yr, &t);
                if (dperp < tels[j].R + W)
                    part[(size_t)tid * ng + (size_t)segs[i].shower * n_tel + j] +=
                        w * logistic((tels[j].R - dperp) / s);
            }
        }
    }
    for (size_t g = 0; g < ng; g++) {
        double acc = 0;
        for (int t = 0; t < nt; t++) acc += part[(size_t)t * ng + g];
        yield[g] = acc;
    }
    free(part);
}

void or_eval_rays(const or_segment *segs, const int64_t *seg_idx, const uint32_t *k,
                  const uint32_t *tel, const uint32_t *n_bunch_c, const uint32_t *n_bunch_f,
                  int64_t n, const or_atmosphere *a, const or_telescope *tels,
                  const or_params *p, double *out, int threads)
{
    gl_init();
    int nt = 1;
#ifdef _OPENMP
    nt = threads > 0 ? threads : omp_get_max_threads();
#endif
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
    for (int64_t i = 0; i < n; i++) {
        int64_t si = seg_idx[i];
        seg_yield y;
        frozen_yield(&segs[si], a, p, n_bunch_c[si], n_bunch_f[si], &y);
        double ph[10], pr[10];
        photon_of(&segs[si], p->seg_base + si, k[i], &y, a, p, ph);
        or_propagate(a, ph, ph + 3, ph[6], ph[7], pr);
        double *o = out + 5 * i;
        if ((int)pr[0] != OR_TRACED) {
            for (int m = 0; m < 5; m++) o[m] = NAN;
            continue;
        }
        double dperp, xr, yr, t;
        line_to_tel(pr + 1, pr + 4, pr[7], pr[9], &tels[tel[i]], &dperp, &xr, &yr, &t);
        o[0] = xr; o[1] = yr; o[2] = t; o[3] = ph[8] * exp(-pr[8]); o[4] = dperp;
    }
}

/* ========================================================================
 * FP64 reference gradient, written separately from the finite differences:
 * forward-mode dual numbers carried through the same physics with one
 * tangent per parameter theta = (c_1..c_L, K, L0) (b_i, the layer edges,
 * the random numbers and the bunch counts fixed).  The propagation
 * integrals have fixed limits (h_obs, h_e), so their tangents are the
 * integrals of the differentiated integrands, taken by Gauss-Legendre on
 * 32 panels per smooth piece.
 * ====================================================================== */
#define OR_NP 10
typedef struct { double v, d[OR_NP]; } dn;

static dn dn_c(double v) { dn r; r.v = v; for (int i = 0; i < OR_NP; i++) r.d[i] = 0; return r; }
static dn dn_add(dn a, dn b) { dn r; r.v = a.v + b.v; for (int i = 0; i < OR_NP; i++) r.d[i] = a.d[i] + b.d[i]; return r; }
static dn dn_sub(dn a, dn b) { dn r; r.v = a.v - b.v; for (int i = 0; i < OR_NP; i++) r.d[i] = a.d[i] - b.d[i]; return r; }
static dn dn_mul(dn a, dn b)
{
    dn r; r.v = a.v * b.v;
    for (int i = 0; i < OR_NP; i++) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
    return r;
}
static dn dn_scale(dn a, double s) { dn r; r.v = a.v * s; for (int i = 0; i < OR_NP; i++) r.d[i] = a.d[i] * s; return r; }
static dn dn_div(dn a, dn b)
{
    dn r; r.v = a.v / b.v;
    for (int i = 0; i < OR_NP; i++) r.d[i] = (a.d[i] - r.v * b.d[i]) / b.v;
    return r;
}
static dn dn_sqrt(dn a)
{
    dn r; r.v = sqrt(a.v);
    for (int i = 0; i < OR_NP; i++) r.d[i] = r.v > 0 ? a.d[i] / (2.0 * r.v) : 0.0;
    return r;
}
static dn dn_exp(dn a) { dn r; r.v = exp(a.v); for (int i = 0; i < OR_NP; i++) r.d[i] = a.d[i] * r.v; return r; }
static dn dn_cos(dn a) { dn r; r.v = cos(a.v); double s = -sin(a.v); for (int i = 0; i < OR_NP; i++) r.d[i] = a.d[i] * s; return r; }
static dn dn_sin(dn a) { dn r; r.v = sin(a.v); double c = cos(a.v); for (int i = 0; i < OR_NP; i++) r.d[i] = a.d[i] * c; return r; }

/* rho(h) and n(h) - 1 with their tangents: d rho/d c_i = rho (h/c_i^2 - 1/c_i)
 * in the layer of h, d delta / d K = rho */
static void dn_atm(const or_atmosphere *a, double h, dn *rho, dn *delta)
{
    int L = a->n_layers;
    *rho = dn_c(0);
    *delta = dn_c(0);
    if (h >= a->h_top) return;
    int i = layer_of(a, h);
    double c = a->c[i];
    double r = a->b[i] / (100.0 * c) * exp(-h / c);
    rho->v = r;
    rho->d[i] = r * (h / (c * c) - 1.0 / c);
    *delta = dn_scale(*rho, a->K);
    delta->d[L] = r;
}

typedef struct {
    const or_atmosphere *a;
    dn p;
    int refr;
} dn_ray;

static void dn_integrand(const dn_ray *c, double h, dn f[3])
{
    const or_atmosphere *a = c->a;
    dn rho, delta;
    dn_atm(a, h, &rho, &delta);
    dn n = dn_add(dn_c(1.0), delta);
    double rr = a->spherical ? (a->R_E + h) : 1.0;
    dn nn = c->refr ? n : dn_c(1.0);
    dn q = dn_sub(dn_scale(dn_mul(nn, nn), rr * rr), dn_mul(c->p, c->p));
    dn sq = dn_sqrt(q);
    f[0] = dn_div(c->p, dn_scale(sq, rr));
    f[1] = dn_div(dn_scale(dn_mul(n, nn), rr), sq);
    f[2] = dn_div(dn_scale(dn_mul(rho, nn), rr / a->rho_ref), sq);
}

static void dn_integrate(const dn_ray *c, double h0, double h1, dn out[3])
{
    gl_init();
    const or_atmosphere *a = c->a;
    double br[12];
    int nb = 0;
    br[nb++] = h0;
    for (int i = 1; i < a->n_layers; i++)
        if (a->h_lo[i] > h0 && a->h_lo[i] < h1) br[nb++] = a->h_lo[i];
    if (a->h_top > h0 && a->h_top < h1) br[nb++] = a->h_top;
    br[nb++] = h1;
    out[0] = out[1] = out[2] = dn_c(0);
    const int panels = 32;
    for (int s = 0; s + 1 < nb; s++) {
        double w = (br[s + 1] - br[s]) / panels;
        for (int q = 0; q < panels; q++) {
            double mid = br[s] + (q + 0.5) * w;
            for (int i = 0; i < GLN; i++) {
                dn f[3];
                dn_integrand(c, mid + 0.5 * w * gl_x[i], f);
                for (int k = 0; k < 3; k++) out[k] = dn_add(out[k], dn_scale(f[k], 0.5 * w * gl_w[i]));
            }
        }
    }
}

/* One ray with tangents: landing point P, arrival direction dL, arrival
 * time t_L, optical depth tau and n_obs, mirroring or_propagate.  Returns
 * the status. */
static int dn_propagate(const or_atmosphere *a, const double r_e[3], const dn dg[3], double t_e, double lambda,
                        dn P[3], dn dL[3], dn *tL, dn *tau, dn *n_obs_out)
{
    int L = a->n_layers;
    double h_e = altitude(a, r_e);
    dn rho_e, del_e, rho_o, del_o;
    dn_atm(a, h_e, &rho_e, &del_e);
    dn_atm(a, a->h_obs, &rho_o, &del_o);
    dn n_e = dn_add(dn_c(1.0), del_e), n_obs = dn_add(dn_c(1.0), del_o);
    *n_obs_out = n_obs;
    dn nd = dn_sqrt(dn_add(dn_add(dn_mul(dg[0], dg[0]), dn_mul(dg[1], dg[1])), dn_mul(dg[2], dg[2])));
    dn d[3] = {dn_div(dg[0], nd), dn_div(dg[1], nd), dn_div(dg[2], nd)};
    dn_ray c;
    c.a = a;
    c.refr = a->refraction;
    dn I[3];
    if (!a->spherical) {
        dn cos_e = dn_scale(d[2], -1.0);
        if (cos_e.v <= 0) return OR_ESCAPED;
        if (h_e <= a->h_obs) return OR_UNDER;
        dn sin_e = dn_sqrt(dn_add(dn_mul(d[0], d[0]), dn_mul(d[1], d[1])));
        c.p = a->refraction ? dn_mul(n_e, sin_e) : sin_e;
        dn_integrate(&c, a->h_obs, h_e, I);
        dn ux = sin_e.v > 0 ? dn_div(d[0], sin_e) : dn_c(1.0), uy = sin_e.v > 0 ? dn_div(d[1], sin_e) : dn_c(0.0);
        P[0] = dn_add(dn_c(r_e[0]), dn_mul(I[0], ux));
        P[1] = dn_add(dn_c(r_e[1]), dn_mul(I[0], uy));
        P[2] = dn_c(a->h_obs);
        dn sL, cL;
        if (a->refraction) {
            sL = dn_div(c.p, n_obs);
            cL = dn_div(dn_sqrt(dn_sub(dn_mul(n_obs, n_obs), dn_mul(c.p, c.p))), n_obs);
        } else {
            sL = sin_e;
            cL = cos_e;
        }
        dL[0] = dn_mul(sL, ux); dL[1] = dn_mul(sL, uy); dL[2] = dn_scale(cL, -1.0);
    } else {
        double R[3] = {r_e[0], r_e[1], r_e[2] + a->R_E};
        double r = sqrt(R[0] * R[0] + R[1] * R[1] + R[2] * R[2]);
        double rh[3] = {R[0] / r, R[1] / r, R[2] / r};
        dn cos_psi = dn_scale(dn_add(dn_add(dn_scale(d[0], rh[0]), dn_scale(d[1], rh[1])), dn_scale(d[2], rh[2])), -1.0);
        if (cos_psi.v <= 0) return OR_ESCAPED;
        if (h_e <= a->h_obs) return OR_UNDER;
        dn cr[3] = {dn_sub(dn_scale(d[1], rh[2]), dn_scale(d[2], rh[1])),
                    dn_sub(dn_scale(d[2], rh[0]), dn_scale(d[0], rh[2])),
                    dn_sub(dn_scale(d[0], rh[1]), dn_scale(d[1], rh[0]))};
        dn sin_psi = dn_sqrt(dn_add(dn_add(dn_mul(cr[0], cr[0]), dn_mul(cr[1], cr[1])), dn_mul(cr[2], cr[2])));
        double r_obs = a->R_E + a->h_obs;
        c.p = a->refraction ? dn_scale(dn_mul(n_e, sin_psi), r) : dn_scale(sin_psi, r);
        dn q_obs = a->refraction ? dn_sub(dn_scale(dn_mul(n_obs, n_obs), r_obs * r_obs), dn_mul(c.p, c.p))
                                 : dn_sub(dn_c(r_obs * r_obs), dn_mul(c.p, c.p));
        if (q_obs.v <= 0) return OR_TURNED;
        dn_integrate(&c, a->h_obs, h_e, I);
        dn et[3];
        if (sin_psi.v > 0) {
            for (int i = 0; i < 3; i++) et[i] = dn_div(dn_add(d[i], dn_scale(cos_psi, rh[i])), sin_psi);
        } else {
            double t0[3] = {1, 0, 0};
            double dd = t0[0] * rh[0] + t0[1] * rh[1] + t0[2] * rh[2];
            double e3[3];
            for (int i = 0; i < 3; i++) e3[i] = t0[i] - dd * rh[i];
            double ne = sqrt(e3[0] * e3[0] + e3[1] * e3[1] + e3[2] * e3[2]);
            for (int i = 0; i < 3; i++) et[i] = dn_c(e3[i] / ne);
        }
        dn cp = dn_cos(I[0]), sp = dn_sin(I[0]);
        dn rL[3], eL[3];
        for (int i = 0; i < 3; i++) {
            rL[i] = dn_add(dn_scale(cp, rh[i]), dn_mul(sp, et[i]));
            eL[i] = dn_add(dn_scale(sp, -rh[i]), dn_mul(cp, et[i]));
        }
        P[0] = dn_scale(rL[0], r_obs);
        P[1] = dn_scale(rL[1], r_obs);
        P[2] = dn_sub(dn_scale(rL[2], r_obs), dn_c(a->R_E));
        dn sL, cL;
        if (a->refraction) {
            dn nr = dn_scale(n_obs, r_obs);
            sL = dn_div(c.p, nr);
            cL = dn_div(dn_sqrt(q_obs), nr);
        } else {
            sL = dn_scale(c.p, 1.0 / r_obs);
            cL = dn_scale(dn_sqrt(q_obs), 1.0 / r_obs);
        }
        for (int i = 0; i < 3; i++) dL[i] = dn_sub(dn_mul(sL, eL[i]), dn_mul(cL, rL[i]));
    }
    *tL = dn_add(dn_c(t_e), dn_scale(I[1], 1.0 / OR_C));
    if (a->absorption) {
        dn L0 = dn_c(a->L0);
        L0.d[L + 1] = 1.0;
        dn Lext = dn_scale(L0, pow(lambda / a->lambda_ref, 4.0));
        *tau = dn_div(I[2], Lext);
    } else {
        *tau = dn_c(0);
    }
    return OR_TRACED;
}

/* The photon with tangents: the step's midpoint refractivity moves theta_c
 * and the yield (per-bunch weight N / n_b with n_b frozen); fluorescence
 * emission does not depend on theta. */
static void dn_photon(const or_segment *s, int64_t seg_index, uint32_t k, uint32_t nbc, uint32_t nbf,
                      const or_atmosphere *a, const or_params *p, double r_e[3], dn dg[3], double *t_e,
                      double *lambda, dn *w)
{
    int L = a->n_layers;
    seg_yield y;
    frozen_yield(s, a, p, nbc, nbf, &y);
    double ph[10];
    photon_of(s, seg_index, k, &y, a, p, ph);
    r_e[0] = ph[0]; r_e[1] = ph[1]; r_e[2] = ph[2];
    *t_e = ph[6];
    *lambda = ph[7];
    if ((int)ph[9] == 1) {
        for (int i = 0; i < 3; i++) dg[i] = dn_c(ph[3 + i]);
        *w = dn_c(y.w_f);
        return;
    }
    double d[3];
    float df[3] = {s->dx, s->dy, s->dz};
    unit3(df, d);
    double rm[3] = {s->x + 0.5 * s->L * d[0], s->y + 0.5 * s->L * d[1], s->z + 0.5 * s->L * d[2]};
    dn rho, delta;
    dn_atm(a, altitude(a, rm), &rho, &delta);
    (void)L;
    double eps = (double)s->eps;
    dn g1 = dn_sub(dn_scale(delta, 1.0 - eps), dn_c(eps));
    dn bn = dn_add(dn_c(1.0), g1);
    dn sin2 = dn_div(dn_mul(g1, dn_add(g1, dn_c(2.0))), dn_mul(bn, bn));
    dn cos_tc = dn_div(dn_c(1.0), bn), sin_tc = dn_sqrt(sin2);
    double z2 = (double)s->charge * (double)s->charge;
    double band = (1.0 / p->lambda1 - 1.0 / p->lambda2) * 1e9;
    *w = dn_scale(sin2, 2.0 * OR_PI * OR_ALPHA * z2 * band * (double)s->L / (double)nbc);
    /* the azimuth of bunch k, recovered from the primal direction */
    double M[9];
    or_rotation(d, M);
    double pv[3];                         /* M^T d_gamma = (cos c sin, sin c sin, -cos) */
    for (int i = 0; i < 3; i++) pv[i] = M[i] * ph[3] + M[3 + i] * ph[4] + M[6 + i] * ph[5];
    double cc = pv[0], sc = pv[1], sn = sqrt(cc * cc + sc * sc);
    cc = sn > 0 ? cc / sn : 1.0;
    sc = sn > 0 ? sc / sn : 0.0;
    dn pd[3] = {dn_scale(sin_tc, cc), dn_scale(sin_tc, sc), dn_scale(cos_tc, -1.0)};
    for (int i = 0; i < 3; i++)
        dg[i] = dn_add(dn_add(dn_scale(pd[0], M[3 * i]), dn_scale(pd[1], M[3 * i + 1])), dn_scale(pd[2], M[3 * i + 2]));
}

/* Gradient of sum_i (gx_i x_rel_i + gy_i y_rel_i + gt_i t_i + gw_i weight_i)
 * over the given hits, in FP64 by dual numbers: grad[0 .. n_layers + 1]. */
void or_grad_rays(const or_segment *segs, const int64_t *seg_idx, const uint32_t *k, const uint32_t *tel,
                  const uint32_t *n_bunch_c, const uint32_t *n_bunch_f, int64_t n, const or_atmosphere *a,
                  const or_telescope *tels, const or_params *p, const double *gx, const double *gy,
                  const double *gt, const double *gw, double *grad, int threads)
{
    gl_init();
    int np = a->n_layers + 2;
    int nt = 1;
#ifdef _OPENMP
    nt = threads > 0 ? threads : omp_get_max_threads();
#endif
    double *part = (double *)calloc((size_t)nt * OR_NP, sizeof(double));
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
    for (int64_t i = 0; i < n; i++) {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        int64_t si = seg_idx[i];
        double r_e[3], t_e, lam;
        dn dg[3], w;
        dn_photon(&segs[si], p->seg_base + si, k[i], n_bunch_c[si], n_bunch_f[si], a, p, r_e, dg, &t_e, &lam, &w);
        dn P[3], dL[3], tL, tau, n_obs;
        if (dn_propagate(a, r_e, dg, t_e, lam, P, dL, &tL, &tau, &n_obs) != OR_TRACED) continue;
        const or_telescope *T = &tels[tel[i]];
        dn sj = dn_div(dn_sub(dn_c(T->z), P[2]), dL[2]);
        dn xr = dn_sub(dn_add(P[0], dn_mul(sj, dL[0])), dn_c(T->x));
        dn yr = dn_sub(dn_add(P[1], dn_mul(sj, dL[1])), dn_c(T->y));
        dn tt = dn_add(tL, dn_scale(dn_mul(n_obs, sj), 1.0 / OR_C));
        dn wt = dn_mul(w, dn_exp(dn_scale(tau, -1.0)));
        for (int j = 0; j < np; j++)
            part[(size_t)tid * OR_NP + j] += (gx ? gx[i] * xr.d[j] : 0) + (gy ? gy[i] * yr.d[j] : 0) +
                                             (gt ? gt[i] * tt.d[j] : 0) + (gw ? gw[i] * wt.d[j] : 0);
    }
    for (int j = 0; j < np; j++) {
        double s = 0;
        for (int t = 0; t < nt; t++) s += part[(size_t)t * OR_NP + j];
        grad[j] = s;
    }
    free(part);
}

/* Gradient of sum_g gY_g Y_g for the soft yield of or_soft_yield. */
void or_grad_soft(const or_segment *segs, int64_t n_segs, const uint32_t *n_bunch_c, const uint32_t *n_bunch_f,
                  const or_atmosphere *a, const or_telescope *tels, int n_tel, const or_params *p, int n_showers,
                  double s, double W, const double *gY, double *grad, int threads)
{
    gl_init();
    (void)n_showers;
    int np = a->n_layers + 2;
    int nt = 1;
#ifdef _OPENMP
    nt = threads > 0 ? threads : omp_get_max_threads();
#endif
    double *part = (double *)calloc((size_t)nt * OR_NP, sizeof(double));
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
    for (int64_t i = 0; i < n_segs; i++) {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        uint32_t nb = n_bunch_c[i] + n_bunch_f[i];
        for (uint32_t kk = 0; kk < nb; kk++) {
            double r_e[3], t_e, lam;
            dn dg[3], w;
            dn_photon(&segs[i], p->seg_base + i, kk, n_bunch_c[i], n_bunch_f[i], a, p, r_e, dg, &t_e, &lam, &w);
            dn P[3], dL[3], tL, tau, n_obs;
            if (dn_propagate(a, r_e, dg, t_e, lam, P, dL, &tL, &tau, &n_obs) != OR_TRACED) continue;
            dn wt = dn_mul(w, dn_exp(dn_scale(tau, -1.0)));
            for (int j = 0; j < n_tel; j++) {
                const or_telescope *T = &tels[j];
                dn wv[3] = {dn_sub(dn_c(T->x), P[0]), dn_sub(dn_c(T->y), P[1]), dn_sub(dn_c(T->z), P[2])};
                dn wd = dn_add(dn_add(dn_mul(wv[0], dL[0]), dn_mul(wv[1], dL[1])), dn_mul(wv[2], dL[2]));
                dn d2 = dn_sub(dn_add(dn_add(dn_mul(wv[0], wv[0]), dn_mul(wv[1], wv[1])), dn_mul(wv[2], wv[2])),
                               dn_mul(wd, wd));
                dn dp = dn_sqrt(d2);
                if (!(dp.v < T->R + W)) continue;
                dn u = dn_scale(dn_sub(dn_c(T->R), dp), 1.0 / s);
                dn sg = dn_div(dn_c(1.0), dn_add(dn_c(1.0), dn_exp(dn_scale(u, -1.0))));
                double gyv = gY[(size_t)segs[i].shower * n_tel + j];
                dn y = dn_mul(wt, sg);
                for (int q = 0; q < np; q++) part[(size_t)tid * OR_NP + q] += gyv * y.d[q];
            }
        }
    }
    for (int j = 0; j < np; j++) {
        double sum = 0;
        for (int t = 0; t < nt; t++) sum += part[(size_t)t * OR_NP + j];
        grad[j] = sum;
    }
    free(part);
}
