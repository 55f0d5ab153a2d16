// clight_api.cu -- the C ABI declared in include/clight.h: context, tables,
// scratch memory, the launch sequence and its CUDA-graph replay.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "internal.h"

using namespace clight;

// Device buffer that only grows; every reallocation bumps *gen so that a
// captured graph holding the old address is rebuilt.
template <class T> struct Buf {
    T *p = nullptr;
    int64_t n = 0;
    cudaError_t ensure(int64_t need, uint64_t *gen)
    {
        need = std::max<int64_t>(need, 1);
        if (p && need <= n) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
        cudaError_t e = cudaMalloc((void **)&p, sizeof(T) * (size_t)need);
        if (e == cudaSuccess) n = need;
        ++*gen;
        return e;
    }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
};


struct GraphKey {
    const void *segs;
    int64_t n_segs;
    int32_t n_showers;
    const void *hits;
    int64_t cap;
    const void *counts;
    const void *sums;
    uint64_t version;
    int64_t defer_use;
    bool operator==(const GraphKey &o) const
    {
        return segs == o.segs && n_segs == o.n_segs && n_showers == o.n_showers && hits == o.hits &&
               cap == o.cap && counts == o.counts && sums == o.sums && version == o.version &&
               defer_use == o.defer_use;
    }
};

struct clight_ctx {
    int device = 0, n_sm = 0;
    bool atm_set = false, tel_set = false;
    uint64_t version = 1;             // bumped by every set_* call
    DevAtm atm{};
    DevTel tel{};
    DevPar par{};
    clight_params upar{};
    clight_atmosphere uatm{};
    // telescope tables (device)
    float4 *d_tel = nullptr;
    int *d_cell_start = nullptr, *d_cell_tel = nullptr;
    uint8_t *d_clr = nullptr;
    uint8_t *d_fclr = nullptr;
    // scratch (device)
    unsigned long long *d_ctr = nullptr;
    Buf<clight_hit> rec;
    Buf<unsigned long long> keys, keys_alt;
    Buf<unsigned long long> defer;              // rays left to the deferred kernel
    int64_t defer_use = 0;                      // entries of it in use (0 = no queue)
    int64_t defer_piece = 0;                    // steps per launch with the default queue
    int64_t defer_min = 0;                      // queue size learned from calls that filled it
    bool defer_off = false;                     // this call runs without the queue
    Buf<uint32_t> vals, vals_alt, hist, bsums;
    Buf<int64_t> gstart, gend;
    uint64_t scratch_gen = 0;
    // staging for the host-buffer entry point
    Buf<double> adj_partial, adj_out;
    Buf<unsigned long long> adj_cand, adj_ctr;   // soft-yield candidates and their cursor
    Buf<unsigned long long> adj_keys_alt, adj_yfix;   // candidate sort; fixed-point soft yield
    Buf<uint32_t> adj_vals, adj_vals_alt, adj_hist, adj_bsums;
    Buf<clight_segment> stage_segs;
    Buf<clight_segment> tune_segs;              // the autotuner's sample
    Buf<clight_hit> stage_hits;
    Buf<int64_t> stage_counts;
    Buf<double> stage_sums;
    // pinned host copy of the counters
    unsigned long long *h_ctr = nullptr;
    // graph replay
    cudaStream_t cap_stream = nullptr;
    // host-buffer entry point: chunked copies on their own stream
    cudaStream_t copy_stream = nullptr;
    std::vector<cudaEvent_t> chunk_ev;
    cudaEvent_t ev = nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr, t2 = nullptr;   // phase timing
    bool timed = false;
    // the last clight_trace_adjoint: phase events and counts
    cudaEvent_t a_ev[4] = {nullptr, nullptr, nullptr, nullptr};
    bool a_timed = false;
    int64_t a_cand = 0, a_hits = 0;
    cudaGraphExec_t gexec = nullptr;
    GraphKey gkey{};
    void *noalloc_slots[2] = {nullptr, nullptr};  // device addresses of the no-allocation scratch and queue
};

#define CK(x)                                   \
    do {                                        \
        cudaError_t e_ = (x);                   \
        if (e_ != cudaSuccess) return CLIGHT_ERR_CUDA; \
    } while (0)

static int bits_for(int64_t x)   // bits needed to hold values 0..x
{
    int b = 0;
    while (x > 0) { ++b; x >>= 1; }
    return b;
}

extern "C" {

const char *clight_status_string(clight_status s)
{
    switch (s) {
    case CLIGHT_OK: return "ok";
    case CLIGHT_ERR_ARG: return "invalid argument";
    case CLIGHT_ERR_CUDA: return "CUDA runtime error";
    case CLIGHT_ERR_HIT_CAPACITY: return "hit capacity exceeded";
    case CLIGHT_ERR_BAD_SEGMENT: return "invalid segment";
    case CLIGHT_ERR_LIMIT: return "size or index beyond a documented limit";
    case CLIGHT_ERR_NO_DEVICE: return "no usable CUDA device";
    }
    return "unknown status";
}

int clight_version(void) { return 10000; }

clight_status clight_last_timing(clight_ctx *c, float ms[2])
{
    if (!c || !ms || !c->timed) return CLIGHT_ERR_ARG;
    if (cudaEventElapsedTime(&ms[0], c->t0, c->t1) != cudaSuccess) return CLIGHT_ERR_CUDA;
    if (cudaEventElapsedTime(&ms[1], c->t1, c->t2) != cudaSuccess) return CLIGHT_ERR_CUDA;
    return CLIGHT_OK;
}

clight_status clight_last_adjoint(clight_ctx *c, int64_t *h_candidates, int64_t *h_hits, float ms[3])
{
    if (!c || !c->a_timed) return CLIGHT_ERR_ARG;
    if (h_candidates) *h_candidates = c->a_cand;
    if (h_hits) *h_hits = c->a_hits;
    if (ms)
        for (int i = 0; i < 3; ++i)
            if (cudaEventElapsedTime(&ms[i], c->a_ev[i], c->a_ev[i + 1]) != cudaSuccess) return CLIGHT_ERR_CUDA;
    return CLIGHT_OK;
}

clight_status clight_create(clight_ctx **out, int device)
{
    if (!out) return CLIGHT_ERR_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return CLIGHT_ERR_NO_DEVICE;
    }
    DeviceGuard dg(device);
    if (!dg.ok) return CLIGHT_ERR_NO_DEVICE;
    clight_ctx *c = new clight_ctx();
    c->device = device;
    cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, device);
    if (cudaMalloc((void **)&c->d_ctr, sizeof(unsigned long long) * CTR_N) != cudaSuccess ||
        cudaMallocHost((void **)&c->h_ctr, sizeof(unsigned long long) * CTR_N) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreate(&c->t0) != cudaSuccess || cudaEventCreate(&c->t1) != cudaSuccess ||
        cudaEventCreate(&c->t2) != cudaSuccess || cudaEventCreate(&c->a_ev[0]) != cudaSuccess ||
        cudaEventCreate(&c->a_ev[1]) != cudaSuccess || cudaEventCreate(&c->a_ev[2]) != cudaSuccess ||
        cudaEventCreate(&c->a_ev[3]) != cudaSuccess) {
        clight_destroy(c);
        return CLIGHT_ERR_CUDA;
    }
    clight_params p{};
    p.lambda1 = 300; p.lambda2 = 600; p.bunch = 1; p.seed = 1; p.stream = 0;
    p.fl_lambda1 = 340; p.fl_lambda2 = 450;
    *out = c;
    clight_set_params(c, &p);
    return CLIGHT_OK;
}

void clight_destroy(clight_ctx *c)
{
    if (!c) return;
    DeviceGuard dg(c->device);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    void *dev[] = {c->d_tel, c->d_cell_start, c->d_cell_tel, c->d_clr, c->d_fclr, c->d_ctr};
    for (void *p : dev)
        if (p) cudaFree(p);
    c->rec.release(); c->keys.release(); c->keys_alt.release(); c->vals.release(); c->vals_alt.release();
    c->defer.release();
    c->hist.release(); c->bsums.release(); c->gstart.release(); c->gend.release();
    c->stage_segs.release(); c->tune_segs.release(); c->stage_hits.release(); c->stage_counts.release(); c->stage_sums.release();
    c->adj_partial.release(); c->adj_out.release(); c->adj_cand.release(); c->adj_ctr.release();
    c->adj_keys_alt.release(); c->adj_yfix.release(); c->adj_vals.release(); c->adj_vals_alt.release();
    c->adj_hist.release(); c->adj_bsums.release();
    if (c->h_ctr) cudaFreeHost(c->h_ctr);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    for (cudaEvent_t e : c->chunk_ev) cudaEventDestroy(e);
    if (c->ev) cudaEventDestroy(c->ev);
    if (c->t0) cudaEventDestroy(c->t0);
    if (c->t1) cudaEventDestroy(c->t1);
    if (c->t2) cudaEventDestroy(c->t2);
    for (cudaEvent_t e : c->a_ev)
        if (e) cudaEventDestroy(e);
    delete c;
}

clight_status clight_set_atmosphere(clight_ctx *c, const clight_atmosphere *a)
{
    if (!c || !a) return CLIGHT_ERR_ARG;
    if (a->n_layers < 1 || a->n_layers > kMaxLayers) return CLIGHT_ERR_ARG;
    for (int i = 0; i < a->n_layers; ++i) {
        if (!(a->c[i] > 0) || !(a->b[i] >= 0) || !std::isfinite(a->h_lo[i])) return CLIGHT_ERR_ARG;
        if (i > 0 && !(a->h_lo[i] > a->h_lo[i - 1])) return CLIGHT_ERR_ARG;
    }
    if (!(a->K >= 0) || !(a->rho_ref > 0) || !(a->h_top > a->h_obs) || !std::isfinite(a->h_obs))
        return CLIGHT_ERR_ARG;
    if (a->absorption && (!(a->L0 > 0) || !(a->lambda_ref > 0))) return CLIGHT_ERR_ARG;
    if (a->spherical && !(a->R_E > 0)) return CLIGHT_ERR_ARG;
    if (a->n_layers > 1 && a->h_lo[0] > a->h_obs) return CLIGHT_ERR_ARG;
    if (!(a->disp_B >= 0) || !std::isfinite(a->disp_B) || (a->disp_B > 0 && !(a->disp_lref > 0)))
        return CLIGHT_ERR_ARG;
    DevAtm &A = c->atm;
    A = DevAtm{};
    A.n_layers = a->n_layers;
    A.spherical = a->spherical ? 1 : 0;
    A.refraction = a->refraction ? 1 : 0;
    A.absorption = a->absorption ? 1 : 0;
    const double LOG2E = 1.4426950408889634;
    auto Bc = [&](int i) { return a->b[i] / (100.0 * a->c[i]); };   // rho = Bc e^{-h/c}
    for (int i = 0; i < a->n_layers; ++i) {
        A.h_lo[i] = (float)a->h_lo[i];
        A.h_lo_d[i] = a->h_lo[i];
        A.kb[i] = (float)(a->K * Bc(i));
        A.kb_lo[i] = (float)(a->K * Bc(i) - (double)A.kb[i]);
        A.kb_d[i] = a->K * Bc(i);
        A.rb[i] = (float)(Bc(i) / a->rho_ref);
        A.rb_d[i] = Bc(i) / a->rho_ref;
        A.nl2c[i] = (float)(-LOG2E / a->c[i]);
        A.nl2c_lo[i] = (float)(-LOG2E / a->c[i] - (double)A.nl2c[i]);
        A.inv_c_d[i] = 1.0 / a->c[i];
    }
    A.h_top = (float)a->h_top; A.h_top_d = a->h_top;
    A.h_obs = (float)a->h_obs; A.h_obs_d = a->h_obs;
    A.R_E = (float)a->R_E; A.R_E_d = a->spherical ? a->R_E : 0.0;
    A.r_obs_d = a->R_E + a->h_obs; A.r_obs = (float)A.r_obs_d;
    A.inv_r_obs_d = 1.0 / A.r_obs_d; A.inv_r_obs = (float)A.inv_r_obs_d;
    auto delta_at = [&](double h) {
        if (h >= a->h_top) return 0.0;
        int i = 0;
        for (int j = 1; j < a->n_layers; ++j)
            if (h >= a->h_lo[j]) i = j;
        return a->K * Bc(i) * std::exp(-h / a->c[i]);
    };
    auto split = [](double x, float &hi, float &lo) {
        hi = (float)x;
        lo = (float)(x - (double)hi);
    };
    split(a->h_obs, A.hobs_hi, A.hobs_lo);
    split(A.R_E_d, A.re_hi, A.re_lo);
    split(a->h_obs + 2.0 * A.R_E_d, A.k2_hi, A.k2_lo);
    A.k2_d = a->h_obs + 2.0 * A.R_E_d;
    split(3.3356409519815204, A.invc_hi, A.invc_lo);   // ns per m
    A.R_E = (float)A.R_E_d;
    A.delta_obs_d = delta_at(a->h_obs);
    A.delta_obs = (float)A.delta_obs_d;
    A.n_obs = (float)(1.0 + A.delta_obs_d);
    {
        // each layer's largest refractivity above h_obs sits at its bottom
        double dm = A.delta_obs_d;
        for (int i = 0; i < a->n_layers; ++i) {
            double top = i + 1 < a->n_layers ? a->h_lo[i + 1] : a->h_top;
            if (top <= a->h_obs) continue;
            dm = std::max(dm, a->K * Bc(i) * std::exp(-std::max(a->h_lo[i], a->h_obs) / a->c[i]));
        }
        A.delta_max = (float)dm;
    }
    {
        // closed-form layer integrals for the straight-line propagator
        double above_d = 0.0, above_r = 0.0;   // integrals over the layers above layer i
        for (int i = a->n_layers - 1; i >= 0; --i) {
            double top = i + 1 < a->n_layers ? a->h_lo[i + 1] : a->h_top;
            double kd = a->K * Bc(i), kr = Bc(i) / a->rho_ref, ci = a->c[i];
            double et = std::exp(-top / ci);
            A.lay_c[i] = (float)ci;
            A.lay_E[i] = (float)(above_d - ci * kd * et);
            A.lay_F[i] = (float)(above_r - ci * kr * et);
            double bottom = i > 0 ? a->h_lo[i] : (a->n_layers > 1 ? a->h_lo[0] : std::min(a->h_lo[0], a->h_obs));
            double eb = std::exp(-bottom / ci);
            above_d += ci * kd * (eb - et);
            above_r += ci * kr * (eb - et);
        }
        int io = 0;
        for (int j = 1; j < a->n_layers; ++j)
            if (a->h_obs >= a->h_lo[j]) io = j;
        double eo = std::exp(-a->h_obs / a->c[io]);
        A.D_obs = (float)(a->c[io] * a->K * Bc(io) * eo + A.lay_E[io]);
        A.R_obs = (float)(a->c[io] * Bc(io) / a->rho_ref * eo + A.lay_F[io]);
    }
    A.disp = a->disp_B > 0 ? 1 : 0;
    A.disp_B_d = a->disp_B;
    A.disp_ig0_d = A.disp ? 1.0 / (1.0 + a->disp_B / (a->disp_lref * a->disp_lref)) : 1.0;
    A.disp_B = (float)A.disp_B_d;
    A.disp_ig0 = (float)A.disp_ig0_d;
    A.inv_L0_d = a->absorption ? 1.0 / a->L0 : 0.0;
    A.inv_L0 = (float)A.inv_L0_d;
    A.lambda_ref_d = a->absorption ? a->lambda_ref : 1.0;
    A.lambda_ref = (float)A.lambda_ref_d;
    // 3-node Gauss-Legendre on [-1, 1] (closed form): 0, +-sqrt(3/5); 8/9, 5/9
    const double xl = std::sqrt(3.0 / 5.0);
    const double gx[3] = {-xl, 0.0, xl}, gw[3] = {5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0};
    for (int i = 0; i < kGLNodes; ++i) {
        A.gl_x[i] = (float)gx[i]; A.gl_w[i] = (float)gw[i];
        A.gl_x_d[i] = gx[i]; A.gl_w_d[i] = gw[i];
    }
    c->uatm = *a;
    c->atm_set = true;
    ++c->version;
    // Altitude cells of the ray quadrature: each inside one layer and no
    // wider than cell_width scale heights.  Above the altitude where the
    // density has fallen below 1e-9 of its value at the observation level the
    // integrands are negligible, and one last cell reaches the top.
    float cw = c->upar.cell_width > 0 ? c->upar.cell_width : 1.5f;
    const double rho_floor = 1e-9 * (A.delta_obs_d / (a->K > 0 ? a->K : 1.0));
    int nc = 0;
    auto add_cell = [&](double l0, double l1, int i) {
        if (nc >= kMaxCells) return false;
        DevCell &C = A.cells[nc];
        C.lo = (float)l0; C.hi = (float)l1;
        C.kb = A.kb[i]; C.rb = A.rb[i]; C.nl2c = A.nl2c[i];
        C.pad0 = (float)i;                // the cell's layer (the adjoint's tangents)
        A.cell_lo_d[nc] = (double)C.lo;   // identical edges in both precisions
        A.cell_hi_d[nc] = (double)C.hi;
        A.cell_kb_d[nc] = A.kb_d[i]; A.cell_rb_d[nc] = A.rb_d[i]; A.cell_ic_d[nc] = A.inv_c_d[i];
        ++nc;
        return true;
    };
    for (int i = 0; i < a->n_layers; ++i) {
        double lo = std::max(a->h_lo[i], a->h_obs);
        double hi = (i + 1 < a->n_layers) ? a->h_lo[i + 1] : a->h_top;
        hi = std::min(hi, a->h_top);
        if (i == 0 && a->h_lo[0] > a->h_obs) lo = a->h_obs;
        if (!(hi > lo)) continue;
        double h_cut = hi;
        if (a->K > 0 && Bc(i) > 0 && rho_floor > 0) {
            double hc = -a->c[i] * std::log(rho_floor / Bc(i));
            if (hc < hi) h_cut = std::max(lo, hc);
        }
        if (h_cut > lo) {
            int m = std::max(1, (int)std::ceil((h_cut - lo) / (cw * a->c[i])));
            for (int q = 0; q < m; ++q) {
                double l0 = lo + (h_cut - lo) * q / m, l1 = (q + 1 == m) ? h_cut : lo + (h_cut - lo) * (q + 1) / m;
                if (!add_cell(l0, l1, i)) return CLIGHT_ERR_LIMIT;
            }
        }
        if (hi > h_cut && !add_cell(h_cut, hi, i)) return CLIGHT_ERR_LIMIT;
    }
    A.n_cells = nc;
    return CLIGHT_OK;
}

// A clearance map of at most max_cells square cells over the array's box
// widened by 20 m.  A cell's value is the distance from the closed cell to
// the nearest centre, less 1 cm (rounding of the cell index), rounded down to
// kClrQuantum (255: at least 255 quanta).  The byte count is padded to 16.
struct ClrMap {
    std::vector<uint8_t> map;
    int nx, ny;
    double x0, y0, cs;
};
static ClrMap build_clearance(const clight_telescope *t, int n, float xmin, float xmax, float ymin, float ymax,
                              int max_cells)
{
    const double margin = 20.0, q = kClrQuantum, reach = 255.0 * q;
    ClrMap m;
    m.x0 = xmin - margin;
    m.y0 = ymin - margin;
    const double wx = (double)(xmax - xmin) + 2 * margin, wy = (double)(ymax - ymin) + 2 * margin;
    m.cs = std::max(0.5, std::sqrt(wx * wy / max_cells));
    m.nx = (int)std::ceil(wx / m.cs);
    m.ny = (int)std::ceil(wy / m.cs);
    while ((int64_t)m.nx * m.ny > max_cells) {
        m.cs *= 1.05;
        m.nx = (int)std::ceil(wx / m.cs);
        m.ny = (int)std::ceil(wy / m.cs);
    }
    m.map.assign((size_t)m.nx * m.ny, 255);
    for (int i = 0; i < n; ++i) {
        const int ix0 = std::max(0, (int)std::floor((t[i].x - reach - m.x0) / m.cs) - 1);
        const int ix1 = std::min(m.nx - 1, (int)std::floor((t[i].x + reach - m.x0) / m.cs) + 1);
        const int iy0 = std::max(0, (int)std::floor((t[i].y - reach - m.y0) / m.cs) - 1);
        const int iy1 = std::min(m.ny - 1, (int)std::floor((t[i].y + reach - m.y0) / m.cs) + 1);
        for (int iy = iy0; iy <= iy1; ++iy)
            for (int ix = ix0; ix <= ix1; ++ix) {
                const double lx = m.x0 + ix * m.cs, ly = m.y0 + iy * m.cs;
                const double dx = std::max(0.0, std::max(lx - t[i].x, t[i].x - (lx + m.cs)));
                const double dy = std::max(0.0, std::max(ly - t[i].y, t[i].y - (ly + m.cs)));
                const double d = std::sqrt(dx * dx + dy * dy) - 0.01;
                const double v = d <= 0 ? 0.0 : std::floor(d / q);
                const uint8_t u = (uint8_t)std::min(255.0, v);
                uint8_t &cell = m.map[(size_t)iy * m.nx + ix];
                if (u < cell) cell = u;
            }
    }
    m.map.resize((m.map.size() + 15) / 16 * 16, 0);
    return m;
}

clight_status clight_set_telescopes(clight_ctx *c, const clight_telescope *t, int32_t n)
{
    if (!c || !t || n < 1) return CLIGHT_ERR_ARG;
    float xmin = 1e30f, xmax = -1e30f, ymin = 1e30f, ymax = -1e30f, zmin = 1e30f, zmax = -1e30f, rmax = 0;
    for (int i = 0; i < n; ++i) {
        if (!(t[i].R > 0) || !std::isfinite(t[i].x) || !std::isfinite(t[i].y) || !std::isfinite(t[i].z))
            return CLIGHT_ERR_ARG;
        xmin = std::min(xmin, t[i].x - t[i].R); xmax = std::max(xmax, t[i].x + t[i].R);
        ymin = std::min(ymin, t[i].y - t[i].R); ymax = std::max(ymax, t[i].y + t[i].R);
        zmin = std::min(zmin, t[i].z); zmax = std::max(zmax, t[i].z);
        rmax = std::max(rmax, t[i].R);
    }
    // uniform grid: cells of at least 2 Rmax, about one telescope per cell
    double area = std::max(1.0, (double)(xmax - xmin) * (double)(ymax - ymin));
    double gs = std::max(2.0 * rmax, std::sqrt(area / n));
    int nx = (int)std::ceil((xmax - xmin) / gs) + 1, ny = (int)std::ceil((ymax - ymin) / gs) + 1;
    while ((int64_t)nx * ny > (1 << 22)) { gs *= 2; nx = (int)std::ceil((xmax - xmin) / gs) + 1; ny = (int)std::ceil((ymax - ymin) / gs) + 1; }
    std::vector<int> count((size_t)nx * ny + 1, 0), cell_of(n);
    for (int i = 0; i < n; ++i) {
        int ix = std::min(nx - 1, std::max(0, (int)std::floor((t[i].x - xmin) / gs)));
        int iy = std::min(ny - 1, std::max(0, (int)std::floor((t[i].y - ymin) / gs)));
        cell_of[i] = iy * nx + ix;
        count[cell_of[i] + 1]++;
    }
    for (size_t q = 1; q < count.size(); ++q) count[q] += count[q - 1];
    std::vector<int> fill(count.begin(), count.end() - 1), tel_idx(n);
    for (int i = 0; i < n; ++i) tel_idx[fill[cell_of[i]]++] = i;
    std::vector<float4> tv(n);
    for (int i = 0; i < n; ++i) tv[i] = make_float4(t[i].x, t[i].y, t[i].z, t[i].R);

    // clearance maps over the array's box widened by 20 m: a ray whose search
    // radius is below its cell's value cannot reach any sphere.  The coarse
    // map (<= kClrMaxCells) is staged in shared memory by the kernels that
    // trace rays (the hit test of most rays ends with one shared-memory
    // byte); the fine one (<= kClrFineMaxCells) is read from global memory
    // (L1/L2) by the classification, where a smaller cell defers fewer rays.
    ClrMap cm = build_clearance(t, n, xmin, xmax, ymin, ymax, kClrMaxCells);
    ClrMap fm = build_clearance(t, n, xmin, xmax, ymin, ymax, kClrFineMaxCells);
    std::vector<uint8_t> &clr = cm.map;
    const int cnx = cm.nx, cny = cm.ny;
    const double bx0 = cm.x0, by0 = cm.y0, cgs = cm.cs;
    int clr_bytes = (int)clr.size();

    DeviceGuard dg(c->device);
    if (!dg.ok) return CLIGHT_ERR_CUDA;
    if (c->d_tel) cudaFree(c->d_tel);
    if (c->d_cell_start) cudaFree(c->d_cell_start);
    if (c->d_cell_tel) cudaFree(c->d_cell_tel);
    if (c->d_clr) cudaFree(c->d_clr);
    if (c->d_fclr) cudaFree(c->d_fclr);
    c->d_tel = nullptr; c->d_cell_start = nullptr; c->d_cell_tel = nullptr; c->d_clr = nullptr; c->d_fclr = nullptr;
    CK(cudaMalloc((void **)&c->d_tel, sizeof(float4) * n));
    CK(cudaMalloc((void **)&c->d_cell_start, sizeof(int) * count.size()));
    CK(cudaMalloc((void **)&c->d_cell_tel, sizeof(int) * n));
    CK(cudaMalloc((void **)&c->d_clr, (size_t)clr_bytes));
    CK(cudaMalloc((void **)&c->d_fclr, fm.map.size()));
    CK(cudaMemcpy(c->d_tel, tv.data(), sizeof(float4) * n, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->d_cell_start, count.data(), sizeof(int) * count.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->d_cell_tel, tel_idx.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->d_clr, clr.data(), (size_t)clr_bytes, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->d_fclr, fm.map.data(), fm.map.size(), cudaMemcpyHostToDevice));
    DevTel &T = c->tel;
    {
        double sx = 0, sy = 0, sz = 0;
        for (int i = 0; i < n; ++i) { sx += t[i].x; sy += t[i].y; sz += t[i].z; }
        sx /= n; sy /= n; sz /= n;
        double r = 0;
        for (int i = 0; i < n; ++i) {
            double dx = t[i].x - sx, dy = t[i].y - sy, dz = t[i].z - sz;
            r = std::max(r, std::sqrt(dx * dx + dy * dy + dz * dz));
        }
        T.mx = (float)sx; T.my = (float)sy; T.mz = (float)sz;
        T.mr = (float)(r * (1 + 1e-6) + 1e-3);  // covers the rounding of the centre
        double cab = 0;
        for (int i = 0; i < n; ++i) cab = std::max(cab, (double)std::fabs(t[i].x) + std::fabs(t[i].y) + std::fabs(t[i].z));
        T.cabs = (float)(cab * (1 + 1e-6));
    }
    T.clr = c->d_clr; T.cnx = cnx; T.cny = cny; T.clr_bytes = clr_bytes;
    T.cx0 = (float)bx0; T.cy0 = (float)by0; T.inv_cgs = (float)(1.0 / cgs);
    T.fclr = c->d_fclr; T.fcnx = fm.nx; T.fcny = fm.ny;
    T.fcx0 = (float)fm.x0; T.fcy0 = (float)fm.y0; T.finv_cgs = (float)(1.0 / fm.cs);
    T.tel = c->d_tel; T.cell_start = c->d_cell_start; T.cell_tel = c->d_cell_tel;
    T.n_tel = n; T.nx = nx; T.ny = ny;
    T.gx0 = xmin; T.gy0 = ymin; T.gs = (float)gs; T.inv_gs = (float)(1.0 / gs);
    T.xmin = xmin; T.xmax = xmax; T.ymin = ymin; T.ymax = ymax; T.Rmax = rmax; T.zmin = zmin; T.zmax = zmax;
    c->tel_set = true;
    ++c->version;
    return CLIGHT_OK;
}

clight_status clight_set_params(clight_ctx *c, const clight_params *p)
{
    if (!c || !p) return CLIGHT_ERR_ARG;
    if (!(p->lambda1 > 0) || !(p->lambda2 > p->lambda1) || !(p->bunch > 0) || !(p->fluor_yield >= 0) ||
        !(p->fl_lambda1 > 0) || !(p->fl_lambda2 >= p->fl_lambda1) || p->seg_base < 0)
        return CLIGHT_ERR_ARG;
    if (p->block != 0 && (p->block < 32 || p->block > 256 || p->block % 32)) return CLIGHT_ERR_ARG;
    if (p->ctas_per_sm < 0 || p->ctas_per_sm > 32) return CLIGHT_ERR_ARG;
    if (p->precision != CLIGHT_PREC_FLOAT_PAIR && p->precision != CLIGHT_PREC_FP64_GUARD) return CLIGHT_ERR_ARG;
    if (p->cell_width < 0 || p->cell_width > 8) return CLIGHT_ERR_ARG;
    if (p->key_bunch_bits < 0 || p->key_bunch_bits > 32) return CLIGHT_ERR_ARG;
    if (p->cut_mode < CLIGHT_CUT_OFF || p->cut_mode > CLIGHT_CUT_TELESCOPES) return CLIGHT_ERR_ARG;
    if (p->cut_mode != CLIGHT_CUT_OFF && (!(p->cut_deg >= 0) || !(p->cut_deg < 180) ||
                                          !std::isfinite(p->cut_centre[0]) || !std::isfinite(p->cut_centre[1]) ||
                                          !std::isfinite(p->cut_centre[2])))
        return CLIGHT_ERR_ARG;
    if (p->fl_beaming != 0 && p->fl_beaming != 1) return CLIGHT_ERR_ARG;
    if (p->fl_roulette != 0 && p->fl_roulette != 1) return CLIGHT_ERR_ARG;
    if (p->defer_cap > (int64_t(1) << 31)) return CLIGHT_ERR_ARG;
    if (p->trace_all != 0 && p->trace_all != 1) return CLIGHT_ERR_ARG;
    if (p->work_chunk < 0 || p->work_chunk > 64) return CLIGHT_ERR_ARG;
    if (p->propagator != CLIGHT_PROP_EXACT && p->propagator != CLIGHT_PROP_STRAIGHT) return CLIGHT_ERR_ARG;
    if (p->fl_beaming && (!(p->beam_radius > 0) || !std::isfinite(p->beam_radius) ||
                          !std::isfinite(p->beam_centre[0]) || !std::isfinite(p->beam_centre[1]) ||
                          !std::isfinite(p->beam_centre[2])))
        return CLIGHT_ERR_ARG;
    float old_cw = c->upar.cell_width;
    c->upar = *p;
    DevPar &P = c->par;
    const double alpha = 7.2973525643e-3, pi = 3.14159265358979323846;
    P.band_d = 2.0 * pi * alpha * (1.0 / p->lambda1 - 1.0 / p->lambda2) * 1e9;
    P.band = (float)P.band_d;
    P.fta_d = 2.0 * pi * alpha * 1e9;
    P.fta = (float)P.fta_d;
    P.bunch_d = p->bunch;
    P.bunch = (float)p->bunch;
    P.inv_bunch = (float)(1.0 / p->bunch);
    P.il1_d = 1.0 / p->lambda1;
    P.dil_d = 1.0 / p->lambda1 - 1.0 / p->lambda2;
    P.il1 = (float)P.il1_d;
    P.dil = (float)P.dil_d;
    P.fl1_d = p->fl_lambda1;
    P.fdl_d = p->fl_lambda2 - p->fl_lambda1;
    P.fl1 = (float)P.fl1_d;
    P.fdl = (float)P.fdl_d;
    P.fyield_d = p->fluor_yield;
    P.fyield = (float)p->fluor_yield;
    P.seed = p->seed;
    P.stream = p->stream;
    P.seg_base = p->seg_base;
    P.key_off = 0;
    P.cut_mode = p->cut_mode;
    const double cut_deg = p->cut_deg > 0 ? p->cut_deg : 6.0;
    P.cut_cos_d = std::cos(cut_deg * (3.14159265358979323846 / 180.0));
    P.cut_cos = (float)P.cut_cos_d;
    P.cut_cx_d = p->cut_centre[0]; P.cut_cy_d = p->cut_centre[1]; P.cut_cz_d = p->cut_centre[2];
    P.cut_cx = (float)P.cut_cx_d; P.cut_cy = (float)P.cut_cy_d; P.cut_cz = (float)P.cut_cz_d;
    P.cut_rad = (float)(cut_deg * (3.14159265358979323846 / 180.0));
    P.beam = p->fl_beaming;
    P.roulette = p->fl_roulette;
    P.prop = p->propagator;
    P.cull = p->trace_all ? 0 : 1;
    P.chunk = p->work_chunk > 0 ? p->work_chunk : 1;
    P.beam_cx_d = p->beam_centre[0]; P.beam_cy_d = p->beam_centre[1]; P.beam_cz_d = p->beam_centre[2];
    P.beam_r_d = p->beam_radius;
    P.beam_cx = (float)P.beam_cx_d; P.beam_cy = (float)P.beam_cy_d; P.beam_cz = (float)P.beam_cz_d;
    P.beam_r = (float)P.beam_r_d;
    ++c->version;
    if (c->atm_set && p->cell_width != old_cw) {
        clight_atmosphere a = c->uatm;
        return clight_set_atmosphere(c, &a);
    }
    return CLIGHT_OK;
}

}  // extern "C"

// The tables and launch shape the no-allocation entry point needs.
bool clight::ctx_view(clight_ctx *c, CtxView *v)
{
    if (!c || !v || !c->atm_set || !c->tel_set) return false;
    v->atm = c->atm;
    v->tel = c->tel;
    v->par = c->par;
    v->par.cut_tel = c->tel.tel;
    v->par.cut_n_tel = c->tel.n_tel;
    v->par.cut_tx = c->tel.mx; v->par.cut_ty = c->tel.my; v->par.cut_tz = c->tel.mz; v->par.cut_tr = c->tel.mr;
    v->par.cut_cell_start = c->tel.cell_start; v->par.cut_cell_tel = c->tel.cell_tel;
    v->par.cut_cabs = std::max(c->tel.cabs, (float)(std::fabs(v->par.cut_cx_d) + std::fabs(v->par.cut_cy_d) + std::fabs(v->par.cut_cz_d)));
    v->par.cut_nx = c->tel.nx; v->par.cut_ny = c->tel.ny;
    v->par.cut_gx0 = c->tel.gx0; v->par.cut_gy0 = c->tel.gy0; v->par.cut_inv_gs = c->tel.inv_gs;
    v->device = c->device;
    v->n_sm = c->n_sm;
    v->block = c->upar.block > 0 ? c->upar.block : 256;
    v->ctas_per_sm = c->upar.ctas_per_sm > 0 ? c->upar.ctas_per_sm : 3 * 256 / v->block;
    v->precision = c->upar.precision;
    return true;
}

void **clight::ctx_noalloc_slot(clight_ctx *c) { return c ? c->noalloc_slots : nullptr; }

// ------------------------------------------------------------------ pipeline
namespace {

struct Plan {
    int key_bits, group_shift;
    int64_t n_groups, tiles;
};

clight_status prepare(clight_ctx *c, int64_t n_segs, int32_t n_showers, int64_t cap, Plan &pl)
{
    if (!c->atm_set || !c->tel_set) return CLIGHT_ERR_ARG;
    if (n_segs < 0 || n_showers < 1 || cap < 0) return CLIGHT_ERR_ARG;
    if (n_segs > (int64_t(1) << 31)) return CLIGHT_ERR_LIMIT;
    if ((int64_t)n_showers * c->tel.n_tel > (int64_t(1) << 24)) return CLIGHT_ERR_LIMIT;
    if (cap > (int64_t(1) << 32) - 1) return CLIGHT_ERR_LIMIT;
    int gbits = bits_for((int64_t)n_showers * c->tel.n_tel - 1);
    int sbits = bits_for(std::max<int64_t>(n_segs - 1, 0));
    int kbits = c->upar.key_bunch_bits > 0 ? c->upar.key_bunch_bits : 16;
    if (gbits + sbits + kbits > 64) kbits = 64 - gbits - sbits;
    if (kbits < 8) return CLIGHT_ERR_LIMIT;
    pl.key_bits = gbits + sbits + kbits;
    pl.group_shift = sbits + kbits;
    pl.n_groups = (int64_t)n_showers * c->tel.n_tel;
    pl.tiles = std::max<int64_t>(1, (cap + sort_tile_items() - 1) / sort_tile_items());
    c->par.n_showers = n_showers;
    c->par.seg_bits = sbits;
    c->par.k_bits = kbits;
    c->par.cut_tel = c->tel.tel;
    c->par.cut_n_tel = c->tel.n_tel;
    c->par.cut_tx = c->tel.mx; c->par.cut_ty = c->tel.my; c->par.cut_tz = c->tel.mz; c->par.cut_tr = c->tel.mr;
    c->par.cut_cell_start = c->tel.cell_start; c->par.cut_cell_tel = c->tel.cell_tel;
    c->par.cut_cabs = std::max(c->tel.cabs, (float)(std::fabs(c->par.cut_cx_d) + std::fabs(c->par.cut_cy_d) + std::fabs(c->par.cut_cz_d)));
    c->par.cut_nx = c->tel.nx; c->par.cut_ny = c->tel.ny;
    c->par.cut_gx0 = c->tel.gx0; c->par.cut_gy0 = c->tel.gy0; c->par.cut_inv_gs = c->tel.inv_gs;
    uint64_t *g = &c->scratch_gen;
    if (c->rec.ensure(cap, g) || c->keys.ensure(cap, g) || c->keys_alt.ensure(cap, g) ||
        c->vals.ensure(cap, g) || c->vals_alt.ensure(cap, g) || c->hist.ensure(256 * pl.tiles, g) ||
        c->bsums.ensure(scan_block_sums_needed(256 * pl.tiles), g) || c->gstart.ensure(pl.n_groups, g) ||
        c->gend.ensure(pl.n_groups, g))
        return CLIGHT_ERR_CUDA;
    // the deferred-ray queue: by default two entries per step (at least
    // 2^20, at most 2^28) and launches of half as many steps, which covers
    // every workload measured (0.2 to 0.9 queued rays per step); a call that
    // fills it runs again with twice the queue (default) or without it
    const int64_t dc = c->upar.defer_cap;
    const int64_t dflt = std::min<int64_t>(std::max<int64_t>(2 * n_segs, 1 << 20), 1 << 28);
    c->defer_piece = dflt / 2;
    if (c->defer_off || dc < 0 || c->upar.trace_all)
        c->defer_use = 0;
    else if (dc > 0)
        c->defer_use = dc;
    else
        c->defer_use = std::min<int64_t>(std::max(dflt, c->defer_min), int64_t(1) << 31);
    if (c->defer_use > 0 && c->defer.ensure(c->defer_use, g) != cudaSuccess) {
        cudaGetLastError();                      // no room for the queue: trace in place
        c->defer_use = 0;
    }
    return CLIGHT_OK;
}

// chunk > 0: the fused kernel runs once per `chunk` steps, each launch first
// waiting on chunk_ev[i] (the copy of its steps), with the sort keys offset
// to the whole call's step indices; one sort at the end.
cudaError_t enqueue(clight_ctx *c, const clight_segment *segs, int64_t n_segs, const Plan &pl, clight_hit *hits,
                    int64_t cap, int64_t *counts, double *sums, bool fp64, cudaStream_t s, bool capturing,
                    int64_t chunk = 0, const cudaEvent_t *chunk_ev = nullptr)
{
    // inside a capture an event record is a real graph node only when external
    const unsigned evf = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
    DevOut O;
    O.rec = c->rec.p;
    O.keys = c->keys.p;
    O.vals = c->vals.p;
    O.capacity = cap;
    O.ctr = c->d_ctr;
    O.soft_w = 0.0f;
    O.defer = c->defer_use > 0 ? c->defer.p : nullptr;
    O.defer_cap = c->defer_use;
    SortScratch S;
    S.keys_alt = c->keys_alt.p;
    S.vals_alt = c->vals_alt.p;
    S.hist = c->hist.p;
    S.block_sums = c->bsums.p;
    S.max_tiles = pl.tiles;
    S.gstart = c->gstart.p;
    S.gend = c->gend.p;
    cudaError_t e = cudaMemsetAsync(c->d_ctr, 0, sizeof(unsigned long long) * CTR_N, s);
    if (e != cudaSuccess) return e;
    if ((e = cudaEventRecordWithFlags(c->t0, s, evf)) != cudaSuccess) return e;
    if (n_segs > 0) {
        if (fp64) {
            e = launch_trace_fp64(segs, n_segs, c->atm, c->tel, c->par, O, s);
        } else {
            int block = c->upar.block > 0 ? c->upar.block : 256;
            // the first pass of the deferred path fits 4 CTAs of 256 per SM, the in-place kernel 3
            const bool ext = c->par.cut_mode != CLIGHT_CUT_OFF || c->par.beam || c->par.roulette;
            const bool deferred = c->defer_use > 0 &&
                                  !(c->atm.disp && (ext || c->par.prop == CLIGHT_PROP_STRAIGHT)) &&
                                  (c->upar.precision == CLIGHT_PREC_FLOAT_PAIR || !(ext || c->atm.disp));
            int per_sm = c->upar.ctas_per_sm > 0 ? c->upar.ctas_per_sm : (deferred ? 4 : 3) * 256 / block;
            int64_t step = chunk > 0 ? chunk : n_segs;
            // with the default queue size, launches of at most half as many
            // steps as the queue holds entries, so that it does not fill
            if (chunk == 0 && c->defer_use > 0 && c->upar.defer_cap == 0)
                step = std::min(step, std::max<int64_t>(c->defer_piece, 1));
            for (int64_t off = 0, i = 0; off < n_segs && e == cudaSuccess; off += step, ++i) {
                int64_t n = std::min(step, n_segs - off);
                int64_t groups = (n + 31) / 32;
                int64_t grid = std::min<int64_t>((int64_t)c->n_sm * per_sm, (groups * 32 + block - 1) / block);
                grid = std::max<int64_t>(grid, 1);
                DevPar P = c->par;
                if (chunk > 0 && (e = cudaStreamWaitEvent(s, chunk_ev[i], 0)) != cudaSuccess) break;
                if (off > 0) {
                    if ((e = cudaMemsetAsync(c->d_ctr + CTR_WORK, 0, sizeof(unsigned long long), s)) != cudaSuccess)
                        break;
                    P.seg_base += off;
                    P.key_off = off;
                }
                e = launch_trace_fused(segs + off, n, c->atm, c->tel, P, O, c->upar.precision, (int)grid, block, s);
            }
        }
        if (e != cudaSuccess) return e;
    }
    if ((e = cudaEventRecordWithFlags(c->t1, s, evf)) != cudaSuccess) return e;
    e = launch_sort_and_finalize(O, S, pl.key_bits, pl.group_shift, pl.n_groups, hits, counts, sums, s);
    if (e != cudaSuccess) return e;
    if ((e = cudaEventRecordWithFlags(c->t2, s, evf)) != cudaSuccess) return e;
    return cudaMemcpyAsync(c->h_ctr, c->d_ctr, sizeof(unsigned long long) * CTR_N, cudaMemcpyDeviceToHost, s);
}

clight_status finish(clight_ctx *c, int64_t cap, clight_stats *st, int64_t *n_hits)
{
    const unsigned long long *h = c->h_ctr;
    unsigned long long cursor = h[CTR_CURSOR];
    if (n_hits) *n_hits = (int64_t)cursor;
    unsigned long long bits = h[CTR_STATS + ST_STATUS];
    if (st) {
        st->rays = (int64_t)h[CTR_STATS + ST_RAYS];
        st->escaped = (int64_t)h[CTR_STATS + ST_ESCAPED];
        st->under = (int64_t)h[CTR_STATS + ST_UNDER];
        st->turned = (int64_t)h[CTR_STATS + ST_TURNED];
        st->reached = (int64_t)h[CTR_STATS + ST_REACHED];
        st->hits = (int64_t)h[CTR_STATS + ST_HITS];
        st->guarded = (int64_t)h[CTR_STATS + ST_GUARDED];
        st->status = (int64_t)bits;
        st->cells = (int64_t)h[CTR_STATS + ST_CELLS];
        st->cut = (int64_t)h[CTR_STATS + ST_CUT];
        st->skipped = (int64_t)h[CTR_STATS + ST_SKIPPED];
        st->deferred = (int64_t)h[CTR_STATS + ST_DEFERRED];
        st->step_skipped = (int64_t)h[CTR_STATS + ST_STEP_SKIPPED];
    }
    c->timed = true;
    if ((int64_t)cursor > cap) return CLIGHT_ERR_HIT_CAPACITY;
    if (bits & (1ull << CLIGHT_ERR_BAD_SEGMENT)) return CLIGHT_ERR_BAD_SEGMENT;
    if (bits & (1ull << CLIGHT_ERR_LIMIT)) return CLIGHT_ERR_LIMIT;
    return CLIGHT_OK;
}

// After a call: whether a launch found the deferred-ray queue full, in which
// case the call must run again -- with twice the queue (default size, up to
// 2^31 entries, remembered for later calls) or without the queue.
bool defer_retry(clight_ctx *c)
{
    if (!(c->h_ctr[CTR_STATS + ST_STATUS] & (1ull << kBitDeferFull))) return false;
    if (c->upar.defer_cap == 0 && c->defer_use < (int64_t(1) << 31))
        c->defer_min = std::min<int64_t>(2 * c->defer_use, int64_t(1) << 31);
    else
        c->defer_off = true;
    return true;
}

clight_status run_once(clight_ctx *c, const clight_segment *segs, int64_t n_segs, int32_t n_showers,
                       clight_hit *hits, int64_t cap, int64_t *counts, double *sums, void *stream, bool fp64)
{
    Plan pl;
    clight_status r = prepare(c, n_segs, n_showers, cap, pl);
    if (r != CLIGHT_OK) return r;
    cudaStream_t s = (cudaStream_t)stream;
    if (!fp64 && c->upar.use_graph) {
        GraphKey k{segs, n_segs, n_showers, hits, cap, counts, sums, c->version * 1000003ull + c->scratch_gen,
                   c->defer_use};
        if (!c->gexec || !(k == c->gkey)) {
            if (c->gexec) { cudaGraphExecDestroy(c->gexec); c->gexec = nullptr; }
            cudaGraph_t g;
            CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = enqueue(c, segs, n_segs, pl, hits, cap, counts, sums, false, c->cap_stream, true);
            cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &g);
            if (e != cudaSuccess || e2 != cudaSuccess) return CLIGHT_ERR_CUDA;
            e = cudaGraphInstantiate(&c->gexec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) { c->gexec = nullptr; return CLIGHT_ERR_CUDA; }
            c->gkey = k;
        }
        CK(cudaEventRecord(c->ev, s));
        CK(cudaStreamWaitEvent(c->cap_stream, c->ev, 0));
        CK(cudaGraphLaunch(c->gexec, c->cap_stream));
        CK(cudaEventRecord(c->ev, c->cap_stream));
        CK(cudaStreamWaitEvent(s, c->ev, 0));         // later work on `stream` follows the graph
        CK(cudaStreamSynchronize(c->cap_stream));
    } else {
        CK(enqueue(c, segs, n_segs, pl, hits, cap, counts, sums, fp64, s, false));
        CK(cudaStreamSynchronize(s));
    }
    return CLIGHT_OK;
}

clight_status run(clight_ctx *c, const clight_segment *segs, int64_t n_segs, int32_t n_showers, clight_hit *hits,
                  int64_t cap, int64_t *counts, double *sums, clight_stats *st, int64_t *n_hits, void *stream,
                  bool fp64)
{
    if (!c || (n_segs > 0 && !segs) || (cap > 0 && !hits) || !n_hits) return CLIGHT_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(segs) & 15u) return CLIGHT_ERR_ARG;   // records are copied in 16-byte pieces
    DeviceGuard dg(c->device);
    if (!dg.ok) return CLIGHT_ERR_CUDA;
    clight_status r;
    c->defer_off = false;
    do {
        r = run_once(c, segs, n_segs, n_showers, hits, cap, counts, sums, stream, fp64);
    } while (r == CLIGHT_OK && defer_retry(c));
    c->defer_off = false;
    if (r != CLIGHT_OK) return r;
    return finish(c, cap, st, n_hits);
}

}  // namespace

extern "C" {

clight_status clight_trace(clight_ctx *c, const clight_segment *d_segs, int64_t n_segs, int32_t n_showers,
                           clight_hit *d_hits, int64_t cap, int64_t *d_counts, double *d_sums, clight_stats *st,
                           int64_t *h_n_hits, void *stream)
{
    return run(c, d_segs, n_segs, n_showers, d_hits, cap, d_counts, d_sums, st, h_n_hits, stream, false);
}

clight_status clight_trace_fp64(clight_ctx *c, const clight_segment *d_segs, int64_t n_segs, int32_t n_showers,
                                clight_hit *d_hits, int64_t cap, int64_t *d_counts, double *d_sums,
                                clight_stats *st, int64_t *h_n_hits, void *stream)
{
    return run(c, d_segs, n_segs, n_showers, d_hits, cap, d_counts, d_sums, st, h_n_hits, stream, true);
}

clight_status clight_trace_host(clight_ctx *c, const clight_segment *h_segs, int64_t n_segs, int32_t n_showers,
                                clight_hit *h_hits, int64_t cap, int64_t *h_counts, double *h_sums,
                                clight_stats *st, int64_t *h_n_hits, void *stream)
{
    if (!c || (n_segs > 0 && !h_segs) || (cap > 0 && !h_hits) || !h_n_hits || n_showers < 1 || !c->tel_set)
        return CLIGHT_ERR_ARG;
    DeviceGuard dg(c->device);
    if (!dg.ok) return CLIGHT_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    int64_t ng = (int64_t)n_showers * c->tel.n_tel;
    uint64_t *g = &c->scratch_gen;
    if (c->stage_segs.ensure(n_segs, g) || c->stage_hits.ensure(cap, g) || c->stage_counts.ensure(ng, g) ||
        c->stage_sums.ensure(ng, g))
        return CLIGHT_ERR_CUDA;
    clight_status r;
    const int64_t chunk = int64_t(1) << 22;          // 268 MB of steps per copy
    // The steps go to the device by DMA copies (from pinned memory at about
    // 210 GB/s over NVLink-C2C, faster than the kernel reading them in place
    // over the same link), chunk by chunk on the copy stream, each launch
    // waiting for its chunk only, so that copies and tracing overlap.
    if (n_segs >= 2 * chunk) {
        int64_t nck = (n_segs + chunk - 1) / chunk;
        while ((int64_t)c->chunk_ev.size() < nck) {
            cudaEvent_t e;
            CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            c->chunk_ev.push_back(e);
        }
        CK(cudaEventRecord(c->ev, s));                 // earlier work on the staging buffer
        CK(cudaStreamWaitEvent(c->copy_stream, c->ev, 0));
        for (int64_t i = 0; i < nck; ++i) {
            int64_t off = i * chunk, n = std::min(chunk, n_segs - off);
            CK(cudaMemcpyAsync(c->stage_segs.p + off, h_segs + off, sizeof(clight_segment) * (size_t)n,
                               cudaMemcpyHostToDevice, c->copy_stream));
            CK(cudaEventRecord(c->chunk_ev[i], c->copy_stream));
        }
        c->defer_off = false;
        do {
            Plan pl;
            if ((r = prepare(c, n_segs, n_showers, cap, pl)) != CLIGHT_OK) break;
            CK(enqueue(c, c->stage_segs.p, n_segs, pl, c->stage_hits.p, cap, c->stage_counts.p, c->stage_sums.p,
                       false, s, false, chunk, c->chunk_ev.data()));
            CK(cudaStreamSynchronize(s));
        } while (defer_retry(c));
        c->defer_off = false;
        if (r != CLIGHT_OK) return r;
        r = finish(c, cap, st, h_n_hits);
    } else {
        if (n_segs > 0)
            CK(cudaMemcpyAsync(c->stage_segs.p, h_segs, sizeof(clight_segment) * (size_t)n_segs,
                               cudaMemcpyHostToDevice, s));
        r = run(c, c->stage_segs.p, n_segs, n_showers, c->stage_hits.p, cap, c->stage_counts.p, c->stage_sums.p,
                st, h_n_hits, stream, false);
    }
    if (r != CLIGHT_OK && r != CLIGHT_ERR_BAD_SEGMENT && r != CLIGHT_ERR_LIMIT) return r;
    int64_t n = std::min<int64_t>(*h_n_hits, cap);
    if (n > 0) CK(cudaMemcpyAsync(h_hits, c->stage_hits.p, sizeof(clight_hit) * (size_t)n, cudaMemcpyDeviceToHost, s));
    if (h_counts) CK(cudaMemcpyAsync(h_counts, c->stage_counts.p, sizeof(int64_t) * ng, cudaMemcpyDeviceToHost, s));
    if (h_sums) CK(cudaMemcpyAsync(h_sums, c->stage_sums.p, sizeof(double) * ng, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return r;
}

}  // extern "C"

extern "C" clight_status clight_autotune(clight_ctx *c, const clight_segment *d_segs, int64_t n_segs,
                                         int64_t n_sample, int32_t n_showers, clight_hit *d_hits,
                                         int64_t hit_capacity, double bunch_max, int32_t reps, clight_tune *out,
                                         void *stream)
{
    if (!c || !out || !d_segs || n_segs < 1 || n_sample < 1 || reps < 1 || !(bunch_max > 0) || n_showers < 1 ||
        hit_capacity < 0 || (hit_capacity > 0 && !d_hits) || (reinterpret_cast<uintptr_t>(d_segs) & 15u))
        return CLIGHT_ERR_ARG;
    if (!c->atm_set || !c->tel_set) return CLIGHT_ERR_ARG;
    if (n_segs > (int64_t(1) << 31)) return CLIGHT_ERR_LIMIT;
    DeviceGuard dg(c->device);
    if (!dg.ok) return CLIGHT_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const clight_params saved = c->upar;
    // the sample: kBlocks blocks spread evenly over all n_segs steps (every
    // shower of a batch contributes in proportion to its size), gathered into
    // context memory
    const clight_segment *sample = d_segs;
    int64_t n = n_segs;
    if (n_sample < n_segs) {
        const int64_t kBlocks = 64;
        int64_t blk = std::max<int64_t>(32, (n_sample / kBlocks + 31) / 32 * 32);
        int64_t nb = std::min<int64_t>(kBlocks, std::max<int64_t>(1, n_segs / blk));
        n = nb * blk;
        if (c->tune_segs.ensure(n, &c->scratch_gen)) return CLIGHT_ERR_CUDA;
        for (int64_t i = 0; i < nb; ++i) {
            const int64_t off = nb > 1 ? (i * (n_segs - blk)) / (nb - 1) : 0;
            CK(cudaMemcpyAsync(c->tune_segs.p + i * blk, d_segs + off, sizeof(clight_segment) * (size_t)blk,
                               cudaMemcpyDeviceToDevice, s));
        }
        sample = c->tune_segs.p;
    }
    int64_t n_hits = 0;
    clight_stats st;
    struct Timing { double med, spread; };
    // median step time (ms) of one setting over `reps` calls after one warm-up
    // call, and its spread (interquartile range for 5 or more calls, else the
    // range); med < 0 on failure
    auto time_of = [&](const clight_params &p) -> Timing {
        if (clight_set_params(c, &p) != CLIGHT_OK) return {-1.0, 0.0};
        std::vector<float> t;
        for (int r = 0; r < reps + 1; ++r) {
            clight_status e = run(c, sample, n, n_showers, d_hits, hit_capacity, nullptr, nullptr, &st, &n_hits,
                                  stream, false);
            if (e != CLIGHT_OK && e != CLIGHT_ERR_HIT_CAPACITY) return {-1.0, 0.0};
            float ms = 0;
            if (cudaEventElapsedTime(&ms, c->t0, c->t2) != cudaSuccess) return {-1.0, 0.0};
            if (r > 0) t.push_back(ms);
        }
        std::sort(t.begin(), t.end());
        const size_t m = t.size();
        const double spread = m >= 5 ? (double)(t[(3 * m) / 4] - t[m / 4]) : (double)(t[m - 1] - t[0]);
        return {(double)t[m / 2], spread};
    };
    // the library defaults at the caller's bunch size (capped at bunch_max)
    clight_params inc = saved;
    inc.use_graph = 0;
    inc.block = 0;
    inc.ctas_per_sm = 0;
    inc.cell_width = 0;
    inc.work_chunk = 0;
    inc.bunch = std::min(saved.bunch, bunch_max);
    Timing ti = time_of(inc);
    if (ti.med < 0) { clight_set_params(c, &saved); return CLIGHT_ERR_CUDA; }
    const double def_ms = ti.med;
    int tried = 1;
    // one knob at a time from the defaults; a candidate replaces the
    // incumbent only when faster by more than the incumbent's spread (and 1%)
    auto consider = [&](const clight_params &p) -> bool {
        Timing tc = time_of(p);
        ++tried;
        if (tc.med < 0) return false;
        if (tc.med < ti.med - std::max(0.01 * ti.med, ti.spread)) {
            inc = p;
            ti = tc;
        }
        return true;
    };
    bool ok = true;
    std::vector<double> bunches;
    for (double b : {1.0, 2.0, 5.0, bunch_max})
        if (b <= bunch_max && b != inc.bunch && std::find(bunches.begin(), bunches.end(), b) == bunches.end())
            bunches.push_back(b);
    const clight_params base_bunch = inc;
    for (double b : bunches) {
        clight_params p = base_bunch;
        p.bunch = b;
        ok = ok && consider(p);
    }
    struct Shape { int block, per_sm; };
    const Shape shapes[] = {{256, 4}, {256, 3}, {128, 8}, {128, 6}, {64, 16}};
    const clight_params base_shape = inc;
    for (const Shape &sh : shapes) {
        clight_params p = base_shape;
        p.block = sh.block;
        p.ctas_per_sm = sh.per_sm;
        ok = ok && consider(p);
    }
    const clight_params base_chunk = inc;
    for (int ch : {2, 4}) {
        clight_params p = base_chunk;
        p.work_chunk = ch;
        ok = ok && consider(p);
    }
    {
        clight_params p = inc;
        p.cell_width = 1.0f;                 // narrower than the default 1.5 scale heights
        ok = ok && consider(p);
    }
    if (!ok) { clight_set_params(c, &saved); return CLIGHT_ERR_CUDA; }
    clight_tune best{};
    best.block = inc.block > 0 ? inc.block : 256;
    best.ctas_per_sm = inc.ctas_per_sm;
    best.cell_width = inc.cell_width > 0 ? inc.cell_width : 1.5f;
    best.bunch = inc.bunch;
    best.best_ms = ti.med;
    best.default_ms = def_ms;
    best.n_tried = tried;
    best.work_chunk = inc.work_chunk > 0 ? inc.work_chunk : 1;
    best.n_sample = n;
    // the context keeps the choice, with the caller's other settings
    clight_params p = saved;
    p.block = inc.block;
    p.ctas_per_sm = inc.ctas_per_sm;
    p.cell_width = inc.cell_width;
    p.work_chunk = inc.work_chunk;
    p.bunch = inc.bunch;
    clight_status r = clight_set_params(c, &p);
    if (r != CLIGHT_OK) { clight_set_params(c, &saved); return r; }
    *out = best;
    return CLIGHT_OK;
}

extern "C" clight_status clight_trace_adjoint(clight_ctx *c, const clight_segment *d_segs, int64_t n_segs,
                                              int32_t n_showers, const clight_hit *d_hits, int64_t n_hits,
                                              const float *d_gx, const float *d_gy, const float *d_gt,
                                              const double *d_gyield, float soft_s, float soft_w, double *d_yield,
                                              double *h_grad, void *stream)
{
    if (!c || !c->atm_set || !c->tel_set || !h_grad || n_segs < 0 || n_hits < 0 || n_showers < 1)
        return CLIGHT_ERR_ARG;
    if (c->atm.disp) return CLIGHT_ERR_ARG;       // the tangents assume no dispersion
    if (c->par.prop == CLIGHT_PROP_STRAIGHT) return CLIGHT_ERR_ARG;   // they are those of the exact propagator
    if ((n_segs > 0 && !d_segs) || (n_hits > 0 && !d_hits) || !(soft_s > 0) || !(soft_w >= 0) ||
        (reinterpret_cast<uintptr_t>(d_segs) & 15u))
        return CLIGHT_ERR_ARG;
    if (n_segs > (int64_t(1) << 31)) return CLIGHT_ERR_LIMIT;
    if ((int64_t)n_showers * c->tel.n_tel > (int64_t(1) << 24)) return CLIGHT_ERR_LIMIT;
    DeviceGuard dg(c->device);
    if (!dg.ok) return CLIGHT_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    int np = adjoint_params(c->atm.n_layers);
    int blocks = c->n_sm * 8;
    const int64_t n_groups = (int64_t)n_showers * c->tel.n_tel;
    uint64_t *g = &c->scratch_gen;
    if (c->adj_partial.ensure((int64_t)2 * blocks * np, g) || c->adj_out.ensure(np, g) ||
        c->adj_ctr.ensure(CTR_N, g) || c->adj_yfix.ensure(n_groups, g))
        return CLIGHT_ERR_CUDA;
    DevPar P = c->par;
    P.n_showers = n_showers;
    // candidate keys: local step << k_bits | bunch
    P.k_bits = c->upar.key_bunch_bits > 0 ? c->upar.key_bunch_bits : 16;
    P.seg_bits = bits_for(std::max<int64_t>(n_segs - 1, 0));
    P.cut_tel = c->tel.tel;
    P.cut_n_tel = c->tel.n_tel;
    P.cut_tx = c->tel.mx; P.cut_ty = c->tel.my; P.cut_tz = c->tel.mz; P.cut_tr = c->tel.mr;
    P.cut_cell_start = c->tel.cell_start; P.cut_cell_tel = c->tel.cell_tel;
    P.cut_cabs = std::max(c->tel.cabs, (float)(std::fabs(P.cut_cx_d) + std::fabs(P.cut_cy_d) + std::fabs(P.cut_cz_d)));
    P.cut_nx = c->tel.nx; P.cut_ny = c->tel.ny;
    P.cut_gx0 = c->tel.gx0; P.cut_gy0 = c->tel.gy0; P.cut_inv_gs = c->tel.inv_gs;
    CK(cudaMemsetAsync(c->adj_yfix.p, 0, sizeof(unsigned long long) * (size_t)n_groups, s));
    c->a_timed = false;
    CK(cudaEventRecord(c->a_ev[0], s));
    // candidate pass: the rays near a telescope, compacted by the forward
    // kernel (grown and repeated if the list overflows), then sorted, so that
    // the adjoint kernels see them in one order on every call
    int64_t n_cand = 0;
    const unsigned long long *cand = nullptr;
    if ((d_gyield || d_yield) && n_segs > 0) {
        int block = c->upar.block > 0 ? c->upar.block : 256;
        int per_sm = c->upar.ctas_per_sm > 0 ? c->upar.ctas_per_sm : 3 * 256 / block;
        int64_t grid = std::max<int64_t>(1, std::min<int64_t>((int64_t)c->n_sm * per_sm,
                                                              ((n_segs + 31) / 32 * 32 + block - 1) / block));
        int64_t cap = std::max<int64_t>(1 << 20, c->adj_cand.n > 0 ? c->adj_cand.n : n_segs);
        for (int attempt = 0; attempt < 2; ++attempt) {
            if (c->adj_cand.ensure(cap, g)) return CLIGHT_ERR_CUDA;
            DevOut Oc{};
            Oc.keys = c->adj_cand.p;
            Oc.capacity = cap;
            Oc.ctr = c->adj_ctr.p;
            Oc.soft_w = soft_w;
            CK(cudaMemsetAsync(c->adj_ctr.p, 0, sizeof(unsigned long long) * CTR_N, s));
            CK(launch_soft_candidates(d_segs, n_segs, c->atm, c->tel, P, Oc, (int)grid, block, s));
            unsigned long long hc[CTR_N];
            CK(cudaMemcpyAsync(hc, c->adj_ctr.p, sizeof(hc), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            if (hc[CTR_STATS + ST_STATUS] & (1ull << CLIGHT_ERR_LIMIT)) return CLIGHT_ERR_LIMIT;
            n_cand = (int64_t)hc[CTR_CURSOR];
            if (n_cand <= cap) break;
            if (attempt == 1) return CLIGHT_ERR_LIMIT;
            cap = n_cand + n_cand / 8 + 1024;
        }
        CK(cudaEventRecord(c->a_ev[1], s));
        const int64_t tiles = std::max<int64_t>(1, (cap + sort_tile_items() - 1) / sort_tile_items());
        if (c->adj_keys_alt.ensure(cap, g) || c->adj_vals.ensure(cap, g) || c->adj_vals_alt.ensure(cap, g) ||
            c->adj_hist.ensure(256 * tiles, g) || c->adj_bsums.ensure(scan_block_sums_needed(256 * tiles), g))
            return CLIGHT_ERR_CUDA;
        unsigned long long *kin = c->adj_cand.p, *kout = c->adj_keys_alt.p;
        uint32_t *vin = c->adj_vals.p, *vout = c->adj_vals_alt.p;
        CK(radix_sort_pairs(&kin, &vin, &kout, &vout, c->adj_ctr.p, cap, P.seg_bits + P.k_bits, c->adj_hist.p,
                            c->adj_bsums.p, tiles, s));
        cand = kin;
    } else {
        CK(cudaEventRecord(c->a_ev[1], s));
    }
    CK(cudaEventRecord(c->a_ev[2], s));
    CK(launch_adjoint(d_segs, cand, n_cand, d_hits, n_hits, d_gx, d_gy, d_gt, d_gyield, c->adj_yfix.p, d_yield,
                      n_groups, c->atm, c->tel, P, soft_s, soft_w, (float)c->uatm.K, (float)c->uatm.L0,
                      c->adj_partial.p, blocks, c->adj_out.p, s));
    CK(cudaEventRecord(c->a_ev[3], s));
    double out[10];
    CK(cudaMemcpyAsync(out, c->adj_out.p, sizeof(double) * (size_t)np, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int i = 0; i < c->atm.n_layers + 2; ++i) h_grad[i] = out[i];
    c->a_cand = n_cand;
    c->a_hits = n_hits;
    c->a_timed = true;
    return CLIGHT_OK;
}
