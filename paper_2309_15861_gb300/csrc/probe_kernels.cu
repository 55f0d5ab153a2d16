// probe_kernels.cu -- instruction-throughput probes that give the roofline
// of the tracing kernels its measured denominators: FP32 FMA, MUFU ex2,
// FP64 FMA, 32-bit integer multiply and 3-input logic, each as operations
// per second and per SM per clock on this GPU.  The path is bound by
// arithmetic issue (no dense contraction, little HBM traffic), so these
// rates -- not a copy bandwidth or a GEMM rate -- bound it.
//
// Each probe runs 8 independent dependency chains per thread in a full grid
// (every SM at its thread limit), so the pipe, not latency, limits it.  The
// operations are inline PTX with volatile asm, so the compiler neither
// removes nor merges them; each thread stores its chains' sum, so nothing is
// dead.  The SM clock during a probe is measured on the device: thread 0 of
// every block reads clock64() and %globaltimer at its start and end.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <vector>

#include "internal.h"

namespace clight {

__device__ __forceinline__ unsigned long long gtimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

enum ProbeKind { PROBE_FFMA = 0, PROBE_MUFU = 1, PROBE_DFMA = 2, PROBE_IMAD = 3, PROBE_LOP3 = 4 };

template <int KIND>
__global__ void __launch_bounds__(256, 8) k_probe(int iters, float seed, float *sink, unsigned long long *clk)
{
    unsigned long long c0 = 0, t0 = 0;
    if (threadIdx.x == 0) {
        c0 = clock64();
        t0 = gtimer_ns();
    }
    const float fs = seed + 1.0e-7f * (float)threadIdx.x;
    float r = 0.0f;
    if (KIND == PROBE_FFMA) {
        float a[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) a[j] = fs + (float)j;
        const float m = 0.999999f, c = 1.0e-6f;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int j = 0; j < 8; ++j) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(a[j]) : "f"(m), "f"(c));
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) r += a[j];
    } else if (KIND == PROBE_MUFU) {
        float a[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) a[j] = 1.0e-3f * (fs + (float)j);
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int j = 0; j < 8; ++j) asm volatile("ex2.approx.ftz.f32 %0, %0;" : "+f"(a[j]));
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) r += a[j];
    } else if (KIND == PROBE_DFMA) {
        double a[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) a[j] = (double)fs + (double)j;
        const double m = 0.9999999, c = 1.0e-7;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int j = 0; j < 8; ++j) asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(a[j]) : "d"(m), "d"(c));
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) r += (float)a[j];
    } else if (KIND == PROBE_IMAD) {
        uint32_t a[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) a[j] = __float_as_uint(fs) + (uint32_t)j;
        const uint32_t m = 0xD2511F53u, c = 0x9E3779B9u;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int j = 0; j < 8; ++j) asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a[j]) : "r"(m), "r"(c));
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) r += (float)(a[j] & 0xffffu);
    } else {
        uint32_t a[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) a[j] = __float_as_uint(fs) + (uint32_t)j;
        const uint32_t m = 0xCD9E8D57u, c = 0xBB67AE85u;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int j = 0; j < 8; ++j)
                asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a[j]) : "r"(m), "r"(c));   // a ^ m ^ c
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) r += (float)(a[j] & 0xffffu);
    }
    sink[blockIdx.x * blockDim.x + threadIdx.x] = r;
    if (threadIdx.x == 0) {
        clk[2 * blockIdx.x] = clock64() - c0;
        clk[2 * blockIdx.x + 1] = gtimer_ns() - t0;
    }
}

}  // namespace clight

extern "C" clight_status clight_measure_pipes(int device, clight_pipe_rates *out)
{
    using namespace clight;
    if (!out) return CLIGHT_ERR_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return CLIGHT_ERR_NO_DEVICE;
    }
    DeviceGuard dg(device);
    if (!dg.ok) return CLIGHT_ERR_NO_DEVICE;
    int n_sm = 0;
    if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return CLIGHT_ERR_CUDA;
    int max_thr = 0;
    if (cudaDeviceGetAttribute(&max_thr, cudaDevAttrMaxThreadsPerMultiProcessor, device) != cudaSuccess)
        return CLIGHT_ERR_CUDA;
    const int block = 256;
    const int grid = n_sm * std::max(1, max_thr / block);
    float *sink = nullptr;
    unsigned long long *clk = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    clight_status st = CLIGHT_OK;
    if (cudaMalloc((void **)&sink, sizeof(float) * (size_t)grid * block) != cudaSuccess ||
        cudaMalloc((void **)&clk, sizeof(unsigned long long) * 2 * (size_t)grid) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        st = CLIGHT_ERR_CUDA;
    std::vector<unsigned long long> hc(2 * (size_t)grid);
    // one probe: best of 3 timed launches after one warm-up
    auto run = [&](auto kern, int iters, double ops_per_iter, double *per_s, double *mhz) -> bool {
        float best = 1e30f;
        for (int r = 0; r < 4; ++r) {
            if (cudaEventRecord(e0, 0) != cudaSuccess) return false;
            kern<<<grid, block>>>(iters, 0.5f, sink, clk);
            if (cudaEventRecord(e1, 0) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return false;
            float ms = 0;
            if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) return false;
            if (r > 0) best = std::min(best, ms);
        }
        if (cudaMemcpy(hc.data(), clk, sizeof(unsigned long long) * hc.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
            return false;
        double cyc = 0, ns = 0;
        for (int b = 0; b < grid; ++b) { cyc += (double)hc[2 * b]; ns += (double)hc[2 * b + 1]; }
        *mhz = ns > 0 ? 1e3 * cyc / ns : 0.0;
        *per_s = (double)grid * block * iters * ops_per_iter / (best * 1e-3);
        return true;
    };
    clight_pipe_rates o{};
    o.n_sm = n_sm;
    if (st == CLIGHT_OK) {
        // a few milliseconds per launch on GB300
        bool ok = run(k_probe<PROBE_FFMA>, 65536, 8.0, &o.ffma_per_s, &o.ffma_mhz) &&
                  run(k_probe<PROBE_MUFU>, 8192, 8.0, &o.mufu_ex2_per_s, &o.mufu_mhz) &&
                  run(k_probe<PROBE_DFMA>, 512, 8.0, &o.dfma_per_s, &o.dfma_mhz) &&
                  run(k_probe<PROBE_IMAD>, 16384, 8.0, &o.imad_per_s, &o.imad_mhz) &&
                  run(k_probe<PROBE_LOP3>, 32768, 8.0, &o.lop3_per_s, &o.lop3_mhz);
        if (!ok || cudaGetLastError() != cudaSuccess) st = CLIGHT_ERR_CUDA;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    if (clk) cudaFree(clk);
    if (st == CLIGHT_OK) *out = o;
    return st;
}
