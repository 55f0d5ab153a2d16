// trace_twopass.cu -- launches of the two-pass forward path: the first
// pass (k_classify, with the features the call uses) and k_trace_deferred
// for the rays it queued.
#include "trace_kernels.cuh"

namespace clight {

template <class P, bool SPH, bool REFR, int FEAT>
static void launch_deferred_pair(const clight_segment *segs, int64_t n_segs, const DevAtm &A, const DevTel &T,
                                 const DevPar &Pp, const DevOut &O, int grid, int block, cudaStream_t s)
{
    constexpr bool EXT = (FEAT & FEAT_EXT) != 0;
    // the queue's fill and work counters
    cudaMemsetAsync(O.ctr + CTR_DEFER, 0, 2 * sizeof(unsigned long long), s);
    {
        // the classification kernel, with the features the call uses
        constexpr bool DISP = (FEAT & FEAT_DISP) != 0;
        const int smem = cls_smem_bytes(block, T, EXT);
        cudaFuncSetAttribute(k_classify<SPH, REFR, EXT, DISP>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        k_classify<SPH, REFR, EXT, DISP><<<grid, block, smem, s>>>(segs, n_segs, A, T, Pp, O);
    }
    // the second pass as many CTAs as are resident at once (its own
    // register and shared-memory limits)
    const int smem2 = !EXT && T.clr ? T.clr_bytes : 0;
    int dev = 0, n_sm = 1, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace_deferred<SPH, REFR, FEAT, P>, block, smem2);
    const int grid2 = std::max(1, std::min(grid, n_sm * std::max(per_sm, 1)));
    k_trace_deferred<SPH, REFR, FEAT, P><<<grid2, block, smem2, s>>>(segs, A, T, Pp, O);
}

template <class P, int FEAT>
static void two_pass_geo(const clight_segment *segs, int64_t n_segs, const DevAtm &A, const DevTel &T,
                         const DevPar &Pp, const DevOut &O, int grid, int block, cudaStream_t s)
{
    if (A.spherical && A.refraction)
        launch_deferred_pair<P, true, true, FEAT>(segs, n_segs, A, T, Pp, O, grid, block, s);
    else if (A.spherical)
        launch_deferred_pair<P, true, false, FEAT>(segs, n_segs, A, T, Pp, O, grid, block, s);
    else if (A.refraction)
        launch_deferred_pair<P, false, true, FEAT>(segs, n_segs, A, T, Pp, O, grid, block, s);
    else
        launch_deferred_pair<P, false, false, FEAT>(segs, n_segs, A, T, Pp, O, grid, block, s);
}

template <>
void launch_two_pass<df>(int feat, const clight_segment *segs, int64_t n_segs, const DevAtm &A, const DevTel &T,
                         const DevPar &Pp, const DevOut &O, int grid, int block, cudaStream_t s)
{
    switch (feat) {
    case 0: two_pass_geo<df, 0>(segs, n_segs, A, T, Pp, O, grid, block, s); break;
    case FEAT_STRAIGHT: two_pass_geo<df, FEAT_STRAIGHT>(segs, n_segs, A, T, Pp, O, grid, block, s); break;
    case FEAT_EXT: two_pass_geo<df, FEAT_EXT>(segs, n_segs, A, T, Pp, O, grid, block, s); break;
    case FEAT_EXT | FEAT_STRAIGHT:
        two_pass_geo<df, FEAT_EXT | FEAT_STRAIGHT>(segs, n_segs, A, T, Pp, O, grid, block, s);
        break;
    case FEAT_DISP: two_pass_geo<df, FEAT_DISP>(segs, n_segs, A, T, Pp, O, grid, block, s); break;
    default: break;
    }
}

template <>
void launch_two_pass<double>(int feat, const clight_segment *segs, int64_t n_segs, const DevAtm &A,
                             const DevTel &T, const DevPar &Pp, const DevOut &O, int grid, int block, cudaStream_t s)
{
    switch (feat) {
    case 0: two_pass_geo<double, 0>(segs, n_segs, A, T, Pp, O, grid, block, s); break;
    case FEAT_STRAIGHT: two_pass_geo<double, FEAT_STRAIGHT>(segs, n_segs, A, T, Pp, O, grid, block, s); break;
    default: break;
    }
}

}  // namespace clight
