// trace_inplace.cu -- launches of the forward path: the fused kernel with
// every ray traced in place (the binary64-guard and feature-complete
// instances, or no deferred-ray queue), the dispatch to the two-pass path,
// and the plain binary64 kernel.
#include "trace_kernels.cuh"

namespace clight {

template <class P, int FEAT>
static void launch_fused_pe(const clight_segment *segs, int64_t n_segs, const DevAtm &A, const DevTel &T,
                            const DevPar &Pp, const DevOut &O, int grid, int block, cudaStream_t s)
{
    int smem = fused_smem_bytes_f(block, T, (FEAT & FEAT_EXT) != 0);  // < 48 KB for block <= 256
    // the two-pass path for every binary32-pair instance with one propagator
    // compiled in (the straight-line propagator moves a ray by no more than
    // the bound the first pass uses: its first-order shortfall is that
    // bound's first term)
    // (binary64 precise steps: the same two passes for the default feature
    // set and the straight line, the classification being precision-free)
    if constexpr ((FEAT & FEAT_RUNTIME) == 0 &&
                  (std::is_same<P, df>::value || (FEAT & (FEAT_EXT | FEAT_DISP)) == 0)) {
        if (O.defer) {
            launch_two_pass<P>(FEAT, segs, n_segs, A, T, Pp, O, grid, block, s);
            return;
        }
    }
    if (A.spherical && A.refraction)
        k_trace_fused<P, true, true, false, false, FEAT><<<grid, block, smem, s>>>(segs, n_segs, A, T, Pp, O);
    else if (A.spherical)
        k_trace_fused<P, true, false, false, false, FEAT><<<grid, block, smem, s>>>(segs, n_segs, A, T, Pp, O);
    else if (A.refraction)
        k_trace_fused<P, false, true, false, false, FEAT><<<grid, block, smem, s>>>(segs, n_segs, A, T, Pp, O);
    else
        k_trace_fused<P, false, false, false, false, FEAT><<<grid, block, smem, s>>>(segs, n_segs, A, T, Pp, O);
}

// the variant without the angular cut, beaming and the straight-line propagator when none is on
template <class P>
static void launch_fused_p(const clight_segment *segs, int64_t n_segs, const DevAtm &A, const DevTel &T,
                           const DevPar &Pp, const DevOut &O, int grid, int block, cudaStream_t s)
{
    const bool ext = Pp.cut_mode != CLIGHT_CUT_OFF || Pp.beam || Pp.roulette;
    const bool str = Pp.prop == CLIGHT_PROP_STRAIGHT;
    if ((!std::is_same<P, df>::value && (ext || A.disp)) || (A.disp && (ext || str)))
        launch_fused_pe<P, FEAT_ALL>(segs, n_segs, A, T, Pp, O, grid, block, s);
    else if (A.disp)
        launch_fused_pe<P, FEAT_DISP>(segs, n_segs, A, T, Pp, O, grid, block, s);
    else if (ext && str)
        launch_fused_pe<P, FEAT_EXT | FEAT_STRAIGHT>(segs, n_segs, A, T, Pp, O, grid, block, s);
    else if (ext)
        launch_fused_pe<P, FEAT_EXT>(segs, n_segs, A, T, Pp, O, grid, block, s);
    else if (str)
        launch_fused_pe<P, FEAT_STRAIGHT>(segs, n_segs, A, T, Pp, O, grid, block, s);
    else
        launch_fused_pe<P, 0>(segs, n_segs, A, T, Pp, O, grid, block, s);
}

cudaError_t launch_trace_fused(const clight_segment *segs, int64_t n_segs, const DevAtm &A, const DevTel &T,
                               const DevPar &P, const DevOut &O, int precision, int grid, int block,
                               cudaStream_t s)
{
    if (precision == CLIGHT_PREC_FP64_GUARD)
        launch_fused_p<double>(segs, n_segs, A, T, P, O, grid, block, s);
    else
        launch_fused_p<df>(segs, n_segs, A, T, P, O, grid, block, s);
    return cudaGetLastError();
}

cudaError_t launch_trace_fp64(const clight_segment *segs, int64_t n_segs, const DevAtm &A, const DevTel &T,
                              const DevPar &P, const DevOut &O, cudaStream_t s)
{
    int block = 128;
    int64_t grid = (n_segs + block - 1) / block;
    if (grid < 1) grid = 1;
    if (A.spherical && A.refraction)
        k_trace_fp64<true, true><<<(unsigned)grid, block, 0, s>>>(segs, n_segs, A, T, P, O);
    else if (A.spherical)
        k_trace_fp64<true, false><<<(unsigned)grid, block, 0, s>>>(segs, n_segs, A, T, P, O);
    else if (A.refraction)
        k_trace_fp64<false, true><<<(unsigned)grid, block, 0, s>>>(segs, n_segs, A, T, P, O);
    else
        k_trace_fp64<false, false><<<(unsigned)grid, block, 0, s>>>(segs, n_segs, A, T, P, O);
    return cudaGetLastError();
}

}  // namespace clight
