// FP32 rank-split instances of the fused axis kernels (a cluster of ksplit CTAs per tile).
#include "jt_launch_impl.cuh"
#include "jt_launch_warp.cuh"

namespace jt {

cudaError_t launch_axis_f32_split(const dev::AxisDev& A, int log2L, bool fwd, const float* in, float* out,
                                  long long nfib, long long inner, int ksplit, cudaStream_t s) {
    if (log2L < 0 || log2L > MAX_LOG2L_F32) return cudaErrorInvalidValue;
    if (f32_warp_path(log2L)) return warp_dispatch<F32_WARP_MAX_LOG2L, true>(log2L, A, fwd, in, out, nfib, inner, ksplit, s);
    if (log2L < F32_WARP_MIN_LOG2L)
        return generic_dispatch<float, F32_WARP_MIN_LOG2L - 1, 0, true>(log2L, A, fwd, in, out, nfib, inner, ksplit, s);
    return generic_dispatch<float, MAX_LOG2L_F32, F32_WARP_MAX_LOG2L + 1, true>(log2L, A, fwd, in, out, nfib, inner,
                                                                                ksplit, s);
}

}  // namespace jt
