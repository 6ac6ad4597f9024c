// FP32 instances of the fused axis kernels without rank split: the four-step kernel for
// L = 16 .. 4096, the general Stockham kernel for L = 1 .. 8 and 8192 .. 16384.
#include "jt_launch_impl.cuh"
#include "jt_launch_warp.cuh"

namespace jt {

int f32_warp_tile_fibres(int log2L) { return 256 >> (log2L - 4); }

cudaError_t launch_axis_f32(const dev::AxisDev& A, int log2L, bool fwd, const float* in, float* out,
                            long long nfib, long long inner, int ksplit, cudaStream_t s) {
    if (log2L < 0 || log2L > MAX_LOG2L_F32) return cudaErrorInvalidValue;
    if (ksplit > 1) return launch_axis_f32_split(A, log2L, fwd, in, out, nfib, inner, ksplit, s);
    if (f32_warp_path(log2L)) return warp_dispatch<F32_WARP_MAX_LOG2L, false>(log2L, A, fwd, in, out, nfib, inner, 1, s);
    if (log2L < F32_WARP_MIN_LOG2L)
        return generic_dispatch<float, F32_WARP_MIN_LOG2L - 1, 0, false>(log2L, A, fwd, in, out, nfib, inner, 1, s);
    return generic_dispatch<float, MAX_LOG2L_F32, F32_WARP_MAX_LOG2L + 1, false>(log2L, A, fwd, in, out, nfib, inner, 1, s);
}

int auto_ksplit_f32(int log2L, bool fwd, bool strided, long long nfib, int rank) {
    if (log2L < 0 || log2L > MAX_LOG2L_F32) return 1;
    if (f32_warp_path(log2L)) return warp_auto_ksplit<F32_WARP_MAX_LOG2L>(log2L, fwd, strided, nfib, rank);
    if (log2L < F32_WARP_MIN_LOG2L) return generic_auto_ksplit<float, F32_WARP_MIN_LOG2L - 1, 0>(log2L, fwd, nfib, rank);
    return generic_auto_ksplit<float, MAX_LOG2L_F32, F32_WARP_MAX_LOG2L + 1>(log2L, fwd, nfib, rank);
}

}  // namespace jt
