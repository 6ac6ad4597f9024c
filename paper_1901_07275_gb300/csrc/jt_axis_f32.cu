// FP32 instances of the fused axis kernels (L = 1 .. 16384).
#include "jt_launch_impl.cuh"

namespace jt {
cudaError_t launch_axis_f32(const dev::AxisDev& A, int log2L, bool fwd, const float* in, float* out,
                            long long nfib, long long inner, cudaStream_t s) {
    if (log2L < 0 || log2L > MAX_LOG2L_F32) return cudaErrorInvalidValue;
    return dispatch<float, MAX_LOG2L_F32>(log2L, A, fwd, in, out, nfib, inner, s);
}
}  // namespace jt
