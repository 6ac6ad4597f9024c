// Double-word (hi + lo FP32) instances of the fused axis kernels (L = 1 .. 8192).
#include "jt_launch_impl.cuh"

namespace jt {
cudaError_t launch_axis_dw(const dev::AxisDev& A, int log2L, bool fwd, const double* in, double* out,
                           long long nfib, long long inner, cudaStream_t s) {
    if (log2L < 0 || log2L > MAX_LOG2L_DW) return cudaErrorInvalidValue;
    return dispatch<dev::dw, MAX_LOG2L_DW>(log2L, A, fwd, in, out, nfib, inner, s);
}
}  // namespace jt
