// Double-word (hi + lo FP32) instances of the fused axis kernels (L = 1 .. 8192; 16384 in jt_axis_dw_big.cu), no rank split.
#include "jt_launch_impl.cuh"

namespace jt {

cudaError_t launch_axis_dw(const dev::AxisDev& A, int log2L, bool fwd, const double* in, double* out,
                           long long nfib, long long inner, int ksplit, cudaStream_t s) {
    if (log2L < 0 || log2L > DW_SMEM_MAX_LOG2L) return cudaErrorInvalidValue;
    if (ksplit > 1) return launch_axis_dw_split(A, log2L, fwd, in, out, nfib, inner, ksplit, s);
    return generic_dispatch<dev::dw, DW_SMEM_MAX_LOG2L, 0, false>(log2L, A, fwd, in, out, nfib, inner, 1, s);
}

int auto_ksplit_dw(int log2L, bool fwd, long long nfib, int rank) {
    if (log2L < 0 || log2L > DW_SMEM_MAX_LOG2L) return 1;
    return generic_auto_ksplit<dev::dw, DW_SMEM_MAX_LOG2L, 0>(log2L, fwd, nfib, rank);
}

}  // namespace jt
