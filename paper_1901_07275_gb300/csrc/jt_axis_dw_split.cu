// Double-word rank-split instances of the fused axis kernels (a cluster of ksplit CTAs per tile).
#include "jt_launch_impl.cuh"

namespace jt {

cudaError_t launch_axis_dw_split(const dev::AxisDev& A, int log2L, bool fwd, const double* in, double* out,
                                 long long nfib, long long inner, int ksplit, cudaStream_t s) {
    if (log2L < 0 || log2L > DW_SMEM_MAX_LOG2L) return cudaErrorInvalidValue;
    return generic_dispatch<dev::dw, DW_SMEM_MAX_LOG2L, 0, true>(log2L, A, fwd, in, out, nfib, inner, ksplit, s);
}

}  // namespace jt
