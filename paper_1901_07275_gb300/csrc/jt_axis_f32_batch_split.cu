// Batched FP32 launches of the four-step kernel with rank split (a cluster of ksplit CTAs
// per tile).
#include "jt_launch_warp.cuh"

namespace jt {

cudaError_t launch_axis_f32_batched_split(int log2L, bool fwd, bool strided, const dev::BatchJob* jobs, int njobs,
                                          long long total_tiles, const dev::BatchPtrs& ptrs, int ksplit,
                                          cudaStream_t s) {
    if (!f32_warp_path(log2L)) return cudaErrorInvalidValue;
    return warp_batched_dispatch<F32_WARP_MAX_LOG2L, true>(log2L, fwd, strided, jobs, njobs, total_tiles, ptrs, ksplit, s);
}

}  // namespace jt
