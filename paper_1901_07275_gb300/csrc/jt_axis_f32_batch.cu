// Batched FP32 launches of the four-step kernel without rank split: one launch serves the
// concatenated CTA tiles of many jobs (axis sweeps of different plans) with the same FFT
// length, direction and stride kind.
#include "jt_launch_warp.cuh"

namespace jt {

cudaError_t launch_axis_f32_batched(int log2L, bool fwd, bool strided, const dev::BatchJob* jobs, int njobs,
                                    long long total_tiles, const dev::BatchPtrs& ptrs, int ksplit, cudaStream_t s) {
    if (!f32_warp_path(log2L)) return cudaErrorInvalidValue;
    if (ksplit > 1) return launch_axis_f32_batched_split(log2L, fwd, strided, jobs, njobs, total_tiles, ptrs, ksplit, s);
    return warp_batched_dispatch<F32_WARP_MAX_LOG2L, false>(log2L, fwd, strided, jobs, njobs, total_tiles, ptrs, 1, s);
}

}  // namespace jt
