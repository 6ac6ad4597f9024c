// Batched FP32 launches of the four-step kernel: one launch serves the concatenated CTA tiles
// of many jobs (axis sweeps of different plans) with the same FFT length, direction and
// stride kind.
#include <algorithm>
#include <mutex>

#include "jt_launch.hpp"

namespace jt {

template <int LOG2L, bool FWD, bool STRIDED>
static cudaError_t launch_warp_batched(const dev::BatchJob* jobs, int njobs, long long total_tiles,
                                       const dev::BatchPtrs& ptrs, cudaStream_t s) {
    using S = dev::WShape<LOG2L>;
    constexpr size_t smem = dev::warp_smem_bytes<LOG2L>(STRIDED);
    auto kern = dev::warp_axis_kernel<LOG2L, FWD, STRIDED, true>;
    static std::once_flag once;
    static int blocks_per_sm = 0, num_sms = 0;
    static cudaError_t init_err = cudaSuccess;
    std::call_once(once, [&]() {
        int dev_id = 0;
        cudaError_t e = cudaGetDevice(&dev_id);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev_id);
        if (e == cudaSuccess && smem > 48 * 1024)
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, kern, S::THREADS, smem);
        init_err = e;
    });
    if (init_err != cudaSuccess) return init_err;
    if (blocks_per_sm < 1) return cudaErrorInvalidConfiguration;
    long long grid = std::min<long long>(total_tiles, (long long)num_sms * blocks_per_sm);
    if (grid < 1) return cudaSuccess;
    dev::AxisDev none{};
    kern<<<(unsigned)grid, S::THREADS, smem, s>>>(none, nullptr, nullptr, 0, 1, jobs, njobs, total_tiles, ptrs);
    return cudaGetLastError();
}

template <int LOG2L>
static cudaError_t warp_batched_dispatch(int log2L, bool fwd, bool strided, const dev::BatchJob* jobs, int njobs,
                                         long long total_tiles, const dev::BatchPtrs& ptrs, cudaStream_t s) {
    if (log2L == LOG2L) {
        if (fwd)
            return strided ? launch_warp_batched<LOG2L, true, true>(jobs, njobs, total_tiles, ptrs, s)
                           : launch_warp_batched<LOG2L, true, false>(jobs, njobs, total_tiles, ptrs, s);
        return strided ? launch_warp_batched<LOG2L, false, true>(jobs, njobs, total_tiles, ptrs, s)
                       : launch_warp_batched<LOG2L, false, false>(jobs, njobs, total_tiles, ptrs, s);
    }
    if constexpr (LOG2L > F32_WARP_MIN_LOG2L)
        return warp_batched_dispatch<LOG2L - 1>(log2L, fwd, strided, jobs, njobs, total_tiles, ptrs, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_axis_f32_batched(int log2L, bool fwd, bool strided, const dev::BatchJob* jobs, int njobs,
                                    long long total_tiles, const dev::BatchPtrs& ptrs, cudaStream_t s) {
    if (!f32_warp_path(log2L)) return cudaErrorInvalidValue;
    return warp_batched_dispatch<F32_WARP_MAX_LOG2L>(log2L, fwd, strided, jobs, njobs, total_tiles, ptrs, s);
}

}  // namespace jt
