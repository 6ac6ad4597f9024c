// Launcher bodies of the four-step kernel (jt_warp.cuh), single sweeps and batched launches,
// in plain and rank-split (clusters of ksplit CTAs) instances.
#pragma once

#include "jt_launch.hpp"
#include "jt_launch_common.cuh"

namespace jt {

template <int LOG2L, bool FWD, bool STRIDED, bool BATCHED, bool SPLIT>
KernInfo& warp_info() {
    static KernInfo ki;
    return ki;
}

template <int LOG2L, bool FWD, bool STRIDED, bool SPLIT>
cudaError_t warp_launch_one(const dev::AxisDev& A, const float* in, float* out, long long nfib, long long inner,
                            int ksplit, cudaStream_t s) {
    using S = dev::WShape<LOG2L>;
    constexpr size_t smem = dev::warp_smem_bytes<LOG2L>(STRIDED, dev::WStream<LOG2L, FWD, false, SPLIT>::value);
    static const dev::BatchPtrs no_ptrs{};
    const dev::BatchJob* no_jobs = nullptr;
    const long long ntiles = (nfib + S::FT - 1) / S::FT;
    return launch_tiles(warp_info<LOG2L, FWD, STRIDED, false, SPLIT>(),
                        dev::warp_axis_kernel<LOG2L, FWD, STRIDED, false, SPLIT>, S::THREADS, smem, ntiles,
                        SPLIT ? ksplit : 1, s, A, in, out, nfib, inner, no_jobs, 0, 0LL, no_ptrs);
}

template <int LOG2L, bool SPLIT>
cudaError_t warp_dispatch(int log2L, const dev::AxisDev& A, bool fwd, const float* in, float* out, long long nfib,
                          long long inner, int ksplit, cudaStream_t s) {
    if (log2L == LOG2L) {
        const bool strided = inner > 1;
        if (fwd)
            return strided ? warp_launch_one<LOG2L, true, true, SPLIT>(A, in, out, nfib, inner, ksplit, s)
                           : warp_launch_one<LOG2L, true, false, SPLIT>(A, in, out, nfib, inner, ksplit, s);
        return strided ? warp_launch_one<LOG2L, false, true, SPLIT>(A, in, out, nfib, inner, ksplit, s)
                       : warp_launch_one<LOG2L, false, false, SPLIT>(A, in, out, nfib, inner, ksplit, s);
    }
    if constexpr (LOG2L > F32_WARP_MIN_LOG2L)
        return warp_dispatch<LOG2L - 1, SPLIT>(log2L, A, fwd, in, out, nfib, inner, ksplit, s);
    return cudaErrorInvalidValue;
}

template <int LOG2L, bool FWD, bool STRIDED, bool SPLIT>
cudaError_t warp_launch_batched(const dev::BatchJob* jobs, int njobs, long long total_tiles, const dev::BatchPtrs& ptrs,
                                int ksplit, cudaStream_t s) {
    using S = dev::WShape<LOG2L>;
    constexpr size_t smem = dev::warp_smem_bytes<LOG2L>(STRIDED);
    const dev::AxisDev none{};
    const float* no_in = nullptr;
    float* no_out = nullptr;
    return launch_tiles(warp_info<LOG2L, FWD, STRIDED, true, SPLIT>(),
                        dev::warp_axis_kernel<LOG2L, FWD, STRIDED, true, SPLIT>, S::THREADS, smem, total_tiles,
                        SPLIT ? ksplit : 1, s, none, no_in, no_out, 0LL, 1LL, jobs, njobs, total_tiles, ptrs);
}

template <int LOG2L, bool SPLIT>
cudaError_t warp_batched_dispatch(int log2L, bool fwd, bool strided, const dev::BatchJob* jobs, int njobs,
                                  long long total_tiles, const dev::BatchPtrs& ptrs, int ksplit, cudaStream_t s) {
    if (log2L == LOG2L) {
        if (fwd)
            return strided ? warp_launch_batched<LOG2L, true, true, SPLIT>(jobs, njobs, total_tiles, ptrs, ksplit, s)
                           : warp_launch_batched<LOG2L, true, false, SPLIT>(jobs, njobs, total_tiles, ptrs, ksplit, s);
        return strided ? warp_launch_batched<LOG2L, false, true, SPLIT>(jobs, njobs, total_tiles, ptrs, ksplit, s)
                       : warp_launch_batched<LOG2L, false, false, SPLIT>(jobs, njobs, total_tiles, ptrs, ksplit, s);
    }
    if constexpr (LOG2L > F32_WARP_MIN_LOG2L)
        return warp_batched_dispatch<LOG2L - 1, SPLIT>(log2L, fwd, strided, jobs, njobs, total_tiles, ptrs, ksplit, s);
    return cudaErrorInvalidValue;
}

// Default rank split of a four-step sweep (occupancy of the plain single-sweep instance).
template <int LOG2L>
int warp_auto_ksplit(int log2L, bool fwd, bool strided, long long nfib, int rank) {
    if (log2L == LOG2L) {
        using S = dev::WShape<LOG2L>;
        const long long ntiles = (nfib + S::FT - 1) / S::FT;
        KernInfo* ki;
        cudaError_t e;
        if (fwd && strided) {
            ki = &warp_info<LOG2L, true, true, false, false>();
            e = kern_init(*ki, dev::warp_axis_kernel<LOG2L, true, true, false, false>, S::THREADS,
                          dev::warp_smem_bytes<LOG2L>(true, dev::WStream<LOG2L, true, false, false>::value), false);
        } else if (fwd) {
            ki = &warp_info<LOG2L, true, false, false, false>();
            e = kern_init(*ki, dev::warp_axis_kernel<LOG2L, true, false, false, false>, S::THREADS,
                          dev::warp_smem_bytes<LOG2L>(false, dev::WStream<LOG2L, true, false, false>::value), false);
        } else if (strided) {
            ki = &warp_info<LOG2L, false, true, false, false>();
            e = kern_init(*ki, dev::warp_axis_kernel<LOG2L, false, true, false, false>, S::THREADS,
                          dev::warp_smem_bytes<LOG2L>(true, dev::WStream<LOG2L, false, false, false>::value), false);
        } else {
            ki = &warp_info<LOG2L, false, false, false, false>();
            e = kern_init(*ki, dev::warp_axis_kernel<LOG2L, false, false, false, false>, S::THREADS,
                          dev::warp_smem_bytes<LOG2L>(false, dev::WStream<LOG2L, false, false, false>::value), false);
        }
        if (e != cudaSuccess) return 1;
        return auto_ksplit(*ki, ntiles, rank);
    }
    if constexpr (LOG2L > F32_WARP_MIN_LOG2L) return warp_auto_ksplit<LOG2L - 1>(log2L, fwd, strided, nfib, rank);
    return 1;
}

}  // namespace jt
