// Shared launcher body: picks the template instance for log2 L, sizes a persistent grid
// from the occupancy of that instance, and launches it.
#pragma once

#include <mutex>

#include "jt_launch.hpp"

namespace jt {

template <class R, int LOG2L>
static cudaError_t launch_one(const dev::AxisDev& A, bool fwd, const typename dev::RealOps<R>::io* in,
                              typename dev::RealOps<R>::io* out, long long nfib, long long inner,
                              cudaStream_t s) {
    using S = dev::Shape<R, LOG2L>;
    constexpr size_t smem = dev::axis_smem_bytes<R, LOG2L>();
    static std::once_flag once[2];
    static int blocks_per_sm[2] = {0, 0};
    static int num_sms = 0;
    static cudaError_t init_err[2] = {cudaSuccess, cudaSuccess};
    auto kern = fwd ? dev::axis_kernel<R, LOG2L, true> : dev::axis_kernel<R, LOG2L, false>;
    const int w = fwd ? 0 : 1;
    std::call_once(once[w], [&]() {
        int dev_id = 0;
        cudaError_t e = cudaGetDevice(&dev_id);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev_id);
        if (e == cudaSuccess && smem > 48 * 1024)
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm[w], kern, S::THREADS, smem);
        init_err[w] = e;
    });
    if (init_err[w] != cudaSuccess) return init_err[w];
    if (blocks_per_sm[w] < 1) return cudaErrorInvalidConfiguration;
    long long ntiles = (nfib + S::G - 1) / S::G;
    long long grid = std::min<long long>(ntiles, (long long)num_sms * blocks_per_sm[w]);
    if (grid < 1) return cudaSuccess;
    kern<<<(unsigned)grid, S::THREADS, smem, s>>>(A, in, out, nfib, inner);
    return cudaGetLastError();
}

template <class R, int LOG2L>
static cudaError_t dispatch(int log2L, const dev::AxisDev& A, bool fwd, const typename dev::RealOps<R>::io* in,
                            typename dev::RealOps<R>::io* out, long long nfib, long long inner, cudaStream_t s) {
    if (log2L == LOG2L) return launch_one<R, LOG2L>(A, fwd, in, out, nfib, inner, s);
    if constexpr (LOG2L > 0) return dispatch<R, LOG2L - 1>(log2L, A, fwd, in, out, nfib, inner, s);
    return cudaErrorInvalidValue;
}

}  // namespace jt
