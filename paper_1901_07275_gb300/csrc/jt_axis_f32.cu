// FP32 instances of the fused axis kernels: the four-step kernel for L = 16 .. 4096, the
// general Stockham kernel otherwise (L = 1 .. 8 and 8192 .. 16384).
#include "jt_launch_impl.cuh"
#include "jt_warp.cuh"

namespace jt {

template <int LOG2L, bool FWD, bool STRIDED>
static cudaError_t launch_warp(const dev::AxisDev& A, const float* in, float* out, long long nfib, long long inner,
                               cudaStream_t s) {
    using S = dev::WShape<LOG2L>;
    constexpr size_t smem = dev::warp_smem_bytes<LOG2L>(STRIDED);
    auto kern = dev::warp_axis_kernel<LOG2L, FWD, STRIDED>;
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
    long long ntiles = (nfib + S::FT - 1) / S::FT;
    long long grid = std::min<long long>(ntiles, (long long)num_sms * blocks_per_sm);
    if (grid < 1) return cudaSuccess;
    static const dev::BatchPtrs no_ptrs{};
    kern<<<(unsigned)grid, S::THREADS, smem, s>>>(A, in, out, nfib, inner, nullptr, 0, 0, no_ptrs);
    return cudaGetLastError();
}

template <int LOG2L>
static cudaError_t warp_dispatch(int log2L, const dev::AxisDev& A, bool fwd, const float* in, float* out,
                                 long long nfib, long long inner, cudaStream_t s) {
    if (log2L == LOG2L) {
        const bool strided = inner > 1;
        if (fwd)
            return strided ? launch_warp<LOG2L, true, true>(A, in, out, nfib, inner, s)
                           : launch_warp<LOG2L, true, false>(A, in, out, nfib, inner, s);
        return strided ? launch_warp<LOG2L, false, true>(A, in, out, nfib, inner, s)
                       : launch_warp<LOG2L, false, false>(A, in, out, nfib, inner, s);
    }
    if constexpr (LOG2L > F32_WARP_MIN_LOG2L) return warp_dispatch<LOG2L - 1>(log2L, A, fwd, in, out, nfib, inner, s);
    return cudaErrorInvalidValue;
}

int f32_warp_tile_fibres(int log2L) { return 256 >> (log2L - 4); }

cudaError_t launch_axis_f32(const dev::AxisDev& A, int log2L, bool fwd, const float* in, float* out,
                            long long nfib, long long inner, cudaStream_t s) {
    if (log2L < 0 || log2L > MAX_LOG2L_F32) return cudaErrorInvalidValue;
    if (f32_warp_path(log2L)) return warp_dispatch<F32_WARP_MAX_LOG2L>(log2L, A, fwd, in, out, nfib, inner, s);
    return dispatch<float, MAX_LOG2L_F32>(log2L, A, fwd, in, out, nfib, inner, s);
}

}  // namespace jt
