// Launcher body of the general Stockham kernel (jt_axis.cuh): picks the template instance
// for log2 L and launches a persistent grid of it (clusters of ksplit CTAs for SPLIT).
#pragma once

#include "jt_launch.hpp"
#include "jt_launch_common.cuh"

namespace jt {

template <class R, int LOG2L, bool FWD, bool SPLIT>
KernInfo& generic_info() {
    static KernInfo ki;
    return ki;
}

template <class R, int LOG2L, bool SPLIT>
cudaError_t generic_launch_one(const dev::AxisDev& A, bool fwd, const typename dev::RealOps<R>::io* in,
                               typename dev::RealOps<R>::io* out, long long nfib, long long inner, int ksplit,
                               cudaStream_t s) {
    using S = dev::Shape<R, LOG2L>;
    constexpr size_t smem = dev::axis_smem_bytes<R, LOG2L, SPLIT>();
    const long long ntiles = (nfib + S::G - 1) / S::G;
    if (fwd)
        return launch_tiles(generic_info<R, LOG2L, true, SPLIT>(), dev::axis_kernel<R, LOG2L, true, SPLIT>, S::THREADS,
                            smem, ntiles, SPLIT ? ksplit : 1, s, A, in, out, nfib, inner);
    return launch_tiles(generic_info<R, LOG2L, false, SPLIT>(), dev::axis_kernel<R, LOG2L, false, SPLIT>, S::THREADS,
                        smem, ntiles, SPLIT ? ksplit : 1, s, A, in, out, nfib, inner);
}

// Dispatch over log2 L in [LO, LOG2L].
template <class R, int LOG2L, int LO, bool SPLIT>
cudaError_t generic_dispatch(int log2L, const dev::AxisDev& A, bool fwd, const typename dev::RealOps<R>::io* in,
                             typename dev::RealOps<R>::io* out, long long nfib, long long inner, int ksplit,
                             cudaStream_t s) {
    if (log2L == LOG2L) return generic_launch_one<R, LOG2L, SPLIT>(A, fwd, in, out, nfib, inner, ksplit, s);
    if constexpr (LOG2L > LO) return generic_dispatch<R, LOG2L - 1, LO, SPLIT>(log2L, A, fwd, in, out, nfib, inner, ksplit, s);
    return cudaErrorInvalidValue;
}

// Default rank split of a general-kernel sweep (occupancy of the plain instance).
template <class R, int LOG2L, int LO>
int generic_auto_ksplit(int log2L, bool fwd, long long nfib, int rank) {
    if (log2L == LOG2L) {
        using S = dev::Shape<R, LOG2L>;
        constexpr size_t smem = dev::axis_smem_bytes<R, LOG2L>();
        KernInfo& ki = fwd ? generic_info<R, LOG2L, true, false>() : generic_info<R, LOG2L, false, false>();
        cudaError_t e = fwd ? kern_init(ki, dev::axis_kernel<R, LOG2L, true, false>, S::THREADS, smem, false)
                            : kern_init(ki, dev::axis_kernel<R, LOG2L, false, false>, S::THREADS, smem, false);
        if (e != cudaSuccess) return 1;
        return auto_ksplit(ki, (nfib + S::G - 1) / S::G, rank);
    }
    if constexpr (LOG2L > LO) return generic_auto_ksplit<R, LOG2L - 1, LO>(log2L, fwd, nfib, rank);
    return 1;
}

}  // namespace jt
