// Launch helpers shared by the axis-kernel translation units: per-instance occupancy, a
// persistent grid of at most one wave, and cluster launches for the rank split.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

namespace jt {

// Occupancy facts of one kernel instance, measured on first use.
struct KernInfo {
    std::once_flag once;
    cudaError_t err = cudaSuccess;
    int num_sms = 0;
    int blocks_per_sm = 0;
    int max_clusters[4] = {0, 0, 0, 0};  // clusters of 2, 4, 8, 16 CTAs that fit at once
};

inline int cluster_slot(int ksplit) { return ksplit == 2 ? 0 : ksplit == 4 ? 1 : ksplit == 8 ? 2 : ksplit == 16 ? 3 : -1; }

template <class K>
cudaError_t kern_init(KernInfo& ki, K kern, int threads, size_t smem, bool split) {
    std::call_once(ki.once, [&]() {
        int dev_id = 0;
        cudaError_t e = cudaGetDevice(&dev_id);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ki.num_sms, cudaDevAttrMultiProcessorCount, dev_id);
        if (e == cudaSuccess && smem > 48 * 1024)
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ki.blocks_per_sm, kern, threads, smem);
        if (e == cudaSuccess && split) {
            for (int q = 0; q < 3; ++q) {  // portable cluster sizes 2, 4, 8
                const unsigned cs = 2u << q;
                cudaLaunchConfig_t cfg = {};
                cudaLaunchAttribute at[1];
                at[0].id = cudaLaunchAttributeClusterDimension;
                at[0].val.clusterDim.x = cs;
                at[0].val.clusterDim.y = 1;
                at[0].val.clusterDim.z = 1;
                cfg.gridDim = dim3(cs, 1, 1);
                cfg.blockDim = dim3(threads, 1, 1);
                cfg.dynamicSmemBytes = smem;
                cfg.attrs = at;
                cfg.numAttrs = 1;
                int n = 0;
                if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
                    cudaGetLastError();
                    n = 0;
                }
                ki.max_clusters[q] = n;
            }
        }
        ki.err = e;
    });
    return ki.err;
}

// Launch `kern` over ntiles CTA tiles: a persistent grid of at most one wave; with ksplit > 1
// each tile is shared by a cluster of ksplit CTAs (the kernel must be a rank-split instance).
template <class K, class... Args>
cudaError_t launch_tiles(KernInfo& ki, K kern, int threads, size_t smem, long long ntiles, int ksplit,
                         cudaStream_t s, Args... args) {
    cudaError_t e = kern_init(ki, kern, threads, smem, ksplit > 1);
    if (e != cudaSuccess) return e;
    if (ntiles < 1) return cudaSuccess;
    if (ksplit <= 1) {
        if (ki.blocks_per_sm < 1) return cudaErrorInvalidConfiguration;
        const long long grid = std::min<long long>(ntiles, (long long)ki.num_sms * ki.blocks_per_sm);
        kern<<<(unsigned)grid, threads, smem, s>>>(args...);
        return cudaGetLastError();
    }
    // a cluster size that does not fit falls back to the next smaller one (1: a plain launch of
    // the split instance, whose CTAs then take every rank term)
    while (ksplit > 1 && (cluster_slot(ksplit) < 0 || cluster_slot(ksplit) > 2 || ki.max_clusters[cluster_slot(ksplit)] < 1))
        ksplit /= 2;
    if (ksplit <= 1) {
        if (ki.blocks_per_sm < 1) return cudaErrorInvalidConfiguration;
        const long long grid = std::min<long long>(ntiles, (long long)ki.num_sms * ki.blocks_per_sm);
        kern<<<(unsigned)grid, threads, smem, s>>>(args...);
        return cudaGetLastError();
    }
    const int q = cluster_slot(ksplit);
    const long long nc = std::min<long long>(ntiles, ki.max_clusters[q]);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)ksplit;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)(nc * ksplit), 1, 1);
    cfg.blockDim = dim3(threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, kern, args...);
    return e;
}

// The rank split a sweep gets by default: double the CTAs per tile (up to 8) while all of
// them still find a slot in one wave of the plain instance and every CTA keeps a rank term.
inline int auto_ksplit(const KernInfo& plain, long long ntiles, int rank) {
    const long long slots = (long long)plain.num_sms * plain.blocks_per_sm;
    int S = 1;
    while (S < 8 && 2 * S <= rank && ntiles * 2 * S <= slots) S *= 2;
    return S;
}

}  // namespace jt
