// Launchers of the fused axis kernels, one translation unit per precision.
#pragma once

#include <cuda_runtime.h>

#include "jt_axis.cuh"
#include "jt_warp.cuh"

namespace jt {

// Apply one axis (forward or adjoint) to nfib fibres: fibre f = (o, q) with o = f / inner,
// q = f % inner starts at o * n * inner + q and has stride inner.  in may equal out.
cudaError_t launch_axis_f32(const dev::AxisDev& A, int log2L, bool fwd, const float* in, float* out,
                            long long nfib, long long inner, cudaStream_t s);
cudaError_t launch_axis_dw(const dev::AxisDev& A, int log2L, bool fwd, const double* in, double* out,
                           long long nfib, long long inner, cudaStream_t s);

// One launch of the four-step kernel over the concatenated tiles of several jobs of the same
// FFT length, direction and stride kind (jobs: a device array ordered by tile_begin).
cudaError_t launch_axis_f32_batched(int log2L, bool fwd, bool strided, const dev::BatchJob* jobs, int njobs,
                                    long long total_tiles, const dev::BatchPtrs& ptrs, cudaStream_t s);
// Fibres per CTA tile of the four-step kernel (tile counting for batched jobs).
int f32_warp_tile_fibres(int log2L);

constexpr int MAX_LOG2L_F32 = 14;
constexpr int MAX_LOG2L_DW = 13;

// FP32 lengths 16..4096 use the four-step kernel (jt_warp.cuh), whose dense-block table rows
// are padded with zeros to length L: vblk[c * L + j] = sqrt(w_j) P~_c(t_j) for j < n.
constexpr int F32_WARP_MIN_LOG2L = 4;
constexpr int F32_WARP_MAX_LOG2L = 12;
constexpr bool f32_warp_path(int log2L) { return log2L >= F32_WARP_MIN_LOG2L && log2L <= F32_WARP_MAX_LOG2L; }

}  // namespace jt
