// Launchers of the fused axis kernels.  Every launcher takes ksplit, the number of CTAs that
// share a tile of fibres by splitting its rank terms (a thread-block cluster; 1 = no split).
#pragma once

#include <cuda_runtime.h>

#include "jt_axis.cuh"
#include "jt_warp.cuh"

namespace jt {

// Apply one axis (forward or adjoint) to nfib fibres: fibre f = (o, q) with o = f / inner,
// q = f % inner starts at o * n * inner + q and has stride inner.  in may equal out: a tile
// stores only its own fibres, after all of its CTAs have read them.
cudaError_t launch_axis_f32(const dev::AxisDev& A, int log2L, bool fwd, const float* in, float* out,
                            long long nfib, long long inner, int ksplit, cudaStream_t s);
cudaError_t launch_axis_dw(const dev::AxisDev& A, int log2L, bool fwd, const double* in, double* out,
                           long long nfib, long long inner, int ksplit, cudaStream_t s);
// rank-split instances (separate translation units)
cudaError_t launch_axis_f32_split(const dev::AxisDev& A, int log2L, bool fwd, const float* in, float* out,
                                  long long nfib, long long inner, int ksplit, cudaStream_t s);
cudaError_t launch_axis_dw_split(const dev::AxisDev& A, int log2L, bool fwd, const double* in, double* out,
                                 long long nfib, long long inner, int ksplit, cudaStream_t s);

// One launch of the four-step kernel over the concatenated tiles of several jobs of the same
// FFT length, direction and stride kind (jobs: a device array ordered by tile_begin).
cudaError_t launch_axis_f32_batched(int log2L, bool fwd, bool strided, const dev::BatchJob* jobs, int njobs,
                                    long long total_tiles, const dev::BatchPtrs& ptrs, int ksplit, cudaStream_t s);
cudaError_t launch_axis_f32_batched_split(int log2L, bool fwd, bool strided, const dev::BatchJob* jobs, int njobs,
                                          long long total_tiles, const dev::BatchPtrs& ptrs, int ksplit,
                                          cudaStream_t s);
// Fibres per CTA tile of the four-step kernel (tile counting for batched jobs).
int f32_warp_tile_fibres(int log2L);

// The rank split a sweep of nfib fibres gets by default (1, 2, 4 or 8): CTAs per tile are
// doubled while the split tiles still fit in one wave and every CTA keeps a rank term.
int auto_ksplit_f32(int log2L, bool fwd, bool strided, long long nfib, int rank);
int auto_ksplit_dw(int log2L, bool fwd, long long nfib, int rank);

constexpr int MAX_LOG2L_F32 = 14;
constexpr int MAX_LOG2L_DW = 14;
// Double-word lengths up to 2^13 run in shared memory (jt_axis.cuh); 2^14 as two half-length
// transforms (jt_axis_dw_big.cu).
constexpr int DW_SMEM_MAX_LOG2L = 13;

// L = 16384 double-word sweeps (two half-length transforms a rank term, partial sums in the
// plan's buffer B.part, a fixed-order reduction into out).  in may equal out.
cudaError_t launch_axis_dw_big(const dev::BigAxisDev& B, bool fwd, const double* in, double* out, long long nfib,
                               long long inner, cudaStream_t s);
cudaError_t dw_big_init();  // kernel attributes (before any capture)
size_t dw_big_smem_bytes();

// FP32 lengths 16..4096 use the four-step kernel (jt_warp.cuh), whose dense-block table rows
// are padded with zeros to length L: vblk[c * L + j] = sqrt(w_j) P~_c(t_j) for j < n.
constexpr int F32_WARP_MIN_LOG2L = 4;
constexpr int F32_WARP_MAX_LOG2L = 12;
constexpr bool f32_warp_path(int log2L) { return log2L >= F32_WARP_MIN_LOG2L && log2L <= F32_WARP_MAX_LOG2L; }

}  // namespace jt
