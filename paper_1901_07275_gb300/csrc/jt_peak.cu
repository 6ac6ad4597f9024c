// FP32 issue-rate probe: the denominator of the axis kernels' roofline, measured rather than
// derived.  Each thread runs ACC independent chains of fused multiply-adds, either one FP32
// FMA per instruction (fma.rn.f32) or two per instruction (fma.rn.f32x2, sm_100 and later),
// over a persistent grid of CTAs per SM; the caller times the launch on its stream.  The
// multiplier and addend are kernel arguments, so nothing folds at compile time, and every
// accumulator is summed into one store per thread, so no chain is dead.
#include <cuda_runtime.h>

#include "jt.h"

namespace {

constexpr int ACC = 8;
constexpr int THREADS = 256;
constexpr int CTAS_PER_SM = 4;

__global__ void __launch_bounds__(THREADS) fma_scalar(float m, float c, long long iters, float* sink) {
    float a[ACC];
#pragma unroll
    for (int i = 0; i < ACC; ++i) a[i] = (float)(threadIdx.x + i);
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int i = 0; i < ACC; ++i) a[i] = fmaf(a[i], m, c);
    }
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < ACC; ++i) s += a[i];
    sink[blockIdx.x * THREADS + threadIdx.x] = s;
}

__global__ void __launch_bounds__(THREADS) fma_paired(float m, float c, long long iters, float* sink) {
    unsigned long long a[ACC];
    unsigned long long mm, cc;
    asm("mov.b64 %0, {%1, %1};" : "=l"(mm) : "f"(m));
    asm("mov.b64 %0, {%1, %1};" : "=l"(cc) : "f"(c));
#pragma unroll
    for (int i = 0; i < ACC; ++i) {
        const float lo = (float)(threadIdx.x + i), hi = (float)(threadIdx.x + 2 * i);
        asm("mov.b64 %0, {%1, %2};" : "=l"(a[i]) : "f"(lo), "f"(hi));
    }
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int i = 0; i < ACC; ++i) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[i]) : "l"(mm), "l"(cc));
    }
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < ACC; ++i) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a[i]));
        s += lo + hi;
    }
    sink[blockIdx.x * THREADS + threadIdx.x] = s;
}

}  // namespace

extern "C" {

jt_status jt_probe_fp32_fma(int paired, int64_t iters, float* sink, int64_t sink_len, double* flops,
                            jt_stream_t stream) {
    if (iters < 1 || !sink || !flops) return JT_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return JT_ECUDA;
    const long long ctas = (long long)sms * CTAS_PER_SM;
    if (sink_len < ctas * THREADS) return JT_EINVAL;
    const float m = 0.999999f, c = 1e-7f;
    cudaStream_t s = (cudaStream_t)stream;
    if (paired)
        fma_paired<<<(unsigned)ctas, THREADS, 0, s>>>(m, c, (long long)iters, sink);
    else
        fma_scalar<<<(unsigned)ctas, THREADS, 0, s>>>(m, c, (long long)iters, sink);
    if (cudaGetLastError() != cudaSuccess) return JT_ECUDA;
    // FMAs per thread: iters x 16 x ACC instructions, each 1 (scalar) or 2 (paired) FMAs of 2 flops
    *flops = (double)ctas * THREADS * (double)iters * 16.0 * ACC * (paired ? 2.0 : 1.0) * 2.0;
    return JT_OK;
}

}  // extern "C"
