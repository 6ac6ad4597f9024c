// Double-word axis kernels for FFT length L = 16384 (split plans with 8192 < n <= 16384).
//
// A length-L transform of a complex double-word does not fit one CTA's shared memory
// (16 bytes a value, 256 KiB), so the IDFT is split by the parity of the frequency index
// (decimation in frequency for the forward, in time for the adjoint) into two transforms of
// length L' = L / 2 that the Stockham machinery of jt_axis.cuh runs in shared memory:
//
//   forward (Eq. eq:oneJ):  y[m] = sum_nu x[nu] w_L^{m nu}
//                                = E[m mod L'] + w_L^m O[m mod L'],
//     E = IDFT_L'(x[0::2]), O = IDFT_L'(x[1::2]); for every rank term k and parity p the
//     kernel transforms x_p[q] = v_k[2q + p] alpha[2q + p] and adds
//     Re(u_k^(p)[j] Y_p[m_j mod L']) with u_k^(p)[j] = u_k[j] w_L^{p m_j} (a plan table).
//   adjoint (Eq. eq:oneJinv): Y[2q + p] = sum_{m <= L/2} z[m] w_L^{m p} w_L'^{m q}: the bins
//     m_j mod L' with factors u_k^(p)[j] (the same tables) feed IDFT_L', whose output q is
//     degree 2q + p.
//
// So a sweep applies 2 r half-length terms.  They are spread over S CTAs per fibre (S chosen
// from the fibre count), each CTA adding its terms into its own row of a plan-owned partial
// sum buffer in global memory (thread-owned entries, no atomics); a second kernel adds the S
// rows of each fibre in a fixed order and stores the result, so results are deterministic.
// The dense low-degree block is added by the first CTA of each fibre.
#include <cuda_runtime.h>

#include <algorithm>

#include "jt_axis.cuh"
#include "jt_launch.hpp"

namespace jt {
namespace dev {

namespace {

constexpr int BIG_LOG2L = 14;
constexpr int HALF_LOG2 = BIG_LOG2L - 1;
using HS = Shape<dw, HALF_LOG2>;  // E = 8, T = 1024, one fibre per CTA
static_assert(HS::T == 1024 && HS::E == 8 && HS::G == 1, "half-length Stockham geometry");
constexpr int BIG_THREADS = HS::T;
constexpr size_t BIG_SMEM = sizeof(dw) * 2 * (size_t)HS::PADL;

__device__ __forceinline__ long long big_fibre_offset(long long f, int n, long long inner) {
    const long long o = f / inner;
    return o * ((long long)n * inner) + (f - o * inner);
}

// Partial sums of fibres [f0, f0 + nf) (grid: nf x S CTAs; CTA b takes fibre f0 + b / S and
// the half-length terms [2 r c / S, 2 r (c + 1) / S) with c = b % S) into part[b][0..n).
template <bool FWD>
__global__ void __launch_bounds__(BIG_THREADS, 1)
    dw_big_kernel(BigAxisDev B, const double* in, long long f0, long long nf, long long inner, int S) {
    constexpr int Lh = HS::L, E = HS::E, T = HS::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    dw* sre = reinterpret_cast<dw*>(smem_raw);
    dw* sim = sre + HS::PADL;
    const int t = threadIdx.x;
    const long long fl = blockIdx.x / S;
    const int c = (int)(blockIdx.x % S);
    if (fl >= nf) return;  // whole CTA
    const int n = B.n, nu0 = B.nu0, rank = B.rank;
    const long long base = big_fibre_offset(f0 + fl, n, inner);
    dw* acc = B.part + (size_t)blockIdx.x * n;
    const Cx<dw>* __restrict__ vtab = B.vtab;
    const Cx<dw>* __restrict__ tw = B.tw2;
    const int units = 2 * rank;
    const int ub = (int)(((long long)units * c) / S), ue = (int)(((long long)units * (c + 1)) / S);

    // Entries of acc are owned by one thread each: forward point j by thread j % T; adjoint
    // degree nu = 2 q + p by thread q % T (q = nu / 2).
    if constexpr (FWD) {
        for (int j = t; j < n; j += T) {
            dw s = RealOps<dw>::zero();
            if (c == 0)
                for (int cc = 0; cc < nu0; ++cc)
                    s = s + B.vblk[(size_t)cc * n + j] * RealOps<dw>::from_io(in[base + (long long)cc * inner]);
            acc[j] = s;
        }
    } else {
#pragma unroll
        for (int e = 0; e < E; ++e)
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                const int nu = 2 * (t + T * e) + p;
                if (nu < n) acc[nu] = RealOps<dw>::zero();
            }
    }

    for (int uidx = ub; uidx < ue; ++uidx) {
        const int k = uidx >> 1, p = uidx & 1;
        const Cx<dw>* __restrict__ uk = (p ? B.utab1 : B.utab) + (size_t)k * n;
        Cx<dw> x[E];
        if constexpr (FWD) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int nu = 2 * (t + T * e) + p;
                const dw a = (nu < n) ? RealOps<dw>::from_io(in[base + (long long)nu * inner]) : RealOps<dw>::zero();
                x[e] = cscale(vtab[(size_t)k * (2 * Lh) + nu], a);
            }
        } else {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int m = t + T * e;
                Cx<dw> z{RealOps<dw>::zero(), RealOps<dw>::zero()};
                for (int q = B.bin_ptr2[m]; q < B.bin_ptr2[m + 1]; ++q) {
                    const int j = B.bin_idx2[q];
                    z = z + cscale(uk[j], RealOps<dw>::from_io(in[base + (long long)j * inner]));
                }
                x[e] = z;
            }
        }
        __syncthreads();  // the previous term is done with the shared buffer
        fft<dw, HALF_LOG2>(x, sre, sim, tw, t, 0);
        if constexpr (FWD) {
            __syncthreads();  // the last pass is done reading the buffer
#pragma unroll
            for (int e = 0; e < E; ++e) XBuf<dw>{sre, sim}.put<HS>(t + T * e, x[e]);
            __syncthreads();
            for (int j = t; j < n; j += T) {
                const Cx<dw> y = XBuf<dw>{sre, sim}.get<HS>(B.mtab2[j]);
                acc[j] = acc[j] + re_mul(uk[j], y);
            }
        } else {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int nu = 2 * (t + T * e) + p;
                if (nu < n) acc[nu] = acc[nu] + re_mul(vtab[(size_t)k * (2 * Lh) + nu], x[e]);
            }
        }
    }

    if constexpr (!FWD) {
        // dense block: alpha_cc = sum_j vblk[cc][j] g_j (cc < nu0), first CTA of the fibre;
        // per degree a warp-shuffle sum and a fixed-order sum over the 32 warps
        if (c == 0) {
            dw* red = sre;  // [32] partials, free after the last FFT
            const int lane = t & 31, warp = t >> 5;
            for (int cc = 0; cc < nu0; ++cc) {
                dw s = RealOps<dw>::zero();
                for (int j = t; j < n; j += T)
                    s = s + B.vblk[(size_t)cc * n + j] * RealOps<dw>::from_io(in[base + (long long)j * inner]);
#pragma unroll
                for (int off = 16; off >= 1; off >>= 1) {
                    const dw o{__shfl_xor_sync(0xffffffffu, s.hi, off), __shfl_xor_sync(0xffffffffu, s.lo, off)};
                    s = s + o;
                }
                __syncthreads();  // previous degree's partials read (and the FFT done with red)
                if (lane == 0) red[warp] = s;
                __syncthreads();
                if (t == (cc >> 1)) {  // owner of degree cc = 2 q + p with q = cc / 2 < T
                    dw tot = RealOps<dw>::zero();
                    for (int w = 0; w < T / 32; ++w) tot = tot + red[w];
                    acc[cc] = acc[cc] + tot;
                }
            }
        }
    }
}

// out[fibre f0 + fl][j] = sum_{c < S} part[fl S + c][j], in that order.
__global__ void dw_big_reduce(BigAxisDev B, double* out, long long f0, long long nf, long long inner, int S) {
    const int n = B.n;
    const long long total = nf * n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long fl = i / n;
        const int j = (int)(i - fl * n);
        dw s = B.part[(size_t)(fl * S) * n + j];
        for (int c = 1; c < S; ++c) s = s + B.part[(size_t)(fl * S + c) * n + j];
        out[big_fibre_offset(f0 + fl, n, inner) + (long long)j * inner] = RealOps<dw>::to_io(s);
    }
}

}  // namespace

}  // namespace dev

size_t dw_big_smem_bytes() { return dev::BIG_SMEM; }

cudaError_t dw_big_init() {
    static cudaError_t err = [] {
        cudaError_t e = cudaFuncSetAttribute(dev::dw_big_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)dev::BIG_SMEM);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(dev::dw_big_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)dev::BIG_SMEM);
        return e;
    }();
    return err;
}

cudaError_t launch_axis_dw_big(const dev::BigAxisDev& B, bool fwd, const double* in, double* out, long long nfib,
                               long long inner, cudaStream_t s) {
    cudaError_t e = dw_big_init();
    if (e != cudaSuccess) return e;
    if (nfib < 1) return cudaSuccess;
    const long long maxc = B.max_ctas;
    const int units = 2 * B.rank;
    int S = (int)std::max<long long>(1, std::min<long long>(units, maxc / nfib));
    if (S < 1) S = 1;
    const long long chunk = std::max<long long>(1, maxc / S);
    for (long long f0 = 0; f0 < nfib; f0 += chunk) {
        const long long nf = std::min(chunk, nfib - f0);
        const unsigned grid = (unsigned)(nf * S);
        if (fwd)
            dev::dw_big_kernel<true><<<grid, dev::BIG_THREADS, dev::BIG_SMEM, s>>>(B, in, f0, nf, inner, S);
        else
            dev::dw_big_kernel<false><<<grid, dev::BIG_THREADS, dev::BIG_SMEM, s>>>(B, in, f0, nf, inner, S);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        const long long tot = nf * B.n;
        const unsigned rg = (unsigned)std::min<long long>((tot + 255) / 256, 4096);
        dev::dw_big_reduce<<<rg, 256, 0, s>>>(B, out, f0, nf, inner, S);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace jt
