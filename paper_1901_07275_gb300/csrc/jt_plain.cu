// Plain FP64 comparison path (JT_FP64_PLAIN).
//
// Each axis splits into the dense low-degree block V (degrees < nu0) and the high-degree
// block G = Re(sum_k D_{u_k} F D_{v_k}) (Sec. 3.1, Eqs. tf:jn and eq:oneJ).  The
// d-dimensional operator (x)_a (V_a + G_a) expands into 2^d blocks.  The all-G block is
// evaluated in the r^d form of the abstract: with H_{a,k} = D_{u_{a,k}} F_a D_{v_{a,k}},
//   Re(H_0) (x) Re(H_1) (x) Re(H_2) = 2^{1-d} Re sum_{s} H_0 (x) H_1^{s_1} (x) H_2^{s_2},
// s_a in {plain, conjugate}, so it costs 2^{d-1} r_0 r_1 r_2 full d-dimensional FFTs (a
// conjugated axis uses conj(u), conj(v) and the e^{-} transform).  Every block that
// contains a V factor is applied axis by axis: dense V along its axes, and the same r-term
// FFT form, one axis at a time, along the others.  Nothing is fused: each step is a
// separate elementwise kernel or a cuFFT Z2Z call, all in FP64.
#include <cuda_runtime.h>
#include <cufft.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "jt_plain.hpp"

// Fixed work area of the allocation-free entry point (jt_forward_plain_noalloc).  It is part
// of the library image.  Modules load lazily, so a device commits these bytes when the
// module is first used on it: plain_create looks the array up, so this happens when the first
// JT_FP64_PLAIN plan is created on a device, and the device keeps them until the process
// exits.  All calls of that entry point share the array.
static __device__ __align__(256) unsigned char jt_static_scratch[JT_STATIC_SCRATCH_BYTES];

namespace jt {

namespace {

struct Dims {
    int d;
    long long n[3];
    long long L[3];
    int nu0[3];
};

struct PAxis {
    int n = 0, L = 0, nu0 = 0, rank = 0;
    double2* U = nullptr;  // rank x n
    double2* V = nullptr;  // rank x (n - nu0)
    int* m = nullptr;      // n
    double* Vblk = nullptr;  // n x nu0
    int* bin_ptr = nullptr;  // L/2 + 2
    int* bin_idx = nullptr;  // n
};

// one batched 1-D FFT along one axis of a row-major box
struct AxisFFT {
    cufftHandle plan = 0;
    bool have = false;
    long long outer = 1, step = 0;  // calls and the element offset between them
};

__device__ __forceinline__ double2 cmulD(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 conjD(double2 a) { return make_double2(a.x, -a.y); }

struct Fac {  // per-axis factor for one rank term, optionally conjugated
    const double2* p[3];
    int conj[3];
};

__device__ __forceinline__ double2 fac(const Fac& F, int a, long long i) {
    double2 v = F.p[a][i];
    return F.conj[a] ? conjD(v) : v;
}

// The all-G kernels work on nb right-hand sides at once: right-hand side q of the n-box at
// q * ntot, of the L-box at q * ltot.  The d-dimensional transform is the all-plus one; an axis
// whose pattern takes the e^{-} transform reads it at the reversed index (L - b) mod L, since
// e^{-2 pi i b nu / L} = e^{+2 pi i (L - b) nu / L}.
__device__ __forceinline__ long long rev_if(long long b, long long L, int c) { return c ? (L - b) % L : b; }

// X (L-box) = alpha restricted to high degrees, scaled by prod_a v_a[nu_a - nu0_a]
__global__ void k_bins_fwd(double2* X, const double* alpha, Dims D, Fac F, long long nb) {
    const long long ntot = D.n[0] * D.n[1] * D.n[2], ltot = D.L[0] * D.L[1] * D.L[2];
    const long long total = nb * ntot;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const long long q = i / ntot, rest = i - q * ntot;
        long long nu2 = rest % D.n[2], r = rest / D.n[2];
        long long nu1 = r % D.n[1], nu0 = r / D.n[1];
        long long nu[3] = {nu0, nu1, nu2};
        bool ok = true;
        for (int a = 0; a < D.d; ++a) ok = ok && nu[a] >= D.nu0[a];
        if (!ok) continue;
        double2 s = make_double2(alpha[i], 0.0);
        for (int a = 0; a < D.d; ++a) s = cmulD(s, fac(F, a, nu[a] - D.nu0[a]));
        X[q * ltot + (nu0 * D.L[1] + nu1) * D.L[2] + nu2] = s;
    }
}

// acc (n-box) += w Re(prod_a u_a[i_a] X[m_0(i_0), m_1(i_1), m_2(i_2)])
__global__ void k_gather_fwd(double* acc, const double2* X, Dims D, Fac F, const int* m0, const int* m1,
                             const int* m2, double w, long long nb) {
    const long long ntot = D.n[0] * D.n[1] * D.n[2], ltot = D.L[0] * D.L[1] * D.L[2];
    const long long total = nb * ntot;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const long long q = i / ntot, rest = i - q * ntot;
        long long i2 = rest % D.n[2], r = rest / D.n[2];
        long long i1 = r % D.n[1], i0 = r / D.n[1];
        long long b0 = rev_if(m0[i0], D.L[0], F.conj[0]);
        long long b1 = (D.d > 1) ? rev_if(m1[i1], D.L[1], F.conj[1]) : 0;
        long long b2 = (D.d > 2) ? rev_if(m2[i2], D.L[2], F.conj[2]) : 0;
        double2 s = X[q * ltot + (b0 * D.L[1] + b1) * D.L[2] + b2];
        long long ii[3] = {i0, i1, i2};
        for (int a = 0; a < D.d; ++a) s = cmulD(s, fac(F, a, ii[a]));
        acc[i] += w * s.x;
    }
}

// X (L-box) at reachable bins = sum over the points of the bin of g * prod_a u_a (transpose of
// the gather); bins are separable, so each bin sums a Cartesian product of per-axis lists.
__global__ void k_scatter_adj(double2* X, const double* g, Dims D, Fac F, const int* bp0, const int* bi0,
                              const int* bp1, const int* bi1, const int* bp2, const int* bi2, long long nb) {
    const long long ntot = D.n[0] * D.n[1] * D.n[2], ltot = D.L[0] * D.L[1] * D.L[2];
    long long H0 = D.L[0] / 2 + 1, H1 = (D.d > 1) ? D.L[1] / 2 + 1 : 1, H2 = (D.d > 2) ? D.L[2] / 2 + 1 : 1;
    const long long hb = H0 * H1 * H2, total = nb * hb;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const long long q = i / hb, rest = i - q * hb;
        const double* gq = g + q * ntot;
        long long b2 = rest % H2, r = rest / H2;
        long long b1 = r % H1, b0 = r / H1;
        double2 s = make_double2(0.0, 0.0);
        int p0a = bp0[b0], p0b = bp0[b0 + 1];
        int p1a = (D.d > 1) ? bp1[b1] : 0, p1b = (D.d > 1) ? bp1[b1 + 1] : 1;
        int p2a = (D.d > 2) ? bp2[b2] : 0, p2b = (D.d > 2) ? bp2[b2 + 1] : 1;
        for (int p0 = p0a; p0 < p0b; ++p0) {
            long long j0 = bi0[p0];
            double2 f0 = fac(F, 0, j0);
            for (int p1 = p1a; p1 < p1b; ++p1) {
                long long j1 = (D.d > 1) ? bi1[p1] : 0;
                double2 f01 = (D.d > 1) ? cmulD(f0, fac(F, 1, j1)) : f0;
                for (int p2 = p2a; p2 < p2b; ++p2) {
                    long long j2 = (D.d > 2) ? bi2[p2] : 0;
                    double2 f = (D.d > 2) ? cmulD(f01, fac(F, 2, j2)) : f01;
                    double gv = gq[(j0 * D.n[1] + j1) * D.n[2] + j2];
                    s.x += f.x * gv;
                    s.y += f.y * gv;
                }
            }
        }
        X[q * ltot + (b0 * D.L[1] + b1) * D.L[2] + b2] = s;
    }
}

// out (n-box, high degrees) += w Re(prod_a v_a[nu_a - nu0_a] X[nu])
__global__ void k_scale_adj(double* out, const double2* X, Dims D, Fac F, double w, long long nb) {
    const long long ntot = D.n[0] * D.n[1] * D.n[2], ltot = D.L[0] * D.L[1] * D.L[2];
    const long long total = nb * ntot;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const long long q = i / ntot, rest = i - q * ntot;
        long long nu2 = rest % D.n[2], r = rest / D.n[2];
        long long nu1 = r % D.n[1], nu0 = r / D.n[1];
        long long nu[3] = {nu0, nu1, nu2};
        bool ok = true;
        for (int a = 0; a < D.d; ++a) ok = ok && nu[a] >= D.nu0[a];
        if (!ok) continue;
        const long long r0 = rev_if(nu0, D.L[0], F.conj[0]);
        const long long r1 = (D.d > 1) ? rev_if(nu1, D.L[1], F.conj[1]) : 0;
        const long long r2 = (D.d > 2) ? rev_if(nu2, D.L[2], F.conj[2]) : 0;
        double2 s = X[q * ltot + (r0 * D.L[1] + r1) * D.L[2] + r2];
        for (int a = 0; a < D.d; ++a) s = cmulD(s, fac(F, a, nu[a] - D.nu0[a]));
        out[i] += w * s.x;
    }
}

// ---------- one-axis operators on an n-box (outer x n_a x inner), the cross blocks ----------
// dense block along the axis: fwd out[j] = sum_{c<nu0} Vblk[j][c] in[c];
//                             adj out[c] = sum_j Vblk[j][c] in[j] (c < nu0), 0 above
__global__ void k_vop(double* out, const double* in, long long outer, int n, long long inner, const double* Vblk,
                      int nu0, int adj) {
    long long total = outer * n * inner;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        long long q = i % inner, r = i / inner;
        long long j = r % n, o = r / n;
        const double* src = in + o * n * inner + q;
        double s = 0;
        if (!adj) {
            for (int c = 0; c < nu0; ++c) s += Vblk[j * nu0 + c] * src[c * inner];
        } else if (j < nu0) {
            for (long long jj = 0; jj < n; ++jj) s += Vblk[jj * nu0 + j] * src[jj * inner];
        }
        out[i] = s;
    }
}

// Z (outer x L x inner) = bins of the high degrees times v_k (fwd) / scatter of u_k g (adj)
__global__ void k_axis_bins(double2* Z, const double* in, long long outer, int n, int L, long long inner,
                            const double2* fk, int nu0, int adj, const int* bp, const int* bi) {
    long long total = outer * (long long)L * inner;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        long long q = i % inner, r = i / inner;
        long long b = r % L, o = r / L;
        const double* src = in + o * n * inner + q;
        double2 s = make_double2(0.0, 0.0);
        if (!adj) {
            if (b >= nu0 && b < n) {
                double2 v = fk[b - nu0];
                double x = src[b * inner];
                s = make_double2(v.x * x, v.y * x);
            }
        } else if (b <= L / 2) {
            for (int p = bp[b]; p < bp[b + 1]; ++p) {
                int j = bi[p];
                double2 u = fk[j];
                double x = src[(long long)j * inner];
                s.x += u.x * x;
                s.y += u.y * x;
            }
        }
        Z[i] = s;
    }
}

// fwd: out[j] += Re(u_k[j] Z[m_j]);  adj: out[nu] += Re(v_k[nu - nu0] Z[nu]) for nu >= nu0
__global__ void k_axis_acc(double* out, const double2* Z, long long outer, int n, int L, long long inner,
                           const double2* fk, int nu0, const int* m, int adj) {
    long long total = outer * n * inner;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        long long q = i % inner, r = i / inner;
        long long j = r % n, o = r / n;
        const double2* zf = Z + o * (long long)L * inner + q;
        if (!adj) {
            double2 z = zf[(long long)m[j] * inner];
            double2 u = fk[j];
            out[i] += u.x * z.x - u.y * z.y;
        } else if (j >= nu0) {
            double2 z = zf[j * inner];
            double2 v = fk[j - nu0];
            out[i] += v.x * z.x - v.y * z.y;
        }
    }
}

__global__ void k_add(double* out, const double* in, long long count) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x)
        out[i] += in[i];
}

inline unsigned grid_for(long long count) {
    long long g = (count + 255) / 256;
    return (unsigned)std::max<long long>(1, std::min<long long>(g, 152 * 16));
}

}  // namespace

// Work buffers of one apply of nb right-hand sides: X (nb L-boxes, complex), Z (per-axis
// complex work) and two real n-box temporaries, each nb boxes long.
struct PlainScratch {
    double2* X;
    double2* Z;
    double* T1;
    double* T2;
    int nb;  // right-hand sides the buffers hold
};

// cuFFT plans for chunks of nb right-hand sides: the d-dimensional all-plus transform of the
// L-box, and the 1-D transform along each axis of the (n with n_a -> L_a) box.
struct FFTSet {
    int nb = 0;
    AxisFFT fd;     // rank-d plan, batch nb: one call per rank-term tuple
    AxisFFT fz[3];  // along axis a; one call, or one per outer slab when the axis is strided
};

struct PlainPlan {
    int d = 1;
    Dims D{};
    PAxis ax[3];
    int nb_max = 1;         // right-hand sides per chunk of the plan's buffers (a power of two)
    double2* X = nullptr;   // nb_max L-boxes
    double2* Z = nullptr;   // nb_max x max_a (prod_{i != a} n_i) * L_a
    double* T1 = nullptr;   // nb_max n-boxes
    double* T2 = nullptr;
    // plan sets for chunks of 1, 2, 4, .., nb_max right-hand sides; a call of nrhs takes
    // chunks of the largest size that fits what is left.  All plans share one work area.
    static constexpr int NSETS = 11;
    FFTSet fft[NSETS];
    void* fft_work = nullptr;
    std::vector<void*> allocs;
    // device address of the static work area on the plan's device (looked up at creation)
    void* static_scratch = nullptr;
};

namespace {

template <class T>
jt_status dmalloc(PlainPlan* P, T** p, size_t count) {
    if (count == 0) count = 1;
    if (cudaMalloc((void**)p, sizeof(T) * count) != cudaSuccess) {
        cudaGetLastError();
        return JT_ENOMEM;
    }
    P->allocs.push_back(*p);
    return JT_OK;
}

// 1-D transforms along axis a of nb boxes of dims[0..d): one batched call when the axis is the
// last (contiguous), else a plan over the inner index, called once per outer slab.
// Plans are made without a work area of their own (the plan's shared one is set afterwards);
// *work receives the largest size any of them needs.
jt_status make_plan(AxisFFT& f, int rank, int* nn, int istride, int idist, int batch, size_t* work) {
    if (cufftCreate(&f.plan) != CUFFT_SUCCESS) return JT_ECUDA;
    f.have = true;
    size_t ws = 0;
    if (cufftSetAutoAllocation(f.plan, 0) != CUFFT_SUCCESS ||
        cufftMakePlanMany(f.plan, rank, nn, nn, istride, idist, nn, istride, idist, CUFFT_Z2Z, batch, &ws) !=
            CUFFT_SUCCESS)
        return JT_ECUDA;
    *work = std::max(*work, ws);
    return JT_OK;
}

jt_status make_axis_fft(AxisFFT& f, const long long* dims, int d, int a, int nb, size_t* work) {
    long long outer = nb, inner = 1;
    for (int i = 0; i < a; ++i) outer *= dims[i];
    for (int i = a + 1; i < d; ++i) inner *= dims[i];
    int len = (int)dims[a];
    int nn[1] = {len};
    if (inner == 1) {
        f.outer = 1;
        f.step = 0;
        return make_plan(f, 1, nn, 1, len, (int)outer, work);
    }
    f.outer = outer;
    f.step = (long long)len * inner;
    return make_plan(f, 1, nn, (int)inner, 1, (int)inner, work);
}

// The d-dimensional transform of nb contiguous L-boxes in one call.
jt_status make_box_fft(AxisFFT& f, const long long* L, int d, int nb, size_t* work) {
    int nn[3];
    long long tot = 1;
    for (int a = 0; a < d; ++a) {
        nn[a] = (int)L[a];
        tot *= L[a];
    }
    f.outer = 1;
    f.step = 0;
    return make_plan(f, d, nn, 1, (int)tot, nb, work);
}

jt_status make_fft_set(PlainPlan* P, FFTSet& F, int nb, size_t* work) {
    F.nb = nb;
    jt_status st = make_box_fft(F.fd, P->D.L, P->d, nb, work);
    for (int a = 0; a < P->d && st == JT_OK; ++a) {
        long long zd[3] = {P->D.n[0], P->D.n[1], P->D.n[2]};
        zd[a] = P->D.L[a];
        st = make_axis_fft(F.fz[a], zd, P->d, a, nb, work);
    }
    return st;
}

jt_status set_work(FFTSet& F, void* work) {
    if (F.fd.have && cufftSetWorkArea(F.fd.plan, work) != CUFFT_SUCCESS) return JT_ECUDA;
    for (int a = 0; a < 3; ++a)
        if (F.fz[a].have && cufftSetWorkArea(F.fz[a].plan, work) != CUFFT_SUCCESS) return JT_ECUDA;
    return JT_OK;
}

void destroy_fft_set(FFTSet& F) {
    if (F.fd.have) cufftDestroy(F.fd.plan);
    for (int a = 0; a < 3; ++a)
        if (F.fz[a].have) cufftDestroy(F.fz[a].plan);
    F = FFTSet();
}

jt_status run_fft(AxisFFT& f, double2* buf, int sign, cudaStream_t s) {
    if (cufftSetStream(f.plan, s) != CUFFT_SUCCESS) return JT_ECUDA;
    for (long long o = 0; o < f.outer; ++o) {
        cufftDoubleComplex* p = (cufftDoubleComplex*)(buf + o * f.step);
        // CUFFT_INVERSE is the e^{+} transform
        if (cufftExecZ2Z(f.plan, p, p, sign > 0 ? CUFFT_INVERSE : CUFFT_FORWARD) != CUFFT_SUCCESS) return JT_ECUDA;
    }
    return JT_OK;
}

// one axis operator (V or G block, forward or adjoint) from src to dst on nb n-boxes
jt_status axis_op(PlainPlan* P, const PlainScratch& W, FFTSet& F, int a, bool vblock, bool adj, const double* src,
                  double* dst, cudaStream_t s) {
    const PAxis& A = P->ax[a];
    long long outer = F.nb, inner = 1;
    for (int i = 0; i < a; ++i) outer *= P->D.n[i];
    for (int i = a + 1; i < P->d; ++i) inner *= P->D.n[i];
    long long total = outer * A.n * inner;
    if (vblock) {
        k_vop<<<grid_for(total), 256, 0, s>>>(dst, src, outer, A.n, inner, A.Vblk, A.nu0, adj ? 1 : 0);
        return cudaGetLastError() == cudaSuccess ? JT_OK : JT_ECUDA;
    }
    if (cudaMemsetAsync(dst, 0, sizeof(double) * total, s) != cudaSuccess) return JT_ECUDA;
    const long long ztot = outer * (long long)A.L * inner;
    const int N = A.n - A.nu0;
    for (int k = 0; k < A.rank; ++k) {
        const double2* uk = A.U + (size_t)k * A.n;
        const double2* vk = A.V + (size_t)k * N;
        k_axis_bins<<<grid_for(ztot), 256, 0, s>>>(W.Z, src, outer, A.n, A.L, inner, adj ? uk : vk, A.nu0,
                                                    adj ? 1 : 0, A.bin_ptr, A.bin_idx);
        if (cudaGetLastError() != cudaSuccess) return JT_ECUDA;
        jt_status st = run_fft(F.fz[a], W.Z, +1, s);
        if (st != JT_OK) return st;
        k_axis_acc<<<grid_for(total), 256, 0, s>>>(dst, W.Z, outer, A.n, A.L, inner, adj ? vk : uk, A.nu0, A.m,
                                                   adj ? 1 : 0);
        if (cudaGetLastError() != cudaSuccess) return JT_ECUDA;
    }
    return JT_OK;
}

// all-G block by the r^d d-dimensional FFT form, accumulated into acc (nb right-hand sides):
// one d-dimensional cuFFT call per (pattern, rank-term tuple)
jt_status rd_block(PlainPlan* P, const PlainScratch& W, FFTSet& F, const double* src, double* acc, bool adj,
                   cudaStream_t s) {
    const int d = P->d;
    const Dims& D = P->D;
    const long long nb = F.nb;
    const long long ltot = D.L[0] * D.L[1] * D.L[2];
    const long long ntot = D.n[0] * D.n[1] * D.n[2];
    const double w = 1.0 / (double)(1 << (d - 1));
    int r[3] = {1, 1, 1};
    for (int a = 0; a < d; ++a) r[a] = P->ax[a].rank;
    if (r[0] == 0 || (d > 1 && r[1] == 0) || (d > 2 && r[2] == 0)) return JT_OK;
    const int npat = 1 << (d - 1);
    for (int pat = 0; pat < npat; ++pat) {
        int conj[3] = {0, (pat & 1), (pat >> 1) & 1};
        for (int k0 = 0; k0 < r[0]; ++k0)
            for (int k1 = 0; k1 < r[1]; ++k1)
                for (int k2 = 0; k2 < r[2]; ++k2) {
                    int ks[3] = {k0, k1, k2};
                    Fac Fv{}, Fu{};
                    for (int a = 0; a < 3; ++a) {
                        const PAxis& A = P->ax[a < d ? a : 0];
                        Fv.p[a] = A.V + (size_t)ks[a] * (A.n - A.nu0);
                        Fu.p[a] = A.U + (size_t)ks[a] * A.n;
                        Fv.conj[a] = Fu.conj[a] = (a < d) ? conj[a] : 0;
                    }
                    if (cudaMemsetAsync(W.X, 0, sizeof(double2) * ltot * nb, s) != cudaSuccess) return JT_ECUDA;
                    if (!adj) {
                        k_bins_fwd<<<grid_for(ntot * nb), 256, 0, s>>>(W.X, src, D, Fv, nb);
                    } else {
                        const PAxis& A0 = P->ax[0];
                        const PAxis& A1 = P->ax[d > 1 ? 1 : 0];
                        const PAxis& A2 = P->ax[d > 2 ? 2 : 0];
                        long long h = (D.L[0] / 2 + 1) * (d > 1 ? D.L[1] / 2 + 1 : 1) * (d > 2 ? D.L[2] / 2 + 1 : 1);
                        k_scatter_adj<<<grid_for(h * nb), 256, 0, s>>>(W.X, src, D, Fu, A0.bin_ptr, A0.bin_idx,
                                                                        A1.bin_ptr, A1.bin_idx, A2.bin_ptr, A2.bin_idx,
                                                                        nb);
                    }
                    if (cudaGetLastError() != cudaSuccess) return JT_ECUDA;
                    jt_status st = run_fft(F.fd, W.X, +1, s);
                    if (st != JT_OK) return st;
                    if (!adj)
                        k_gather_fwd<<<grid_for(ntot * nb), 256, 0, s>>>(acc, W.X, D, Fu, P->ax[0].m,
                                                                          P->ax[d > 1 ? 1 : 0].m,
                                                                          P->ax[d > 2 ? 2 : 0].m, w, nb);
                    else
                        k_scale_adj<<<grid_for(ntot * nb), 256, 0, s>>>(acc, W.X, D, Fv, w, nb);
                    if (cudaGetLastError() != cudaSuccess) return JT_ECUDA;
                }
    }
    return JT_OK;
}

}  // namespace

jt_status plain_create(PlainPlan** out, const std::vector<const AxisTables*>& axes, cudaStream_t s) {
    *out = nullptr;
    PlainPlan* P = new (std::nothrow) PlainPlan();
    if (!P) return JT_ENOMEM;
    P->d = (int)axes.size();
    P->D.d = P->d;
    for (int a = 0; a < 3; ++a) {
        P->D.n[a] = 1;
        P->D.L[a] = 1;
        P->D.nu0[a] = 0;
    }
    jt_status st = JT_OK;
    for (int a = 0; a < P->d && st == JT_OK; ++a) {
        const AxisTables& T = *axes[a];
        PAxis& A = P->ax[a];
        A.n = (int)T.n;
        A.L = (int)T.L;
        A.nu0 = T.nu0;
        A.rank = T.rank;
        P->D.n[a] = T.n;
        P->D.L[a] = T.L;
        P->D.nu0[a] = T.nu0;
        std::vector<double2> U(T.U.size()), V(T.V.size());
        for (size_t i = 0; i < U.size(); ++i) U[i] = make_double2(T.U[i].real(), T.U[i].imag());
        for (size_t i = 0; i < V.size(); ++i) V[i] = make_double2(T.V[i].real(), T.V[i].imag());
        std::vector<int> bp(T.L / 2 + 2, 0), bi(T.n);
        for (int64_t j = 0; j < T.n; ++j) bp[T.m[j] + 1]++;
        for (int64_t m = 0; m <= T.L / 2; ++m) bp[m + 1] += bp[m];
        std::vector<int> fill(bp.begin(), bp.end() - 1);
        for (int64_t j = 0; j < T.n; ++j) bi[fill[T.m[j]]++] = (int)j;
        if ((st = dmalloc(P, &A.U, U.size())) != JT_OK) break;
        if ((st = dmalloc(P, &A.V, V.size())) != JT_OK) break;
        if ((st = dmalloc(P, &A.m, (size_t)T.n)) != JT_OK) break;
        if ((st = dmalloc(P, &A.Vblk, T.Vblk.size())) != JT_OK) break;
        if ((st = dmalloc(P, &A.bin_ptr, bp.size())) != JT_OK) break;
        if ((st = dmalloc(P, &A.bin_idx, bi.size())) != JT_OK) break;
        bool ok = cudaMemcpy(A.U, U.data(), sizeof(double2) * U.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
                  cudaMemcpy(A.V, V.data(), sizeof(double2) * V.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
                  cudaMemcpy(A.m, T.m.data(), sizeof(int) * T.n, cudaMemcpyHostToDevice) == cudaSuccess &&
                  cudaMemcpy(A.Vblk, T.Vblk.data(), sizeof(double) * T.Vblk.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
                  cudaMemcpy(A.bin_ptr, bp.data(), sizeof(int) * bp.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
                  cudaMemcpy(A.bin_idx, bi.data(), sizeof(int) * bi.size(), cudaMemcpyHostToDevice) == cudaSuccess;
        if (!ok) st = JT_ECUDA;
    }
    if (st == JT_OK) {
        long long ltot = P->D.L[0] * P->D.L[1] * P->D.L[2];
        long long ntot = P->D.n[0] * P->D.n[1] * P->D.n[2];
        long long zmax = 0;
        for (int a = 0; a < P->d; ++a) zmax = std::max(zmax, ntot / P->D.n[a] * P->D.L[a]);
        // right-hand sides per chunk: the buffers of a chunk take at most 256 MiB (at least one
        // right-hand side), and at most 1024 right-hand sides
        const long long per_rhs = 16 * ltot + 16 * zmax + 16 * ntot;
        const long long fit = std::max<long long>(1, std::min<long long>(1024, (256ll << 20) / per_rhs));
        P->nb_max = 1;
        while (2 * (long long)P->nb_max <= fit) P->nb_max *= 2;
        const size_t nbm = (size_t)P->nb_max;
        if (st == JT_OK) st = dmalloc(P, &P->X, (size_t)ltot * nbm);
        if (st == JT_OK) st = dmalloc(P, &P->Z, (size_t)zmax * nbm);
        if (st == JT_OK) st = dmalloc(P, &P->T1, (size_t)ntot * nbm);
        if (st == JT_OK) st = dmalloc(P, &P->T2, (size_t)ntot * nbm);
        size_t work = 0;
        for (int i = 0; st == JT_OK && (1 << i) <= P->nb_max; ++i) st = make_fft_set(P, P->fft[i], 1 << i, &work);
        if (st == JT_OK && work > 0) st = dmalloc(P, reinterpret_cast<unsigned char**>(&P->fft_work), work);
        for (int i = 0; st == JT_OK && (1 << i) <= P->nb_max; ++i) st = set_work(P->fft[i], P->fft_work);
    }
    if (st == JT_OK) {
        // The host-side name of the array is not a device address: look the address up on
        // this device (current during plan creation).  This also loads the module, so the
        // array is committed now rather than inside a later allocation-free call.
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, jt_static_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            st = JT_ECUDA;
        }
        P->static_scratch = p;
    }
    if (st != JT_OK) {
        plain_destroy(P);
        return st;
    }
    (void)s;
    *out = P;
    return JT_OK;
}

namespace {

// The whole plain apply with caller-chosen work buffers holding W.nb right-hand sides (a power
// of two): each chunk is the largest power of two that fits both W.nb and what is left.
jt_status plain_apply_bufs(PlainPlan* P, const PlainScratch& W, const double* in, double* out, int64_t nrhs,
                           bool fwd, cudaStream_t s) {
    const int d = P->d;
    const long long ntot = P->D.n[0] * P->D.n[1] * P->D.n[2];
    const bool adj = !fwd;
    for (int64_t r0 = 0; r0 < nrhs;) {
        int i = 0;
        while ((2ll << i) <= W.nb && (2ll << i) <= nrhs - r0) ++i;
        FFTSet& F = P->fft[i];
        const long long nb = F.nb;
        const double* src = in + r0 * ntot;
        double* dst = out + r0 * ntot;
        // in-place safety: the all-G block reads src while accumulating into T2, copied at the end
        if (cudaMemsetAsync(W.T2, 0, sizeof(double) * ntot * nb, s) != cudaSuccess) return JT_ECUDA;
        jt_status st = rd_block(P, W, F, src, W.T2, adj, s);
        if (st != JT_OK) return st;
        // blocks with at least one dense factor, axis by axis
        for (int mask = 1; mask < (1 << d); ++mask) {
            // chain through T1 and X (free after the all-G block, used as a real buffer) so
            // that src stays intact for the next block
            const double* cur = src;
            double* tmp[2] = {W.T1, reinterpret_cast<double*>(W.X)};
            int which = 0;
            for (int a = d - 1; a >= 0; --a) {
                bool vb = (mask >> a) & 1;
                double* nxt = tmp[which];
                st = axis_op(P, W, F, a, vb, adj, cur, nxt, s);
                if (st != JT_OK) return st;
                cur = nxt;
                which ^= 1;
            }
            k_add<<<grid_for(ntot * nb), 256, 0, s>>>(W.T2, cur, ntot * nb);
            if (cudaGetLastError() != cudaSuccess) return JT_ECUDA;
        }
        if (cudaMemcpyAsync(dst, W.T2, sizeof(double) * ntot * nb, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return JT_ECUDA;
        r0 += nb;
    }
    return JT_OK;
}

}  // namespace

jt_status plain_apply(PlainPlan* P, const double* in, double* out, int64_t nrhs, bool fwd, cudaStream_t s) {
    if (!P) return JT_EINVAL;
    const PlainScratch W{P->X, P->Z, P->T1, P->T2, P->nb_max};
    return plain_apply_bufs(P, W, in, out, nrhs, fwd, s);
}

namespace {

size_t round256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

size_t plain_static_bytes(const PlainPlan* P) {
    const long long ltot = P->D.L[0] * P->D.L[1] * P->D.L[2];
    const long long ntot = P->D.n[0] * P->D.n[1] * P->D.n[2];
    long long zmax = 0;
    for (int a = 0; a < P->d; ++a) zmax = std::max(zmax, ntot / P->D.n[a] * P->D.L[a]);
    return round256(sizeof(double2) * ltot) + round256(sizeof(double2) * zmax) + 2 * round256(sizeof(double) * ntot);
}

jt_status plain_apply_static(PlainPlan* P, const double* in, double* out, int64_t nrhs, bool fwd, cudaStream_t s) {
    if (!P) return JT_EINVAL;
    if (plain_static_bytes(P) > (size_t)JT_STATIC_SCRATCH_BYTES) return JT_EINVAL;
    void* base = P->static_scratch;
    if (!base) return JT_ECUDA;
    const long long ltot = P->D.L[0] * P->D.L[1] * P->D.L[2];
    const long long ntot = P->D.n[0] * P->D.n[1] * P->D.n[2];
    long long zmax = 0;
    for (int a = 0; a < P->d; ++a) zmax = std::max(zmax, ntot / P->D.n[a] * P->D.L[a]);
    unsigned char* q = static_cast<unsigned char*>(base);
    PlainScratch W;
    W.nb = 1;
    W.X = reinterpret_cast<double2*>(q);
    q += round256(sizeof(double2) * ltot);
    W.Z = reinterpret_cast<double2*>(q);
    q += round256(sizeof(double2) * zmax);
    W.T1 = reinterpret_cast<double*>(q);
    q += round256(sizeof(double) * ntot);
    W.T2 = reinterpret_cast<double*>(q);
    // one right-hand side at a time through the single-right-hand-side plans; every buffer that
    // must start at zero is cleared inside the apply (cudaMemsetAsync on the stream), so what
    // an earlier call left in the area does not matter
    return plain_apply_bufs(P, W, in, out, nrhs, fwd, s);
}

void plain_destroy(PlainPlan* P) {
    if (!P) return;
    for (int i = 0; i < PlainPlan::NSETS; ++i) destroy_fft_set(P->fft[i]);
    for (void* p : P->allocs) cudaFree(p);
    delete P;
}

}  // namespace jt
