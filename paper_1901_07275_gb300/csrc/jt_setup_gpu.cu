// The O(n^2) steps of the plan setup on the GPU in FP64 (jt_options.setup_device = 1): the
// Newton iteration for the Gauss--Jacobi nodes with their Christoffel numbers, and the
// sampled columns of B that Algorithm 2.1 needs (Sec. 2.1; Sec. 3.1, Eq. eq:B).  Both are the
// host algorithms of jt_setup.cpp run with one thread per point: the three-term recurrence
// of the orthonormal polynomials p_nu (and of the second-kind h_nu) walked in FP64, and in
// double-word FP64 (pairs of doubles, Dekker 1971; Joldes, Muller, Popescu 2017) for points
// with min(t, pi - t) < 0.35, where FP64 alone loses accuracy.  The column-pivoted QRs of
// Algorithm 2.1 (steps 2-3, the pivots only) run here too, with the host routine's arithmetic
// (jt_linalg.hpp qrcp_pivots); the orthonormal bases, the least-squares middle matrix and its
// SVD (all of rank r or of r columns) stay on the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "jt_internal.hpp"

namespace jt {
namespace {

constexpr double PI_D = 3.14159265358979323846264338327950288;
constexpr double NEAR_END_D = 0.35;

// ------------------------------------------------------------ double-word FP64
struct dd2 {
    double hi, lo;
};
__device__ __forceinline__ dd2 two_sum(double a, double b) {
    double s = a + b;
    double bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ dd2 fast_two_sum(double a, double b) {
    double s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ dd2 two_prod(double a, double b) {
    double p = a * b;
    return {p, __fma_rn(a, b, -p)};
}
__device__ __forceinline__ dd2 operator+(dd2 a, dd2 b) {
    dd2 s = two_sum(a.hi, b.hi);
    dd2 t = two_sum(a.lo, b.lo);
    dd2 v = fast_two_sum(s.hi, s.lo + t.hi);
    return fast_two_sum(v.hi, t.lo + v.lo);
}
__device__ __forceinline__ dd2 operator-(dd2 a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dd2 operator-(dd2 a, dd2 b) { return a + (-b); }
__device__ __forceinline__ dd2 operator*(dd2 a, dd2 b) {
    dd2 p = two_prod(a.hi, b.hi);
    double t = __fma_rn(a.hi, b.lo, a.lo * b.hi);
    return fast_two_sum(p.hi, p.lo + t);
}
__device__ __forceinline__ dd2 operator*(dd2 a, double b) {
    dd2 p = two_prod(a.hi, b);
    return fast_two_sum(p.hi, __fma_rn(a.lo, b, p.lo));
}
__device__ __forceinline__ dd2 mk(double v) { return {v, 0.0}; }
__device__ __forceinline__ double val(dd2 v) { return v.hi + v.lo; }

__device__ __forceinline__ bool near_end(double t) { return fmin(t, PI_D - t) < NEAR_END_D; }

// x = cos t as a double-word number from the exact complements 1 - x = 2 sin^2(t/2) and
// 1 + x = 2 cos^2(t/2)
__device__ __forceinline__ dd2 x_dd(double t) {
    if (t <= 0.5 * PI_D) {
        double s = sin(0.5 * t);
        return mk(1.0) - two_prod(s, s) * 2.0;
    }
    double c = cos(0.5 * t);
    return two_prod(c, c) * 2.0 - mk(1.0);
}

// Recurrence tables: beta[j], sg[j], isg[j] = 1/sg[j] (index 0 .. n+1), FP64 and double-word.
struct Rec {
    const double *beta, *sg, *isg;
    const dd2 *betaD, *sgD, *isgD;
    double p0, sqrt_mu0;
};

// p_n(x), p_n'(x) (FP64) and sum_{j<n} p_j(x)^2 in FP64
__device__ void pn_fp64(const Rec& C, int n, double x, double& p, double& dp, double& ssq) {
    double pm = 0.0, pc = C.p0, dm = 0.0, dc = 0.0, s = 0.0;
    for (int j = 0; j < n; ++j) {
        const double bj = __ldg(C.beta + j), sj = __ldg(C.sg + j), ij = __ldg(C.isg + j + 1);
        s = __fma_rn(pc, pc, s);
        const double xb = x - bj;
        const double pn = (xb * pc - sj * pm) * ij;
        const double dn = (xb * dc + pc - sj * dm) * ij;
        pm = pc;
        pc = pn;
        dm = dc;
        dc = dn;
    }
    p = pc;
    dp = dc;
    ssq = s;
}

// the same with p and the sum of squares in double-word (p' stays FP64: it only scales a step)
__device__ void pn_dd(const Rec& C, int n, dd2 x, dd2& p, double& dp, dd2& ssq) {
    dd2 pm = mk(0.0), pc = mk(C.p0), s = mk(0.0);
    double dm = 0.0, dc = 0.0;
    const double xd = val(x);
    for (int j = 0; j < n; ++j) {
        const dd2 bj = C.betaD[j], sj = C.sgD[j], ij = C.isgD[j + 1];
        s = s + pc * pc;
        const dd2 xb = x - bj;
        const dd2 pn = (xb * pc - sj * pm) * ij;
        const double dn = ((xd - val(bj)) * dc + val(pc) - val(sj) * dm) * val(ij);
        pm = pc;
        pc = pn;
        dm = dc;
        dc = dn;
    }
    p = pc;
    dp = dc;
    ssq = s;
}

// One thread per node: FP64 Newton in t from the host's initial angle (at most 40 steps,
// each clamped to maxstep), then, for points near the ends, two double-word steps (the
// second gives the Christoffel number omega = 1 / sum p_j^2).
__global__ void newton_nodes_kernel(Rec C, int n, double maxstep, double* t, double* omega) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    double tk = t[k];
    const bool dw = near_end(tk);
    const double tol = dw ? 1e-13 : 2e-16;
    double p, dp, s;
    for (int it = 0; it < 40; ++it) {
        pn_fp64(C, n, cos(tk), p, dp, s);
        double dt = p / (sin(tk) * dp);
        if (!isfinite(dt)) dt = 0.0;
        dt = fmax(-maxstep, fmin(maxstep, dt));
        tk += dt;
        if (fabs(dt) <= tol * fmin(tk, PI_D - tk)) break;
    }
    if (!dw) {
        pn_fp64(C, n, cos(tk), p, dp, s);
        t[k] = tk;
        omega[k] = 1.0 / s;
        return;
    }
    dd2 pd, sd;
    for (int step = 0; step < 2; ++step) {
        pn_dd(C, n, x_dd(tk), pd, dp, sd);
        const double dt = val(pd) / (sin(tk) * dp);
        if (step == 0 && isfinite(dt) && fabs(dt) < maxstep) tk += dt;
        if (step == 1) omega[k] = 1.0 / val(sd);
    }
    t[k] = tk;
}

// Columns of Z = W B: thread j walks nu = 0 .. last with p_nu and h_nu and stores the entries
// of the sampled columns, out[j + q n] = (rowP_j p_nu + i rowQ_j h_nu) e^{-2 pi i m_j nu / L}
// for nu = nu0 + cl[q].  A warp with a point near the ends walks in double-word.
struct ColArgs {
    const double *t, *rowP, *rowQ, *S;
    const int* m;
    const double2* phase;  // e^{-2 pi i r / L}, r < L
    const int* slot;       // nu - nu0 -> column index or -1
    int n, nu0, last;
    long long L;
    double2* out;
};

template <bool DW>
__device__ void walk_columns(const Rec& C, const ColArgs& A, int j) {
    using R = typename std::conditional<DW, dd2, double>::type;
    R x, pm, pc, hm, hc;
    if constexpr (DW) {
        x = x_dd(A.t[j]);
        pm = mk(0.0);
        pc = mk(C.p0);
        hm = mk(0.0);
        hc = mk(C.p0) * A.S[j];
    } else {
        x = cos(A.t[j]);
        pm = 0.0;
        pc = C.p0;
        hm = 0.0;
        hc = C.p0 * A.S[j];
    }
    const double rp = A.rowP[j], rq = A.rowQ[j];
    const long long mj = A.m[j];
    for (int nu = 0; nu <= A.last; ++nu) {
        if (nu >= A.nu0) {
            const int q = __ldg(A.slot + (nu - A.nu0));
            if (q >= 0) {
                double pv, hv;
                if constexpr (DW) {
                    pv = val(pc);
                    hv = val(hc);
                } else {
                    pv = pc;
                    hv = hc;
                }
                const double2 ph = A.phase[(mj * nu) & (A.L - 1)];
                const double re = rp * pv, im = rq * hv;
                A.out[(size_t)j + (size_t)q * A.n] = make_double2(re * ph.x - im * ph.y, re * ph.y + im * ph.x);
            }
        }
        if (nu == A.last) break;
        R pn, hn;
        if constexpr (DW) {
            const dd2 xb = x - C.betaD[nu];
            const dd2 i1 = C.isgD[nu + 1];
            if (nu == 0) {
                pn = xb * pc * i1;
                hn = (xb * hc - mk(C.sqrt_mu0)) * i1;
            } else {
                pn = (xb * pc - C.sgD[nu] * pm) * i1;
                hn = (xb * hc - C.sgD[nu] * hm) * i1;
            }
        } else {
            const double xb = x - __ldg(C.beta + nu);
            const double i1 = __ldg(C.isg + nu + 1);
            if (nu == 0) {
                pn = xb * pc * i1;
                hn = (xb * hc - C.sqrt_mu0) * i1;
            } else {
                const double s0 = __ldg(C.sg + nu);
                pn = (xb * pc - s0 * pm) * i1;
                hn = (xb * hc - s0 * hm) * i1;
            }
        }
        pm = pc;
        pc = pn;
        hm = hc;
        hc = hn;
    }
}

__global__ void columns_kernel(Rec C, ColArgs A) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const bool near = j < A.n && near_end(A.t[j]);
    const bool warp_dw = __any_sync(0xffffffffu, near);
    if (j >= A.n) return;
    if (warp_dw)
        walk_columns<true>(C, A, j);
    else
        walk_columns<false>(C, A, j);
}

// device buffers released on every path
// ------------------------------------------------------------ pivoted QR (pivots only)
// Businger--Golub Householder QR with column pivoting of an m x n complex matrix held row by
// row (A[i n + j], so that the threads of a column-parallel update read consecutive words),
// the first k steps, returning the pivot columns in order.  Every product and sum is rounded
// on its own (no fused multiply-add) and each column's sums run over i in increasing order,
// as in the host routine, so both pick the same pivots but for the last bits of |x0| (hypot).
struct QrState {
    double vn;   // squared norm of the current reflector; 0: no reflection this step
    int stop;    // the pivot column was zero: every later step is skipped
};
__device__ __forceinline__ double qr_norm2(double2 z) { return __dadd_rn(__dmul_rn(z.x, z.x), __dmul_rn(z.y, z.y)); }

__global__ void qr_norms_kernel(const double2* __restrict__ A, int m, int n, double* norms, int* perm) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double s = 0.0;
    for (int i = 0; i < m; ++i) s = __dadd_rn(s, qr_norm2(A[(size_t)i * n + j]));
    norms[j] = s;
    perm[j] = j;
}

// Step s, one CTA: the largest remaining norm (first index on ties), the column swap, and
// the reflector v (rows s..m-1) with its squared norm.
constexpr int QR_PIVOT_THREADS = 1024;
__global__ void __launch_bounds__(QR_PIVOT_THREADS) qr_pivot_kernel(double2* A, int m, int n, int s, double* norms,
                                                                    int* perm, double2* v, QrState* st) {
    __shared__ double bv[QR_PIVOT_THREADS];
    __shared__ int bi[QR_PIVOT_THREADS];
    __shared__ int piv;
    if (st->stop) return;  // uniform: written by thread 0 of an earlier step
    double best = -1.0;
    int bidx = n;
    for (int j = s + (int)threadIdx.x; j < n; j += QR_PIVOT_THREADS) {
        const double x = norms[j];
        if (x > best) {
            best = x;
            bidx = j;
        }
    }
    bv[threadIdx.x] = best;
    bi[threadIdx.x] = bidx;
    __syncthreads();
    for (int w = QR_PIVOT_THREADS / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            const double o = bv[threadIdx.x + w];
            const int oi = bi[threadIdx.x + w];
            if (o > bv[threadIdx.x] || (o == bv[threadIdx.x] && oi < bi[threadIdx.x])) {
                bv[threadIdx.x] = o;
                bi[threadIdx.x] = oi;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) piv = (bv[0] > norms[s]) ? bi[0] : s;  // the host keeps s unless strictly larger
    __syncthreads();
    const int p = piv;
    if (p != s) {
        for (int i = threadIdx.x; i < m; i += QR_PIVOT_THREADS) {
            const double2 a = A[(size_t)i * n + s];
            A[(size_t)i * n + s] = A[(size_t)i * n + p];
            A[(size_t)i * n + p] = a;
        }
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    if (p != s) {
        const double t = norms[s];
        norms[s] = norms[p];
        norms[p] = t;
        const int q = perm[s];
        perm[s] = perm[p];
        perm[p] = q;
    }
    double xn = 0.0;
    for (int i = s; i < m; ++i) xn = __dadd_rn(xn, qr_norm2(A[(size_t)i * n + s]));
    xn = sqrt(xn);
    if (xn == 0.0) {
        st->stop = 1;
        st->vn = 0.0;
        return;
    }
    const double2 x0 = A[(size_t)s * n + s];
    const double ax0 = hypot(x0.x, x0.y);
    const double2 ph = (ax0 > 0.0) ? make_double2(__ddiv_rn(x0.x, ax0), __ddiv_rn(x0.y, ax0)) : make_double2(1.0, 0.0);
    const double2 alpha = make_double2(-__dmul_rn(ph.x, xn), -__dmul_rn(ph.y, xn));
    double vn = 0.0;
    for (int i = s; i < m; ++i) {
        double2 vi = A[(size_t)i * n + s];
        if (i == s) vi = make_double2(__dsub_rn(vi.x, alpha.x), __dsub_rn(vi.y, alpha.y));
        v[i] = vi;
        vn = __dadd_rn(vn, qr_norm2(vi));
    }
    st->vn = vn;
}

// Step s: reflect every column j > s (one thread a column) and recompute its trailing norm.
__global__ void qr_update_kernel(double2* A, int m, int n, int s, double* norms, const double2* __restrict__ v,
                                 const QrState* st) {
    const int j = s + 1 + blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n || st->stop || st->vn == 0.0) return;
    double2 w = make_double2(0.0, 0.0);
    for (int i = s; i < m; ++i) {
        const double2 vi = v[i], c = A[(size_t)i * n + j];
        // conj(v_i) c_i
        w.x = __dadd_rn(w.x, __dsub_rn(__dmul_rn(vi.x, c.x), __dmul_rn(-vi.y, c.y)));
        w.y = __dadd_rn(w.y, __dadd_rn(__dmul_rn(vi.x, c.y), __dmul_rn(-vi.y, c.x)));
    }
    const double f = __ddiv_rn(2.0, st->vn);
    w = make_double2(__dmul_rn(w.x, f), __dmul_rn(w.y, f));
    double nn = 0.0;
    for (int i = s; i < m; ++i) {
        const double2 vi = v[i];
        double2 c = A[(size_t)i * n + j];
        const double2 wv = make_double2(__dsub_rn(__dmul_rn(w.x, vi.x), __dmul_rn(w.y, vi.y)),
                                        __dadd_rn(__dmul_rn(w.x, vi.y), __dmul_rn(w.y, vi.x)));
        c = make_double2(__dsub_rn(c.x, wv.x), __dsub_rn(c.y, wv.y));
        A[(size_t)i * n + j] = c;
        if (i > s) nn = __dadd_rn(nn, qr_norm2(c));
    }
    norms[j] = nn;
}

struct DevBufs {
    std::vector<void*> p;
    ~DevBufs() {
        for (void* q : p) cudaFree(q);
    }
    template <class T>
    T* put(const T* host, size_t count) {
        void* d = nullptr;
        if (cudaMalloc(&d, sizeof(T) * std::max<size_t>(count, 1)) != cudaSuccess) return nullptr;
        p.push_back(d);
        if (count && cudaMemcpy(d, host, sizeof(T) * count, cudaMemcpyHostToDevice) != cudaSuccess) return nullptr;
        return static_cast<T*>(d);
    }
    template <class T>
    T* alloc(size_t count) {
        void* d = nullptr;
        if (cudaMalloc(&d, sizeof(T) * std::max<size_t>(count, 1)) != cudaSuccess) return nullptr;
        p.push_back(d);
        return static_cast<T*>(d);
    }
};

bool upload_rec(DevBufs& B, const SetupRec& H, Rec& C) {
    const size_t m = H.beta.size();
    C.beta = B.put(H.beta.data(), m);
    C.sg = B.put(H.sg.data(), m);
    C.isg = B.put(H.isg.data(), m);
    C.betaD = reinterpret_cast<const dd2*>(B.put(H.betaD.data(), 2 * m));
    C.sgD = reinterpret_cast<const dd2*>(B.put(H.sgD.data(), 2 * m));
    C.isgD = reinterpret_cast<const dd2*>(B.put(H.isgD.data(), 2 * m));
    C.p0 = H.p0;
    C.sqrt_mu0 = H.sqrt_mu0;
    return C.beta && C.sg && C.isg && C.betaD && C.sgD && C.isgD;
}

}  // namespace

jt_status gpu_newton_nodes(const SetupRec& H, int64_t n, double maxstep, double* t, double* omega) {
    if (n > (int64_t)1 << 30) return JT_EINVAL;
    DevBufs B;
    Rec C{};
    if (!upload_rec(B, H, C)) {
        cudaGetLastError();
        return JT_ECUDA;
    }
    double* dt = B.put(t, (size_t)n);
    double* dw = B.alloc<double>((size_t)n);
    if (!dt || !dw) {
        cudaGetLastError();
        return JT_ECUDA;
    }
    const int threads = 128;
    newton_nodes_kernel<<<(unsigned)((n + threads - 1) / threads), threads>>>(C, (int)n, maxstep, dt, dw);
    if (cudaGetLastError() != cudaSuccess || cudaMemcpy(t, dt, sizeof(double) * n, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(omega, dw, sizeof(double) * n, cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return JT_ECUDA;
    }
    return JT_OK;
}

// Device copies of one axis's tables for the column walks, made once per setup and reused by
// every gpu_columns call of that setup (the output buffer grows as needed).
struct GpuColumns {
    DevBufs bufs;
    Rec C{};
    ColArgs A{};
    int* slot = nullptr;
    double2* out = nullptr;
    size_t out_cap = 0;
    std::vector<int> hslot;
    cudaStream_t stream = nullptr;
    // pivoted-QR work area (grown as needed): the matrix, its column norms, the permutation,
    // the reflector and the step state
    double2* qa = nullptr;
    size_t qa_cap = 0;
    double* qnorm = nullptr;
    int* qperm = nullptr;
    size_t qn_cap = 0;
    double2* qv = nullptr;
    int qv_cap = 0;
    QrState* qst = nullptr;
    ~GpuColumns() {
        if (out) cudaFree(out);
        if (qa) cudaFree(qa);
        if (qnorm) cudaFree(qnorm);
        if (qperm) cudaFree(qperm);
        if (qv) cudaFree(qv);
        if (qst) cudaFree(qst);
        if (stream) cudaStreamDestroy(stream);
    }
};

GpuColumns* gpu_columns_create(const SetupRec& H, const AxisTables& T) {
    GpuColumns* g = new GpuColumns();
    bool ok = cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking) == cudaSuccess && upload_rec(g->bufs, H, g->C);
    const int64_t n = T.n;
    std::vector<double2> phase((size_t)T.L);
    for (int64_t r = 0; r < T.L; ++r) {
        const double ang = -2.0 * PI_D * (double)r / (double)T.L;
        phase[r] = make_double2(std::cos(ang), std::sin(ang));
    }
    ColArgs& A = g->A;
    if (ok) {
        A.t = g->bufs.put(T.t.data(), (size_t)n);
        A.rowP = g->bufs.put(T.rowP.data(), (size_t)n);
        A.rowQ = g->bufs.put(T.rowQ.data(), (size_t)n);
        A.S = g->bufs.put(T.S.data(), (size_t)n);
        A.m = g->bufs.put(T.m.data(), (size_t)n);
        A.phase = g->bufs.put(phase.data(), phase.size());
        g->slot = g->bufs.alloc<int>((size_t)T.N);
        ok = A.t && A.rowP && A.rowQ && A.S && A.m && A.phase && g->slot;
    }
    A.slot = g->slot;
    A.n = (int)n;
    A.nu0 = T.nu0;
    A.L = T.L;
    g->hslot.assign((size_t)T.N, -1);
    if (!ok) {
        cudaGetLastError();
        delete g;
        return nullptr;
    }
    return g;
}

void gpu_columns_destroy(GpuColumns* g) { delete g; }

jt_status gpu_columns(GpuColumns* g, const std::vector<int>& cl, cd* out) {
    if (!g) return JT_ECUDA;
    if (cl.empty()) return JT_OK;
    const size_t n = (size_t)g->A.n;
    const size_t need = n * cl.size();
    if (need > g->out_cap) {
        if (g->out) cudaFree(g->out);
        g->out = nullptr;
        g->out_cap = 0;
        if (cudaMalloc((void**)&g->out, sizeof(double2) * need) != cudaSuccess) {
            cudaGetLastError();
            return JT_ECUDA;
        }
        g->out_cap = need;
    }
    std::fill(g->hslot.begin(), g->hslot.end(), -1);
    for (size_t q = 0; q < cl.size(); ++q) g->hslot[cl[q]] = (int)q;
    ColArgs A = g->A;
    A.out = g->out;
    A.last = A.nu0 + cl.back();
    static_assert(sizeof(cd) == sizeof(double2), "complex<double> and double2 share a layout");
    const int threads = 128;
    if (cudaMemcpyAsync(g->slot, g->hslot.data(), sizeof(int) * g->hslot.size(), cudaMemcpyHostToDevice, g->stream) !=
        cudaSuccess) {
        cudaGetLastError();
        return JT_ECUDA;
    }
    columns_kernel<<<(unsigned)((n + threads - 1) / threads), threads, 0, g->stream>>>(g->C, A);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(out, g->out, sizeof(double2) * need, cudaMemcpyDeviceToHost, g->stream) != cudaSuccess ||
        cudaStreamSynchronize(g->stream) != cudaSuccess) {
        cudaGetLastError();
        return JT_ECUDA;
    }
    return JT_OK;
}


jt_status gpu_qrcp_pivots(GpuColumns* g, const cd* A, int m, int n, int k, std::vector<int>& pivots) {
    pivots.clear();
    if (!g) return JT_ECUDA;
    k = std::min(k, std::min(m, n));
    if (k <= 0) return JT_OK;
    const size_t need = (size_t)m * (size_t)n;
    auto grow = [](auto*& p, auto& cap, size_t count) -> bool {
        if ((size_t)count <= (size_t)cap) return true;
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        if (cudaMalloc((void**)&p, sizeof(*p) * count) != cudaSuccess) return false;
        cap = count;
        return true;
    };
    bool ok = grow(g->qa, g->qa_cap, need);
    if (ok && (size_t)n > g->qn_cap) {
        if (g->qnorm) cudaFree(g->qnorm);
        if (g->qperm) cudaFree(g->qperm);
        g->qnorm = nullptr;
        g->qperm = nullptr;
        g->qn_cap = 0;
        ok = cudaMalloc((void**)&g->qnorm, sizeof(double) * n) == cudaSuccess &&
             cudaMalloc((void**)&g->qperm, sizeof(int) * n) == cudaSuccess;
        if (ok) g->qn_cap = (size_t)n;
    }
    ok = ok && grow(g->qv, g->qv_cap, (size_t)m);
    if (ok && !g->qst) ok = cudaMalloc((void**)&g->qst, sizeof(QrState)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        return JT_ECUDA;
    }
    static_assert(sizeof(cd) == sizeof(double2), "complex<double> and double2 share a layout");
    cudaStream_t s = g->stream;
    const QrState st0{0.0, 0};
    if (cudaMemcpyAsync(g->qa, A, sizeof(double2) * need, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(g->qst, &st0, sizeof(QrState), cudaMemcpyHostToDevice, s) != cudaSuccess) {
        cudaGetLastError();
        return JT_ECUDA;
    }
    const int threads = 128;
    qr_norms_kernel<<<(unsigned)((n + threads - 1) / threads), threads, 0, s>>>(g->qa, m, n, g->qnorm, g->qperm);
    for (int step = 0; step < k; ++step) {
        qr_pivot_kernel<<<1, QR_PIVOT_THREADS, 0, s>>>(g->qa, m, n, step, g->qnorm, g->qperm, g->qv, g->qst);
        const int rest = n - (step + 1);
        if (rest > 0)
            qr_update_kernel<<<(unsigned)((rest + threads - 1) / threads), threads, 0, s>>>(g->qa, m, n, step, g->qnorm,
                                                                                         g->qv, g->qst);
    }
    pivots.assign((size_t)k, 0);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(pivots.data(), g->qperm, sizeof(int) * k, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        pivots.clear();
        return JT_ECUDA;
    }
    return JT_OK;
}

}  // namespace jt
