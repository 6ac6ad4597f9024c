// Fused axis kernels of the fast Jacobi transform (Sec. 3.1, Eqs. eq:oneJ and eq:oneJinv),
// templated on the arithmetic: `float` (FP32) or `dw` (double-word: an unevaluated sum
// hi + lo of two floats).
//
// One kernel launch applies the 1-D operator A = W [V, Re(sum_k D_{u_k} F D_{v_k})] (forward)
// or its transpose (adjoint) to every fibre of one axis of a row-major array.  Per fibre,
// a group of T threads keeps the fibre's data in registers and, for every rank term k,
//   forward:  x = v_k .* alpha  (bins 0..L-1)  ->  y = IDFT_L(x)  ->  acc_j += Re(u_k[j] y[m_j])
//   adjoint:  z[m] = sum_{j: m_j = m} u_k[j] g_j  ->  y = IDFT_L(z)  ->  acc_nu += Re(v_k[nu] y[nu])
// with IDFT_L the unnormalised e^{+2 pi i m nu / L} transform, then adds the dense low-degree
// block (degrees < nu0) and writes the fibre once.  The weights sqrt(w_j) are folded into
// u_k and into the dense block at plan creation, so no separate scaling pass exists.
//
// FFT: Stockham auto-sort passes of radix <= 16.  Thread t of a group owns elements
// t + T e (e < E = L / T) in registers; the first pass works entirely in registers, each
// later pass exchanges through shared memory (padded one word per 32 against bank
// conflicts), and the last pass leaves its outputs in the same t + T e layout.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace jt {
namespace dev {

// ------------------------------------------------------------ double-word floats
// Dekker (1971) and Joldes, Muller, Popescu (ACM TOMS 2017): TwoSum, Fast2Sum, the
// FMA-based exact product, SloppyDWPlusDW and DWTimesDW.
// 8-byte aligned, so that a double-word (and, below, a complex double-word: 16 bytes) is read
// and written with one vector access rather than one per float.
struct __align__(8) dw {
    float hi, lo;
};

__device__ __forceinline__ dw two_sum(float a, float b) {
    float s = a + b;
    float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ dw fast_two_sum(float a, float b) {
    float s = a + b;
    return {s, b - (s - a)};
}
// Sum of two double-words by SloppyDWPlusDW (Joldes, Muller, Popescu 2017, Algorithm 5):
// TwoSum of the high parts, the low parts added in plain FP32, one Fast2Sum (11 flops, against
// 20 for AccurateDWPlusDW).  Its error is at most a small multiple of u^2 (|x| + |y|) rather
// than of u^2 |x + y|: a bound relative to the operands, which is the form the error analysis
// of an FFT (butterflies a +- w b) and of a sum over rank terms needs, so the transforms keep
// their ~u^2 log L normwise accuracy.
__device__ __forceinline__ dw operator+(dw x, dw y) {
    dw s = two_sum(x.hi, y.hi);
    return fast_two_sum(s.hi, s.lo + (x.lo + y.lo));
}
__device__ __forceinline__ dw operator-(dw x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ dw operator-(dw x, dw y) { return x + (-y); }
__device__ __forceinline__ dw operator*(dw x, dw y) {
    float ch = x.hi * y.hi;
    float cl1 = __fmaf_rn(x.hi, y.hi, -ch);
    float tl0 = x.lo * y.lo;
    float tl1 = __fmaf_rn(x.hi, y.lo, tl0);
    float cl2 = __fmaf_rn(x.lo, y.hi, tl1);
    return fast_two_sum(ch, cl1 + cl2);
}

template <class R>
struct RealOps;
template <>
struct RealOps<float> {
    using io = float;  // element type of the arrays the caller passes
    static __host__ __device__ __forceinline__ float zero() { return 0.0f; }
    static __device__ __forceinline__ float from_io(float v) { return v; }
    static __device__ __forceinline__ float to_io(float v) { return v; }
};
template <>
struct RealOps<dw> {
    using io = double;
    static __host__ __device__ __forceinline__ dw zero() { return {0.0f, 0.0f}; }
    static __device__ __forceinline__ dw from_io(double v) {
        float h = (float)v;
        return {h, (float)(v - (double)h)};
    }
    static __device__ __forceinline__ double to_io(dw v) { return (double)v.hi + (double)v.lo; }
};

// compile-time constant in the working precision
template <class R>
__device__ __forceinline__ R rc(double v);
template <>
__device__ __forceinline__ float rc<float>(double v) {
    return (float)v;
}
template <>
__device__ __forceinline__ dw rc<dw>(double v) {
    float h = (float)v;
    return {h, (float)(v - (double)h)};
}

template <class R>
struct Cx {
    R re, im;
};
template <>
struct __align__(16) Cx<dw> {
    dw re, im;
};
template <class R>
__device__ __forceinline__ Cx<R> operator+(Cx<R> a, Cx<R> b) {
    return {a.re + b.re, a.im + b.im};
}
template <class R>
__device__ __forceinline__ Cx<R> operator-(Cx<R> a, Cx<R> b) {
    return {a.re - b.re, a.im - b.im};
}
// FP32: complex add and subtract as one paired-FP32 instruction each (add/sub.rn.f32x2,
// sm_100 and later), which halves the FP32 instructions of the FFT butterflies.
__device__ __forceinline__ unsigned long long pack2(Cx<float> a) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.re), "f"(a.im));
    return r;
}
__device__ __forceinline__ Cx<float> unpack2(unsigned long long r) {
    Cx<float> o;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(o.re), "=f"(o.im) : "l"(r));
    return o;
}
__device__ __forceinline__ Cx<float> operator+(Cx<float> a, Cx<float> b) {
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pack2(a)), "l"(pack2(b)));
    return unpack2(r);
}
__device__ __forceinline__ Cx<float> operator-(Cx<float> a, Cx<float> b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pack2(a)), "l"(pack2(b)));
    return unpack2(r);
}

template <class R>
__device__ __forceinline__ Cx<R> cmul(Cx<R> a, Cx<R> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
// Double-word operations inside the FFT without the final renormalisation: TwoSum of the high
// parts with the low parts added in FP32 (8 operations against 11), and the FMA-based product
// without its lo x lo term (5 operations against 9).  The result is an unevaluated sum hi + lo
// whose lo may exceed half an ulp of hi; TwoSum and the FMA error term stay exact for such
// inputs, so the rounding left is that of the FP32 low parts (a few u^2 of the values).  Every
// DFT renormalises its outputs once (Fast2Sum), and a twiddle product or a scaling feeds a DFT.
__device__ __forceinline__ dw add_nr(dw x, dw y) {
    const dw s = two_sum(x.hi, y.hi);
    return {s.hi, s.lo + (x.lo + y.lo)};
}
__device__ __forceinline__ dw sub_nr(dw x, dw y) { return add_nr(x, dw{-y.hi, -y.lo}); }
__device__ __forceinline__ dw mul_nr(dw x, dw y) {
    const float ch = x.hi * y.hi;
    const float cl1 = __fmaf_rn(x.hi, y.hi, -ch);
    const float cl2 = __fmaf_rn(x.lo, y.hi, x.hi * y.lo);
    return {ch, cl1 + cl2};
}
__device__ __forceinline__ dw renorm(dw x) { return fast_two_sum(x.hi, x.lo); }
__device__ __forceinline__ Cx<dw> cmul(Cx<dw> a, Cx<dw> b) {
    return {sub_nr(mul_nr(a.re, b.re), mul_nr(a.im, b.im)), add_nr(mul_nr(a.re, b.im), mul_nr(a.im, b.re))};
}
__device__ __forceinline__ Cx<dw> cscale(Cx<dw> a, dw s) { return {mul_nr(a.re, s), mul_nr(a.im, s)}; }
// Re(a b) added at once to a normalised accumulator by the full double-word sum
__device__ __forceinline__ dw re_mul(Cx<dw> a, Cx<dw> b) { return sub_nr(mul_nr(a.re, b.re), mul_nr(a.im, b.im)); }

// Butterfly sums and the products of the constant twiddles inside a DFT (unnormalised for
// double-words).
template <class R>
__device__ __forceinline__ Cx<R> bf_add(Cx<R> a, Cx<R> b) {
    return a + b;
}
template <class R>
__device__ __forceinline__ Cx<R> bf_sub(Cx<R> a, Cx<R> b) {
    return a - b;
}
__device__ __forceinline__ Cx<dw> bf_add(Cx<dw> a, Cx<dw> b) { return {add_nr(a.re, b.re), add_nr(a.im, b.im)}; }
__device__ __forceinline__ Cx<dw> bf_sub(Cx<dw> a, Cx<dw> b) { return {sub_nr(a.re, b.re), sub_nr(a.im, b.im)}; }
template <class R>
__device__ __forceinline__ Cx<R> h_rot(Cx<R> v, R h) {  // ((re - im) h, (re + im) h)
    return {(v.re - v.im) * h, (v.re + v.im) * h};
}
__device__ __forceinline__ Cx<dw> h_rot(Cx<dw> v, dw h) {
    return {mul_nr(sub_nr(v.re, v.im), h), mul_nr(add_nr(v.re, v.im), h)};
}
template <class R>
__device__ __forceinline__ void dft_out(Cx<R>* a, int n) {}
__device__ __forceinline__ void dft_out(Cx<dw>* a, int n) {
    for (int i = 0; i < n; ++i) a[i] = Cx<dw>{renorm(a[i].re), renorm(a[i].im)};
}

template <class R>
__device__ __forceinline__ Cx<R> mul_i(Cx<R> a) {  // multiply by +i
    return {-a.im, a.re};
}
template <class R>
__device__ __forceinline__ Cx<R> cscale(Cx<R> a, R s) {
    return {a.re * s, a.im * s};
}
template <class R>
__device__ __forceinline__ R re_mul(Cx<R> a, Cx<R> b) {  // Re(a b)
    return a.re * b.re - a.im * b.im;
}

// Multiply by the twiddle e^{+2 pi i K / N} with compile-time K, N: the trivial cases
// (1, i, -1, -i, (+-1 + i)/sqrt 2 ...) cost no general complex product.
template <int K, int N, class R>
__device__ __forceinline__ Cx<R> twc(Cx<R> v) {
    constexpr int k = ((K % N) + N) % N;
    if constexpr (k == 0) {
        return v;
    } else if constexpr (4 * k == N) {
        return mul_i(v);
    } else if constexpr (2 * k == N) {
        return {-v.re, -v.im};
    } else if constexpr (4 * k == 3 * N) {
        return {v.im, -v.re};
    } else if constexpr (8 * k == N || 8 * k == 3 * N || 8 * k == 5 * N || 8 * k == 7 * N) {
        const R h = rc<R>(0.70710678118654752440084436210484903928);
        // (1 + i)/sqrt2 rotated by the multiple of i
        Cx<R> r = h_rot(v, h);
        if constexpr (8 * k == N) return r;
        if constexpr (8 * k == 3 * N) return mul_i(r);
        if constexpr (8 * k == 5 * N) return {-r.re, -r.im};
        return {r.im, -r.re};
    } else if constexpr (N == 32 && (k & 1) == 0) {
        return twc<k / 2, 16, R>(v);
    } else {
        // remaining cases: N = 16 or 32 with k odd, from the first-octant values of
        // cos and sin of multiples of pi/16 and the symmetries of the circle
        static_assert((N == 16 || N == 32) && (k & 1), "twiddle table covers radices up to 32");
        constexpr int k32 = (N == 16) ? 2 * k : k;  // angle = 2 pi k32 / 32
        constexpr double C[9] = {1.0,
                                 0.98078528040323044912618223613424033391,
                                 0.92387953251128675612818318939678828682,
                                 0.83146961230254523707878837761790575673,
                                 0.70710678118654752440084436210484903928,
                                 0.55557023301960222474283081394853287438,
                                 0.38268343236508977172845998403039886676,
                                 0.19509032201612826784828486847702224467,
                                 0.0};
        // cos(2 pi q / 32) for any q, from C[] with C[i] = cos(i pi / 16), i = 0..8
        constexpr int q = k32 % 32;
        constexpr int qc = (q <= 8) ? q : (q <= 16) ? 16 - q : (q <= 24) ? q - 16 : 32 - q;
        constexpr double cs = (q <= 8 || q >= 24) ? C[qc] : -C[qc];
        constexpr int qs = (q + 24) % 32;  // sin(x) = cos(x - pi/2)
        constexpr int qsc = (qs <= 8) ? qs : (qs <= 16) ? 16 - qs : (qs <= 24) ? qs - 16 : 32 - qs;
        constexpr double sn = (qs <= 8 || qs >= 24) ? C[qsc] : -C[qsc];
        const Cx<R> w{rc<R>(cs), rc<R>(sn)};
        return cmul(v, w);
    }
}

// Unnormalised DFT of size R with sign +: b_q = sum_r a_r e^{+2 pi i r q / R}, in natural
// order, by radix-2 decimation in time with compile-time twiddles.
template <int R>
struct Bitrev {
    static constexpr int lg = (R <= 1) ? 0 : (R == 2) ? 1 : (R == 4) ? 2 : (R == 8) ? 3 : 4;
    static constexpr __host__ __device__ int rev(int i) {
        int r = 0;
        for (int b = 0; b < lg; ++b)
            if (i & (1 << b)) r |= 1 << (lg - 1 - b);
        return r;
    }
};

template <int LEN, int HALF, int K, class R>
__device__ __forceinline__ void dft_stage_k(Cx<R>* t, int i) {
    Cx<R> u = t[i + K];
    Cx<R> v = twc<K, LEN, R>(t[i + K + HALF]);
    t[i + K] = bf_add(u, v);
    t[i + K + HALF] = bf_sub(u, v);
}

template <int LEN, int R, class Rt>
__device__ __forceinline__ void dft_stage(Cx<Rt>* t) {
    constexpr int HALF = LEN / 2;
#pragma unroll
    for (int i = 0; i < R; i += LEN) {
        if constexpr (HALF > 0) dft_stage_k<LEN, HALF, 0, Rt>(t, i);
        if constexpr (HALF > 1) dft_stage_k<LEN, HALF, 1, Rt>(t, i);
        if constexpr (HALF > 2) {
            dft_stage_k<LEN, HALF, 2, Rt>(t, i);
            dft_stage_k<LEN, HALF, 3, Rt>(t, i);
        }
        if constexpr (HALF > 4) {
            dft_stage_k<LEN, HALF, 4, Rt>(t, i);
            dft_stage_k<LEN, HALF, 5, Rt>(t, i);
            dft_stage_k<LEN, HALF, 6, Rt>(t, i);
            dft_stage_k<LEN, HALF, 7, Rt>(t, i);
        }
    }
}

// 16-point DFT of an input whose entries 9..15 are zero (the adjoint's bins above L/2): the
// first radix-2 stage pairs a[r] with a[r + 8], which is zero for r >= 1.
template <class Rt>
__device__ __forceinline__ void dft16_low9(Cx<Rt>* a) {
    Cx<Rt> t[16];
    t[0] = a[0] + a[8];
    t[1] = a[0] - a[8];
#pragma unroll
    for (int q = 1; q < 8; ++q) {
        const int r = Bitrev<16>::rev(2 * q);  // r < 8, partner r + 8 is zero
        t[2 * q] = a[r];
        t[2 * q + 1] = a[r];
    }
    dft_stage<4, 16, Rt>(t);
    dft_stage<8, 16, Rt>(t);
    dft_stage<16, 16, Rt>(t);
#pragma unroll
    for (int i = 0; i < 16; ++i) a[i] = t[i];
}

template <int R, class Rt>
__device__ __forceinline__ void dft(Cx<Rt>* a) {
    if constexpr (R == 1) {
        return;
    } else {
        Cx<Rt> t[R];
#pragma unroll
        for (int i = 0; i < R; ++i) t[Bitrev<R>::rev(i)] = a[i];
        if constexpr (R >= 2) dft_stage<2, R, Rt>(t);
        if constexpr (R >= 4) dft_stage<4, R, Rt>(t);
        if constexpr (R >= 8) dft_stage<8, R, Rt>(t);
        if constexpr (R >= 16) dft_stage<16, R, Rt>(t);
        dft_out(t, R);
#pragma unroll
        for (int i = 0; i < R; ++i) a[i] = t[i];
    }
}

// ------------------------------------------------------------------ geometry
template <class R>
struct RegRadix {
    static constexpr int lg = 4;  // FP32: 16 complex elements per thread
};
template <>
struct RegRadix<dw> {
    static constexpr int lg = 3;  // double-word: 8 (twice the registers per element)
};

template <class R, int LOG2L>
struct Shape {
    static constexpr int LG = RegRadix<R>::lg;
    static constexpr int EMAX = 1 << LG;
    static constexpr int L = 1 << LOG2L;
    static constexpr int E = (L < EMAX) ? L : EMAX;                      // elements per thread
    static constexpr int T = L / E;                                      // threads per fibre
    static constexpr int G = (T >= 256) ? 1 : 256 / T;                   // fibres per CTA
    static constexpr int THREADS = G * T;
    static constexpr int P = (LOG2L <= LG) ? 1 : (LOG2L + LG - 1) / LG;  // Stockham passes
    static constexpr int R0 = 1 << (LOG2L - LG * (P - 1));               // radix of the first pass
    // FP32: separate re / im arrays of L + L/32 + 1 floats, one word of padding per 32.
    // Double-word: one array of complex double-words (16 bytes), one entry of padding per 8, so
    // that the 8 lanes of a quarter-warp touch 8 different 16-byte bank groups in every pass.
    static constexpr bool CPLX = sizeof(R) == 8;
    static constexpr int PADL = CPLX ? L + (L >> 3) + 1 : L + (L >> 5) + 1;
    static __host__ __device__ constexpr int pad(int i) { return CPLX ? i + (i >> 3) : i + (i >> 5); }
    // per group: the exchange buffer (2 PADL reals), then L reals of fibre data, kept even
    static constexpr int GSTRIDE = ((2 * PADL + L) + 1) & ~1;
};

// FP32 axes longer than 4096 (the Stockham kernel's long instances) get their twiddle table
// in pass order from the plan: at [NS - R0 + (r - 1) NS + k] the twiddle e^{2 pi i r k / (16 NS)}
// of the pass of span NS, so that the 32 lanes of a pass read 32 consecutive entries (in
// natural order they read one 32-byte sector each, and the table missed L1).
// The adjoint of the FP32 long instances and of the double-word instances gathers each bin's
// first two points from a bin-ordered copy of u_k and a bin-ordered point table (AxisDev ubtab
// / bjtab, [k][(s * 2 + i) * T + t] for bin m = t + T s) instead of walking the CSR lists: in
// the walk every bin's loads waited on the previous bin's (one L2 round trip after another in
// FP32), and the trip counts differed from thread to thread; the double-word reads of u_k at
// points two apart also met bank conflicts in the streamed slice.
template <class R, int LOG2L>
struct BinOrd {
    static constexpr bool value = (sizeof(R) == 4 && LOG2L >= 13) || sizeof(R) == 8;
    // bin slots of the table: FP32 the four-step kernel's nine (m = t + T s, s <= 8); double-
    // word E / 2 (E = 8 elements a thread, or L when L < 8), bin L/2 then walked by thread 0
    static constexpr int SLOTS = (sizeof(R) == 4) ? 9 : ((1 << LOG2L) < 8 ? (1 << LOG2L) : 8) / 2;
};
template <class R, int LOG2L>
struct TwPass {
    static constexpr bool value = sizeof(R) == 4 && LOG2L >= 13;
};
// Double-word instances up to L = 2048, and FP32 at L = 8192, read their twiddles from a
// per-CTA copy in shared memory instead of the (L1-cached) table: every rank term of every
// fibre re-reads them.
template <class R, int LOG2L>
struct TwSmem {
    static constexpr bool value = (sizeof(R) == 8 && LOG2L >= 1 && LOG2L <= 11) || (sizeof(R) == 4 && LOG2L == 13);
};

// The exchange buffer of one group: (re, im) arrays for FP32, interleaved complex double-words.
template <class R>
struct XBuf {
    R* re;
    R* im;
    template <class S>
    __device__ __forceinline__ void put(int i, Cx<R> v) const {
        re[S::pad(i)] = v.re;
        im[S::pad(i)] = v.im;
    }
    template <class S>
    __device__ __forceinline__ Cx<R> get(int i) const {
        return Cx<R>{re[S::pad(i)], im[S::pad(i)]};
    }
};
template <>
struct XBuf<dw> {
    dw* re;  // start of the buffer: Cx<dw>[PADL]
    dw* im;  // unused
    template <class S>
    __device__ __forceinline__ void put(int i, Cx<dw> v) const {
        reinterpret_cast<Cx<dw>*>(re)[S::pad(i)] = v;
    }
    template <class S>
    __device__ __forceinline__ Cx<dw> get(int i) const {
        return reinterpret_cast<const Cx<dw>*>(re)[S::pad(i)];
    }
};

// Tables of one axis on the device (all owned by the plan).
struct AxisDev {
    int n, L, nu0, rank;
    int sorted;          // 1 if m_j is non-decreasing in j (bin_idx is the identity)
    const void* vtab;    // rank x L   Cx<R>: v_k at bins nu0..n-1, zero elsewhere
    const void* utab;    // rank x n   Cx<R>: sqrt(w_j) u_k[j]
    const int* mtab;     // n          FFT bin of point j
    const void* vblk;    // nu0 x n    R:     sqrt(w_j) P~_c(t_j)
    const void* twid;    // L          Cx<R>: e^{+2 pi i s / L} (TwPass axes: in Stockham pass order)
    const int* bin_ptr;  // L/2 + 2    points of bin m: bin_idx[bin_ptr[m] .. bin_ptr[m+1])
    const int* bin_idx;  // n
    // FP32 warp kernel only: u_k in bin order, rank x 9 x 2 x T complex; entry
    // [k][(s * 2 + i) * T + t] is u_k at the i-th point of bin m = t + T s (zero if none)
    const void* ubtab;
    const int* bjtab;    // [(s * 2 + i) * T + t]: the point of that slot, or -1 (same layout as ubtab)
    // Points beyond the first two of a bin (FP32 warp kernel, adjoint).  ovmode 0: there are
    // none; 1: per-lane lists, ovftab[2t] the number of extra points of lane t,
    // ovj[i * T + t] its i-th one as j | s << 20 (s the lane's bin slot) and ovu[k][i * T + t]
    // u_k there; 2 (a bin holds more than 17 points): ovftab[2t] != 0 marks the lanes that walk
    // bin_ptr / bin_idx instead.
    // FP32 warp kernel, adjoint: v_k in each lane's output order, [k][o][t] = v_k[Own(t, o)]
    const void* vown;
    const int* ovftab;
    const int* ovj;
    const void* ovu;
    int ovmax, ovmode;
    // FP32 warp kernel, forward, when no bin holds more than two points (fbin = 1): u_k at the
    // points of each lane's output bins after step B, [k][(c * 2 + i) * T + t] for the i-th point
    // of bin Own(t, fslot(c)), c = 0..8 (zero where there is none), and those points (or -1)
    const void* fbtab;
    const int* bjf;
    int fbin;
    // Plan-owned status word: bit 0 is set when a bounded wait of a kernel ran out (the kernel
    // then returns early; the plan reports JT_ETIMEOUT).  skip_copy (tests only): the FP32
    // four-step kernel issues no table copy, so its first wait runs out.
    unsigned* status;
    int skip_copy;
};

// Extra tables of a double-word axis of length L = 16384, applied as two half-length
// transforms (jt_axis_dw_big.cu).  Owned by the plan.
struct BigAxisDev {
    int n = 0, nu0 = 0, rank = 0;
    int max_ctas = 0;             // rows of `part` (CTAs of one launch)
    const Cx<dw>* vtab = nullptr;  // rank x L: v_k at bins nu0..n-1 (the axis table)
    const Cx<dw>* utab = nullptr;  // rank x n: u_k (parity 0)
    const Cx<dw>* utab1 = nullptr; // rank x n: u_k[j] e^{2 pi i m_j / L} (parity 1)
    const dw* vblk = nullptr;      // nu0 x n dense block
    const Cx<dw>* tw2 = nullptr;   // L/2: e^{2 pi i s / (L/2)}
    const int* mtab2 = nullptr;    // n: m_j mod L/2
    const int* bin_ptr2 = nullptr; // L/2 + 1: points of bin m' = m_j mod L/2
    const int* bin_idx2 = nullptr; // n
    dw* part = nullptr;            // max_ctas x n partial sums
};

// Bulk (TMA) copies of contiguous table slices into shared memory, completed on an mbarrier.
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// arrive once, announcing `bytes` of copies that complete on this barrier
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// global -> shared copy of `bytes` (multiple of 16; both addresses 16-byte aligned)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for the phase of `bar` with the given parity to complete, for at most about one second;
// false if the wait ran out.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
    const unsigned a = smem_u32(bar);
    unsigned long long t0 = 0;
    for (unsigned it = 0;; ++it) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if (it == 0) t0 = global_ns();
        else if ((it & 63) == 0 && (global_ns() - t0 > 1000000000ull || it > (1u << 24))) return false;
    }
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// ------------------------------------------------------------------ clusters
// Rank split: the CTAs of one thread-block cluster share a tile of fibres, CTA c of S taking
// the rank terms [rank c / S, rank (c + 1) / S), and add their partial sums through
// distributed shared memory.  A launch without a cluster attribute is a cluster of one CTA,
// so the same code serves S = 1.
__device__ __forceinline__ unsigned cluster_size() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cluster_index() {
    unsigned r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cluster_count() {
    unsigned r;
    asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
    return r;
}
// Every thread of every CTA of the cluster arrives; shared-memory writes made before it are
// visible to the cluster's loads after it.  A hardware barrier: no software spin.
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Load a float of CTA `rank`'s shared memory at the offset of `local` in this CTA's.
__device__ __forceinline__ float ld_cluster(const float* local, unsigned rank) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(local);
    unsigned ra;
    float v;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(ra) : "memory");
    return v;
}
template <class R>
__device__ __forceinline__ R ld_cluster_r(const R* local, unsigned rank);
template <>
__device__ __forceinline__ float ld_cluster_r<float>(const float* local, unsigned rank) {
    return ld_cluster(local, rank);
}
template <>
__device__ __forceinline__ dw ld_cluster_r<dw>(const dw* local, unsigned rank) {
    const float* p = reinterpret_cast<const float*>(local);
    return {ld_cluster(p, rank), ld_cluster(p + 1, rank)};
}

template <int T, int G>
__device__ __forceinline__ void group_sync(int g) {
    if constexpr (T <= 32) {
        __syncwarp();
    } else if constexpr (G == 1) {
        __syncthreads();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "r"(T) : "memory");
    }
}

// One Stockham pass of radix RX over span NS (product of the earlier radices).  Inputs of
// butterfly j = t + T b are x[b + r E/RX]; FIRST passes take them from registers, the others
// from shared memory.  LAST passes leave outputs in registers at x[b + q E/RX] (element
// t + T (b + q E/RX)); the others store them at their Stockham positions.
template <class R, int LOG2L, int RX, int NS, bool FIRST, bool LAST>
__device__ __forceinline__ void stockham_pass(Cx<R>* x, R* sre, R* sim, const Cx<R>* __restrict__ tw, int t,
                                              int g) {
    using S = Shape<R, LOG2L>;
    constexpr int L = S::L, E = S::E, T = S::T, G = S::G;
    constexpr int NB = E / RX;  // butterflies per thread
    if constexpr (!FIRST) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
            int b = e % NB, r = e / NB;
            int idx = t + T * b + r * (L / RX);
            x[e] = XBuf<R>{sre, sim}.template get<S>(idx);
        }
        group_sync<T, G>(g);  // every read done before this pass writes
    }
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        Cx<R> a[RX];
#pragma unroll
        for (int r = 0; r < RX; ++r) a[r] = x[b + r * NB];
        const int j = t + T * b;
        const int k = j & (NS - 1);
        if constexpr (NS > 1) {
#pragma unroll
            for (int r = 1; r < RX; ++r) {
                if constexpr (TwSmem<R, LOG2L>::value || TwPass<R, LOG2L>::value)  // [NS - R0 + (r - 1) NS + k]
                    a[r] = cmul(a[r], tw[(NS - S::R0) + (r - 1) * NS + k]);
                else
                    a[r] = cmul(a[r], tw[(r * k) * (L / (NS * RX))]);
            }
        }
        dft<RX, R>(a);
        if constexpr (LAST) {
#pragma unroll
            for (int q = 0; q < RX; ++q) x[b + q * NB] = a[q];
        } else {
            const int base = (j - k) * RX + k;
#pragma unroll
            for (int q = 0; q < RX; ++q) XBuf<R>{sre, sim}.template put<S>(base + q * NS, a[q]);
        }
    }
    if constexpr (!LAST) group_sync<T, G>(g);  // writes visible to the next pass
}

template <class R, int LOG2L, int PASS, int NS>
__device__ __forceinline__ void fft_passes(Cx<R>* x, R* sre, R* sim, const Cx<R>* __restrict__ tw, int t, int g) {
    using S = Shape<R, LOG2L>;
    constexpr int RX = (PASS == 0) ? S::R0 : S::EMAX;
    constexpr bool LAST = (PASS == S::P - 1);
    stockham_pass<R, LOG2L, RX, NS, PASS == 0, LAST>(x, sre, sim, tw, t, g);
    if constexpr (!LAST) fft_passes<R, LOG2L, PASS + 1, NS * RX>(x, sre, sim, tw, t, g);
}

// In-place unnormalised inverse DFT (sign +) of length L held in the t + T e layout.  The
// caller guarantees that nobody still reads the shared buffer when this is entered.
template <class R, int LOG2L>
__device__ __forceinline__ void fft(Cx<R>* x, R* sre, R* sim, const Cx<R>* __restrict__ tw, int t, int g) {
    fft_passes<R, LOG2L, 0, 1>(x, sre, sim, tw, t, g);
}

// ------------------------------------------------------------------ kernels
// CTAs of 1024 threads get at most 64 registers a thread: those instances keep the fibre's
// input in shared memory and read the bins from the (L1-resident) table instead of holding
// both in registers.
template <class R, int LOG2L>
struct Lean {
    static constexpr bool value = Shape<R, LOG2L>::THREADS >= 1024;
};

// Double-word sweeps of length 16..512 without a rank split stream each rank term's v_k (L)
// and u_k (n) into shared memory with bulk copies, one term ahead: at 16 bytes an entry the
// tables of a few rank terms already exceed what L1 keeps, and the loads right before use
// waited on L2.
template <class R, int LOG2L, bool SPLIT>
struct DwStream {
    static constexpr bool value = sizeof(R) == 8 && !SPLIT && LOG2L >= 4 && LOG2L <= 9;
};

template <class R, int LOG2L, bool SPLIT = false>
constexpr size_t axis_smem_bytes() {
    using S = Shape<R, LOG2L>;
    const size_t base =
        sizeof(R) * (size_t)S::G * S::GSTRIDE + (TwSmem<R, LOG2L>::value ? sizeof(Cx<R>) * (size_t)S::L : 0);
    // streamed slices: two of 2 L complex (v_k, then u_k), 16-byte aligned, two mbarriers, and
    // a copy of the bin pointers (L/2 + 2 ints) for the adjoint's scatter
    return DwStream<R, LOG2L, SPLIT>::value
               ? ((base + 15) & ~(size_t)15) + 2 * 2 * sizeof(Cx<R>) * (size_t)S::L + 16 + 4 * ((size_t)S::L / 2 + 2)
               : base;
}

// CTAs of 256 threads are held to 128 registers a thread, so that two of them fit an SM.
template <class R, int LOG2L, bool FWD, bool SPLIT = false>
__global__ void __launch_bounds__(Shape<R, LOG2L>::THREADS, (Shape<R, LOG2L>::THREADS <= 256) ? 2 : 1)
    axis_kernel(AxisDev A, const typename RealOps<R>::io* in, typename RealOps<R>::io* out, long long nfib,
                long long inner) {
    using S = Shape<R, LOG2L>;
    using IO = typename RealOps<R>::io;
    constexpr int L = S::L, E = S::E, T = S::T, G = S::G;
    constexpr bool LEAN = Lean<R, LOG2L>::value;
    constexpr int EV = LEAN ? 1 : E;  // register copies of the input
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* smem = reinterpret_cast<R*>(smem_raw);
    const int g = threadIdx.x / T;
    const int t = threadIdx.x % T;
    // per group: FFT buffer (2 PADL reals), then an auxiliary buffer of L reals
    R* sre = smem + (size_t)g * S::GSTRIDE;
    R* sim = sre + S::PADL;
    R* aux = sre + 2 * S::PADL;
    const XBuf<R> xb{sre, sim};

    const int n = A.n, nu0 = A.nu0, rank = A.rank;
    const Cx<R>* __restrict__ vtab = reinterpret_cast<const Cx<R>*>(A.vtab);
    const Cx<R>* __restrict__ utab = reinterpret_cast<const Cx<R>*>(A.utab);
    const R* __restrict__ vblk = reinterpret_cast<const R*>(A.vblk);
    const Cx<R>* tw = reinterpret_cast<const Cx<R>*>(A.twid);
    if constexpr (TwSmem<R, LOG2L>::value) {
        // per pass of span NS (NS = R0, 8 R0, .. < L, radix 8 after the first pass) the twiddles
        // w_L^{r k L / (8 NS)}, r = 1..7, k < NS, at [NS - R0 + (r - 1) NS + k]: the lanes of a
        // pass read consecutive k, so the reads of a quarter-warp hit different banks
        Cx<R>* tws = reinterpret_cast<Cx<R>*>(smem + (size_t)G * S::GSTRIDE);
        if constexpr (TwPass<R, LOG2L>::value) {
            for (int i = threadIdx.x; i < L - S::R0; i += S::THREADS) tws[i] = tw[i];
        } else {
            for (int ns = S::R0; ns < L; ns *= S::EMAX)
                for (int i = threadIdx.x; i < (S::EMAX - 1) * ns; i += S::THREADS) {
                    const int r = 1 + i / ns, k = i % ns;
                    tws[ns - S::R0 + i] = tw[((r * k) * (L / (ns * S::EMAX))) & (L - 1)];
                }
        }
        __syncthreads();
        tw = tws;
    }
    const long long ntiles = (nfib + G - 1) / G;
    const unsigned csize = SPLIT ? cluster_size() : 1u, crank = SPLIT ? cluster_rank() : 0u;
    const int kb = (int)(((long long)rank * crank) / csize), ke = (int)(((long long)rank * (crank + 1)) / csize);
    // degrees of the dense block this CTA adds: its share of 0..nu0-1 (all of them without a
    // rank split), so that no CTA of a cluster waits for one that does the whole block
    const int cb0 = (int)(((long long)nu0 * crank) / csize), cb1 = (int)(((long long)nu0 * (crank + 1)) / csize);
    const long long cfirst = SPLIT ? (long long)cluster_index() : (long long)blockIdx.x;
    const long long cstep = SPLIT ? (long long)cluster_count() : (long long)gridDim.x;

    // Streamed tables (DwStream): slice i (the i-th rank term this CTA applies, over all of its
    // tiles) holds v_k then u_k, goes to buffer i & 1 and completes the ((i >> 1) + 1)-th phase
    // of that buffer's mbarrier.  Thread 0 issues slice i + 1 once every thread has passed the
    // barrier after slice i's wait, so nobody still reads the buffer it overwrites.
    constexpr bool STREAM = DwStream<R, LOG2L, SPLIT>::value;
    Cx<R>* tsl = nullptr;
    unsigned long long* tbar = nullptr;
    const int* bin_ptr = A.bin_ptr;
    unsigned long long nslices = 0, slice = 0;
    if constexpr (STREAM) {
        const size_t off = (axis_smem_bytes<R, LOG2L, true>() + 15) & ~(size_t)15;
        tsl = reinterpret_cast<Cx<R>*>(smem_raw + off);
        tbar = reinterpret_cast<unsigned long long*>(tsl + 4 * L);
        if constexpr (!FWD) {
            int* sbp = reinterpret_cast<int*>(tbar + 2);
            for (int i = threadIdx.x; i < L / 2 + 2; i += S::THREADS) sbp[i] = __ldg(A.bin_ptr + i);
            bin_ptr = sbp;  // read by the adjoint's scatter after the barrier below
        }
        if (cfirst < ntiles && ke > kb)
            nslices = (unsigned long long)((ntiles - cfirst + cstep - 1) / cstep) * (unsigned long long)(ke - kb);
        if (threadIdx.x == 0) {
            mbar_init(tbar, 1);
            mbar_init(tbar + 1, 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
    }
    auto issue_slice = [&](unsigned long long i) {
        const int k = kb + (int)(i % (unsigned long long)(ke - kb));
        Cx<R>* dst = tsl + (i & 1) * (2 * L);
        unsigned long long* bar = tbar + (i & 1);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        // forward: u_k in point order (n entries); adjoint: the bin-ordered copy (L entries)
        const unsigned vb = (unsigned)(sizeof(Cx<R>) * L), ub = (unsigned)(sizeof(Cx<R>) * (FWD ? n : L));
        mbar_expect_tx(bar, vb + ub);
        bulk_g2s(dst, vtab + (size_t)k * L, vb, bar);
        bulk_g2s(dst + L, FWD ? utab + (size_t)k * n : reinterpret_cast<const Cx<R>*>(A.ubtab) + (size_t)k * L, ub, bar);
    };
    // wait for this term's slice (bounded), then fetch the next; false if the wait ran out
    auto next_slice = [&](const Cx<R>*& vk, const Cx<R>*& uk) -> bool {
        const bool ok = mbar_wait(tbar + (slice & 1), (unsigned)((slice >> 1) & 1));
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0 && A.status) atomicOr(A.status, 1u);
            return false;
        }
        if (threadIdx.x == 0 && slice + 1 < nslices) issue_slice(slice + 1);
        vk = tsl + (slice & 1) * (2 * L);
        uk = vk + L;
        ++slice;
        return true;
    };
    if constexpr (STREAM) {
        if (threadIdx.x == 0 && nslices > 0) issue_slice(0);
    }

    // BinOrd adjoint: whether one of this thread's bins holds more than two points
    bool binx = false;
    if constexpr (BinOrd<R, LOG2L>::value && !FWD) binx = __ldg(A.ovftab + 2 * t) != 0;
    int mj[LEAN ? 1 : E];  // forward: bins of the owned output points
    if constexpr (FWD && !LEAN) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
            int j = t + T * e;
            mj[e] = (j < n) ? __ldg(A.mtab + j) : 0;
        }
    }

    for (long long tile = cfirst; tile < ntiles; tile += cstep) {
        const long long f = tile * G + g;
        const bool valid = f < nfib;
        const long long o = valid ? f / inner : 0;
        const long long q = valid ? f - o * inner : 0;
        const long long base = o * (long long)n * inner + q;

        R val[EV];  // alpha (forward) or g (adjoint) at elements t + T e (LEAN: in aux)
        group_sync<T, G>(g);  // the previous tile is done with aux
#pragma unroll
        for (int e = 0; e < E; ++e) {
            int i = t + T * e;
            R v = (valid && i < n) ? RealOps<R>::from_io(in[base + (long long)i * inner]) : RealOps<R>::zero();
            if constexpr (LEAN)
                aux[i] = v;
            else
                val[e] = v;
        }
        R acc[E];
#pragma unroll
        for (int e = 0; e < E; ++e) acc[e] = RealOps<R>::zero();

        if constexpr (FWD) {
            // low-degree coefficients for the dense block, shared across the group
            if constexpr (!LEAN) {
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    int i = t + T * e;
                    if (i < nu0) aux[i] = val[e];
                }
            }
            group_sync<T, G>(g);
            for (int k = kb; k < ke; ++k) {
                Cx<R> x[E];
                const Cx<R>* vk = vtab + (size_t)k * L;
                const Cx<R>* uk = utab + (size_t)k * n;
                if constexpr (STREAM)
                    if (!next_slice(vk, uk)) return;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    if constexpr (LEAN)
                        x[e] = cscale(vk[t + T * e], aux[t + T * e]);
                    else
                        x[e] = cscale(vk[t + T * e], val[e]);
                }
                group_sync<T, G>(g);  // previous gather done with the buffer
                fft<R, LOG2L>(x, sre, sim, tw, t, g);
                group_sync<T, G>(g);  // last pass done reading the buffer
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    int m = t + T * e;
                    if (m <= L / 2) xb.template put<S>(m, x[e]);
                }
                group_sync<T, G>(g);
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    int j = t + T * e;
                    if (j < n) {
                        const int m = LEAN ? __ldg(A.mtab + j) : mj[e];
                        const Cx<R> y = xb.template get<S>(m);
                        acc[e] = acc[e] + re_mul(uk[j], y);
                    }
                }
            }
            // dense block: acc_j += sum_{c < nu0} sqrt(w_j) P~_c(t_j) alpha_c (a rank-split
            // cluster shares the degrees out over its CTAs; the partial sums are added anyway)
            {
#pragma unroll 4
                for (int c = cb0; c < cb1; ++c) {
                    R ac = aux[c];
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        int j = t + T * e;
                        if (j < n) acc[e] = acc[e] + vblk[(size_t)c * n + j] * ac;
                    }
                }
            }
        } else {
            // adjoint: g of the fibre in shared memory for the bin scatter
            if constexpr (!LEAN) {
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    int j = t + T * e;
                    if (j < n) aux[j] = val[e];
                }
            }
            group_sync<T, G>(g);
            // BinOrd: g at the first two points of each bin m = t + T e of the table's slots,
            // from the bin-ordered point table (-1: none), held for the whole tile unless LEAN
            constexpr bool BINORD = BinOrd<R, LOG2L>::value;
            constexpr int NSLT = BinOrd<R, LOG2L>::SLOTS;
            R gb[(BINORD && !LEAN && NSLT > 0) ? 2 * NSLT : 1];
            if constexpr (BINORD && !LEAN) {
#pragma unroll
                for (int q = 0; q < 2 * NSLT; ++q) {
                    const int j = __ldg(A.bjtab + q * T + t);
                    gb[q] = (j >= 0) ? aux[j] : RealOps<R>::zero();
                }
            }
            for (int k = kb; k < ke; ++k) {
                const Cx<R>* uk = utab + (size_t)k * n;
                const Cx<R>* vk = vtab + (size_t)k * L;
                if constexpr (STREAM)
                    if (!next_slice(vk, uk)) return;
                Cx<R> x[E];
                if constexpr (BINORD) {
                    // z[m] = u_k g at the bin's first two points (u_k in bin order, so that no
                    // load waits on another; streamed: the slice holds this table), plus, on the
                    // threads flagged for it, the rest of the bin (and the bin L/2 when the table
                    // has no slot for it) from the CSR lists
                    const Cx<R>* ubk = STREAM ? uk : reinterpret_cast<const Cx<R>*>(A.ubtab) + (size_t)k * (2 * NSLT * T);
                    const Cx<R>* ukg = utab + (size_t)k * n;
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        Cx<R> z{RealOps<R>::zero(), RealOps<R>::zero()};
                        if (e < NSLT) {
                            const Cx<R> u0 = ubk[(2 * e) * T + t], u1 = ubk[(2 * e + 1) * T + t];
                            R g0, g1;
                            if constexpr (LEAN) {
                                const int j0 = __ldg(A.bjtab + (2 * e) * T + t), j1 = __ldg(A.bjtab + (2 * e + 1) * T + t);
                                g0 = (j0 >= 0) ? aux[j0] : RealOps<R>::zero();
                                g1 = (j1 >= 0) ? aux[j1] : RealOps<R>::zero();
                            } else {
                                g0 = gb[2 * e];
                                g1 = gb[2 * e + 1];
                            }
                            z = bf_add(cscale(u0, g0), cscale(u1, g1));
                        }
                        if (binx) {
                            const int m = t + T * e;
                            if (m <= L / 2) {
                                const int p2 = bin_ptr[m + 1];
                                for (int p = bin_ptr[m] + (e < NSLT ? 2 : 0); p < p2; ++p) {
                                    const int j = A.sorted ? p : __ldg(A.bin_idx + p);
                                    z = bf_add(z, cscale(ukg[j], aux[j]));
                                }
                            }
                        }
                        x[e] = z;
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        int m = t + T * e;
                        Cx<R> z{RealOps<R>::zero(), RealOps<R>::zero()};
                        if (m <= L / 2) {
                            int p1 = bin_ptr[m], p2 = bin_ptr[m + 1];
                            for (int p = p1; p < p2; ++p) {
                                const int j = A.sorted ? p : __ldg(A.bin_idx + p);  // sorted: identity
                                z = bf_add(z, cscale(uk[j], aux[j]));
                            }
                        }
                        x[e] = z;
                    }
                }
                group_sync<T, G>(g);  // previous FFT done with the buffer
                fft<R, LOG2L>(x, sre, sim, tw, t, g);
#pragma unroll
                for (int e = 0; e < E; ++e) acc[e] = acc[e] + re_mul(vk[t + T * e], x[e]);
            }
            // dense block: alpha_c = sum_j sqrt(w_j) P~_c(t_j) g_j for c < nu0 (a rank-split
            // cluster shares the degrees out over its CTAs), DB degrees at a time: every thread's partial sums over its points go to
            // red[i][t] in the group's FFT buffer (DB T <= 2 PADL reals), a tree over t adds them
            // up with log2 T barriers for all DB degrees together, and element c is owned by
            // thread c % T at e = c / T.  Groups of 512 or more threads take 8 degrees at a time
            // (fewer barriers of the whole CTA); smaller groups one (more degrees at a time cost
            // them registers and occupancy).
            {
                constexpr int DB0 = (T >= 512) ? 8 : 1;
                constexpr int DB = (2 * S::PADL / T < DB0) ? 2 * S::PADL / T : DB0;
                static_assert(DB >= 1 && DB * T <= 2 * S::PADL, "dense-block partials fit the FFT buffer");
                R* red = sre;
                for (int c0 = cb0; c0 < cb1; c0 += DB) {
                    R part[DB];
#pragma unroll
                    for (int i = 0; i < DB; ++i) part[i] = RealOps<R>::zero();
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        const int j = t + T * e;
                        if (j < n) {
                            const R gj = LEAN ? aux[j] : val[e];
#pragma unroll
                            for (int i = 0; i < DB; ++i)
                                if (c0 + i < cb1) part[i] = part[i] + vblk[(size_t)(c0 + i) * n + j] * gj;
                        }
                    }
                    group_sync<T, G>(g);  // the buffer is free (last FFT pass, previous degrees)
#pragma unroll
                    for (int i = 0; i < DB; ++i) red[i * T + t] = part[i];
                    group_sync<T, G>(g);
                    for (int s = T / 2; s > 0; s >>= 1) {
                        if (t < s) {
#pragma unroll
                            for (int i = 0; i < DB; ++i) red[i * T + t] = red[i * T + t] + red[i * T + t + s];
                        }
                        group_sync<T, G>(g);
                    }
#pragma unroll
                    for (int i = 0; i < DB; ++i) {
                        const int c = c0 + i;
                        if (c < cb1) {
                            const R tot = red[i * T];
#pragma unroll
                            for (int e = 0; e < E; ++e)
                                if (t + T * e == c) acc[e] = tot;
                        }
                    }
                }
            }
        }
        if (!SPLIT || csize == 1) {
            if (valid) {
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    int j = t + T * e;
                    if (j < n) out[base + (long long)j * inner] = RealOps<R>::to_io(acc[e]);
                }
            }
        } else {
            // partial sums of the cluster's CTAs: [G][L + 1] over the group buffers, then CTA
            // crank adds up and stores its share of the tile's G x L elements
            constexpr int LP = L + 1;
            R* red = smem;
            __syncthreads();  // every group is done with its buffers
#pragma unroll
            for (int e = 0; e < E; ++e) red[g * LP + t + T * e] = acc[e];
            cluster_sync();
            const int per = (G * L) / (int)csize;
            for (int i = threadIdx.x; i < per; i += S::THREADS) {
                const int el = (int)crank * per + i;
                // strided axes: fibres fastest, so that neighbouring threads store neighbours
                const int fib = (inner > 1) ? el % G : el / L;
                const int j = (inner > 1) ? el / G : el % L;
                const long long ff = tile * G + fib;
                if (j < n && ff < nfib) {
                    R v = RealOps<R>::zero();
                    for (unsigned r = 0; r < csize; ++r) v = v + ld_cluster_r<R>(red + fib * LP + j, r);
                    const long long oo = ff / inner, qq = ff - oo * inner;
                    out[oo * (long long)n * inner + qq + (long long)j * inner] = RealOps<R>::to_io(v);
                }
            }
            cluster_sync();  // the peers are done reading before the buffers are reused
        }
    }
}


}  // namespace dev
}  // namespace jt
