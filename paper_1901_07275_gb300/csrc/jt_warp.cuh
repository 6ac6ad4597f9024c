// Fused axis kernel for FFT lengths L = 16 T, T in {1, 2, .., 256} (L = 16 .. 4096), FP32.
// One group of T lanes owns one fibre: a warp holds 32 / T fibres for T <= 32, a fibre
// spans T / 32 warps for T >= 64.
//
// The length-L inverse DFT (sign +) is split in four steps, L = 16 x T: with input index
// p = t + T s (lane t < T holds s = 0..15 in registers) and output index m = k1 + 16 k2,
//     Y[k1 + 16 k2] = sum_t w_T^{t k2} * ( w_L^{t k1} * sum_s x[t + T s] w_16^{s k1} ).
// Step A (a 16-point DFT over s) and the twiddle w_L^{t k1} stay in registers -- the 15
// twiddles of a lane never change, so they are loaded once per kernel.  One exchange
// through shared memory regroups the values by k1, and step B finishes the T-point DFTs:
// for T <= 16 each lane owns 16/T whole problems; for T = 32 each problem is split over a
// lane pair (16-point DFTs on the even and odd lanes, then one radix-2 stage through a
// shuffle); for T >= 64 over R = T/16 lanes (16-point DFTs, a second exchange, R-point DFTs).
// The forward keeps only the outputs m <= L/2 that the gather can use.
//
// Fibres of a strided axis are staged through a shared-memory tile so that every global
// load and store touches whole 32-byte sectors.
#pragma once

#include "jt_axis.cuh"

// CTAs per SM the register allocation is sized for (2 => at most 128 registers a thread).
#ifndef JT_WARP_MINB
#define JT_WARP_MINB 2
#endif

namespace jt {
namespace dev {

template <int LOG2L>
struct WShape {
    static constexpr int L = 1 << LOG2L;
    static constexpr int E = 16;
    static constexpr int T = L / E;          // lanes per fibre (1 .. 256)
    static constexpr int WARPS = 8;
    static constexpr int THREADS = 32 * WARPS;
    static constexpr int FT = THREADS / T;   // fibres per CTA iteration
    static constexpr int R = (T >= 64) ? T / 16 : 1;  // T >= 64: lanes per step-B problem
    static constexpr int QP = 16 / R;                 // T >= 64: k2' values a lane finishes
    // Exchange rows are padded so that the 64-bit accesses of a half-warp never share a bank:
    // row k1 starts at k1 * XROW float2.  T = 32 reads (k1 = t/2, column 2q + h) need an even
    // pad, T <= 16 reads (k1 = t) an odd one, T >= 64 reads (k1 = t/R, column R q + h) R.
    static constexpr int XROW = (T == 32) ? T + 2 : (T >= 64) ? T + R : T + 1;
    static constexpr int XBUF = 16 * XROW;   // exchange buffer per fibre (float2)
    static constexpr int X2BUF = (T >= 64) ? 16 * 16 * R : 0;      // second exchange (T >= 64)
    static constexpr int YBUF = L / 2 + 1 + ((L / 2) >> 4) + 1;  // gather buffer (float2)
    static constexpr int BUF0 = (XBUF > YBUF ? XBUF : YBUF);
    static constexpr int BUF = (BUF0 > X2BUF ? BUF0 : X2BUF);
    static constexpr int AUX = L + L / 32 + 1;                  // per fibre: alpha_V / g (floats)
    // T >= 64: the step-A twiddles w_L^{t k1} for k1 = 1, 2, 4, 8 live in shared memory,
    // [log2 k1][t], then the step-B twiddles w_T^{h k2} for k2 = 1, 2, 4, 8 at [4 T + log2 k2][h];
    // the other powers are formed from them (apply_powers15)
    static constexpr int TWS = (T >= 64) ? 4 * T + 4 * R : 0;  // float2
    // staging tile rows: consecutive threads cover FT fibres x (32 / FT) rows
    static constexpr int TROW = L + ((FT >= 32) ? 1 : 32 / FT);
    // gather buffer index: a half-warp writes runs m0 + [0, 8) and m0 + 128 + [0, 8)
    static __host__ __device__ constexpr int ypad(int m) { return m + (m >> 4); }
    // adjoint copy of g: lanes read points ~2t (stride 2) in the scatter and consecutive
    // points in the dense block; j + j/32 keeps both patterns free of bank conflicts
    static __host__ __device__ constexpr int apad(int j) { return j + (j >> 5); }
    // second exchange (T >= 64): B_h[k2'] of problem k1, rotated within its R-group so that the
    // reads of a half-warp (different k1, h, rows k2' = h QP + i) hit different banks
    static __host__ __device__ constexpr int x2idx(int k1, int k2, int h) {
        return k2 * (16 * R) + k1 * R + ((h + k2 / QP) % R);
    }
};

// Element offset of fibre f = (o, q), o = f / inner, q = f % inner, of an array whose axis of
// length n has stride inner: o n inner + q.  32-bit division when the operands allow it.
__device__ __forceinline__ long long fibre_offset(long long f, int n, long long inner) {
    if (((unsigned long long)f | (unsigned long long)inner) < 0x100000000ull) {
        const unsigned o = (unsigned)f / (unsigned)inner;
        const unsigned q = (unsigned)f - o * (unsigned)inner;
        return (long long)o * ((long long)n * inner) + q;
    }
    const long long o = f / inner;
    return o * ((long long)n * inner) + (f - o * inner);
}

// Synchronise the T lanes of one fibre group (a warp or less, one CTA, or a named barrier).
template <int T, int FT>
__device__ __forceinline__ void gsync(int fl) {
    if constexpr (T <= 32) {
        __syncwarp();
    } else if constexpr (FT == 1) {
        __syncthreads();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(fl + 1), "r"(T) : "memory");
    }
}

// Input staging buffers: two (the next tile's input is fetched during this tile's rank
// terms) unless that would leave room for only one CTA an SM.
// Contiguous fibres are loaded straight into registers and need none.
template <int LOG2L, bool STRIDED>
constexpr int warp_nstage() {
    using S = WShape<LOG2L>;
    if (!STRIDED) return 0;
    return ((size_t)S::FT * (S::BUF * 8 + S::AUX * 4) + (size_t)S::TWS * 8 + 2 * (size_t)S::FT * S::TROW * 4 <=
            112 * 1024)
               ? 2
               : 1;
}
// Layout: exchange buffers [FT][BUF] float2, step-A twiddles [TWS] float2, fibre copies
// [FT][AUX] float, staging buffers [NSTAGE][FT][TROW] float.
template <int LOG2L>
constexpr size_t warp_smem_bytes(bool strided, bool stream = false) {
    using S = WShape<LOG2L>;
    const int ns = strided ? warp_nstage<LOG2L, true>() : 0;
    const size_t base = (size_t)S::FT * (S::BUF * 8 + S::AUX * 4) + (size_t)S::TWS * 8 + (size_t)ns * S::FT * S::TROW * 4;
    // streamed rank tables: two slices of 34 T float2 (16-byte aligned) and two mbarriers
    return stream ? ((base + 15) & ~(size_t)15) + 2 * (size_t)34 * S::T * 8 + 16 : base;
}

// Single (not batched, not rank-split) forward sweeps of length up to 512 stream the rank
// tables of each term, v_k (L) and the bin-ordered u_k (18 T), into shared memory with bulk
// copies, one term ahead, instead of reading them through L1 right before use.  (The adjoint
// path can stream its bin-ordered u_k and lane-ordered v_k the same way, but the extra
// pointers spilled it and it measured slower, so it keeps the L1 loads.)
template <int LOG2L, bool FWD, bool BATCHED, bool SPLIT>
struct WStream {
    static constexpr bool value = FWD && !BATCHED && !SPLIT && LOG2L <= 9;
    static constexpr int SL = 34 * WShape<LOG2L>::T;  // float2 a slice
};

// Asynchronous 4-byte global -> shared copy (zero-filled when !valid; src must still be a
// mapped address), and the group commit / wait of the issuing thread.
__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(valid ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

__device__ __forceinline__ float2 f2(Cx<float> c) { return make_float2(c.re, c.im); }
__device__ __forceinline__ Cx<float> cx(float2 v) { return Cx<float>{v.x, v.y}; }

// Output ownership after step B.  Forward keeps m <= L/2; adjoint keeps all L.
template <int LOG2L, bool FWD>
struct Own {
    using S = WShape<LOG2L>;
    static constexpr int T = S::T;
    // number of outputs a lane holds
    static constexpr int NOUT = (T == 32) ? 16 : 16;
    // index of output slot o of lane t
    static __host__ __device__ __forceinline__ int idx(int t, int o) {
        if constexpr (T == 32) {
            const int k1 = t >> 1, h = t & 1;
            return k1 + 16 * (h * 8 + (o & 7)) + (o >> 3) * (S::L / 2);  // o < 8: g = 0, o >= 8: g = 1
        } else if constexpr (T >= 64) {
            const int k1 = t / S::R, h = t % S::R;
            const int i = o / S::R, g = o % S::R;
            return k1 + 16 * (h * S::QP + i + 16 * g);
        } else {
            constexpr int P = 16 / T;  // problems per lane
            const int q = o / T, k2 = o % T;
            return (t * P + q) + 16 * k2;
        }
    }
};

// Forward with at most two points a bin: the outputs a lane keeps after step B are the bins
// Own(t, fslot(c)), c = 0..8: slots 0..7 lie at or below L/2 for every lane, slot 8 only on
// lane 0 (bin L/2).  Together they cover the bins 0..L/2 once, so each lane accumulates the
// points of its own bins and no gather through shared memory is needed.
template <int LOG2L>
__host__ __device__ constexpr int fslot(int c) {
    using S = WShape<LOG2L>;
    if (S::T == 1) return c;
    if (S::T <= 16) return (c < 8) ? (c / (S::T / 2)) * S::T + c % (S::T / 2) : S::T / 2;
    if (S::T == 32) return c;
    return (c < 8) ? (c / (S::R / 2)) * S::R + c % (S::R / 2) : S::R / 2;
}

// x[k] *= w^k for k = 1..15, with w^k read from a table only for k = 1, 2, 4, 8 (at
// tab[log2(k) stride]) and the other eleven powers formed as products of two of those (or of
// earlier products): 4 shared-memory reads and 11 extra complex products instead of 15 reads.
// Each derived power carries at most three table roundings and two product roundings.
__device__ __forceinline__ void apply_powers15(Cx<float>* x, const float2* tab, int stride) {
    const Cx<float> w1 = cx(tab[0]), w2 = cx(tab[stride]), w4 = cx(tab[2 * stride]), w8 = cx(tab[3 * stride]);
    x[1] = cmul(x[1], w1);
    x[2] = cmul(x[2], w2);
    x[4] = cmul(x[4], w4);
    x[8] = cmul(x[8], w8);
    const Cx<float> w3 = cmul(w1, w2), w5 = cmul(w1, w4), w6 = cmul(w2, w4);
    x[3] = cmul(x[3], w3);
    x[5] = cmul(x[5], w5);
    x[6] = cmul(x[6], w6);
    x[9] = cmul(x[9], cmul(w1, w8));
    x[10] = cmul(x[10], cmul(w2, w8));
    x[12] = cmul(x[12], cmul(w4, w8));
    const Cx<float> w7 = cmul(w3, w4);
    x[7] = cmul(x[7], w7);
    x[11] = cmul(x[11], cmul(w3, w8));
    x[13] = cmul(x[13], cmul(w5, w8));
    x[14] = cmul(x[14], cmul(w6, w8));
    x[15] = cmul(x[15], cmul(w7, w8));
}

// Sum CNT values per lane over the lanes of a group (xor offsets OFF, OFF/2, .., 1) so that
// each lane keeps a share: at every step the lanes with that offset bit set keep the upper
// half of their live values and add the partner's copy of it, so after log2(CNT) steps lane u
// holds the total of output base(u) (further steps, if any, are plain pairwise sums).
template <int OFF, int CNT>
__device__ __forceinline__ void transpose_reduce(float* v, int u, int& base) {
    if constexpr (OFF >= 1) {
        if constexpr (CNT > 1) {
            constexpr int H = CNT / 2;
            const bool upper = (u & OFF) != 0;
#pragma unroll
            for (int i = 0; i < H; ++i) {
                const float send = upper ? v[i] : v[i + H];
                const float keep = upper ? v[i + H] : v[i];
                v[i] = keep + __shfl_xor_sync(0xffffffffu, send, OFF);
            }
            if (upper) base += H;
            transpose_reduce<OFF / 2, H>(v, u, base);
        } else {
            v[0] += __shfl_xor_sync(0xffffffffu, v[0], OFF);
            transpose_reduce<OFF / 2, 1>(v, u, base);
        }
    }
}

// One sweep of one axis of one transform, as an entry of a batched launch: the CTA tiles of
// all jobs of a launch are numbered consecutively, job i owning [tile_begin, tile_begin + tiles).
// The job tables are built once per batch; the caller's array pointers of one launch travel as
// a by-value kernel parameter (BatchPtrs), so a launch needs no host-to-device copy.
constexpr int BATCH_MAX_JOBS = 256;
struct BatchJob {
    AxisDev A;
    long long nfib, inner, tile_begin;
    int slot;  // index into BatchPtrs
};
struct BatchPtrs {
    const float* in[BATCH_MAX_JOBS];
    float* out[BATCH_MAX_JOBS];
};

// One forward or adjoint sweep over nfib fibres (see jt_axis.cuh for the operator).  With
// BATCHED, the kernel walks the concatenated tiles of njobs jobs instead (same arithmetic;
// the per-job constants are reloaded when a CTA moves on to the next job).
template <int LOG2L, bool FWD, bool STRIDED, bool BATCHED = false, bool SPLIT = false>
__global__ void __launch_bounds__(WShape<LOG2L>::THREADS, JT_WARP_MINB)
    warp_axis_kernel(AxisDev A, const float* in, float* out, long long nfib, long long inner,
                     const BatchJob* __restrict__ jobs, int njobs, long long total_tiles, const __grid_constant__ BatchPtrs ptrs) {
    using S = WShape<LOG2L>;
    constexpr int L = S::L, T = S::T, FT = S::FT;
    constexpr bool VAL_SMEM = FWD && T >= 128;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int fl = threadIdx.x / T;  // fibre slot in the CTA tile
    const int t = threadIdx.x % T;
    float2* buf = reinterpret_cast<float2*>(smem_raw) + (size_t)fl * S::BUF;
    float2* twS = reinterpret_cast<float2*>(smem_raw) + (size_t)FT * S::BUF;
    float* const aux0 = reinterpret_cast<float*>(twS + S::TWS);
    float* aux = aux0 + (size_t)fl * S::AUX;
    // two staging buffers of FT x TROW floats (input of this tile and of the next one)
    float* stage = aux0 + (size_t)FT * S::AUX;
    // streamed rank-table slices [2][SL] and their two mbarriers (WStream instances)
    constexpr bool STREAM = WStream<LOG2L, FWD, BATCHED, SPLIT>::value;
    constexpr int SL = WStream<LOG2L, FWD, BATCHED, SPLIT>::SL;
    float2* tstream = nullptr;
    unsigned long long* tbar = nullptr;
    if constexpr (STREAM) {
        const size_t off = (warp_smem_bytes<LOG2L>(STRIDED, false) + 15) & ~(size_t)15;
        tstream = reinterpret_cast<float2*>(smem_raw + off);
        tbar = reinterpret_cast<unsigned long long*>(tstream + 2 * SL);
    }

    if constexpr (BATCHED) {
        if (njobs <= 0) return;
        A = jobs[0].A;  // replaced below by the job of the first tile
    }
    int n = A.n, nu0 = A.nu0, rank = A.rank;
    const float2* __restrict__ vtab = reinterpret_cast<const float2*>(A.vtab);
    const float2* __restrict__ utab = reinterpret_cast<const float2*>(A.utab);
    const float* __restrict__ vblk = reinterpret_cast<const float*>(A.vblk);  // [c][0..L), zero beyond n
    const float2* __restrict__ tw = reinterpret_cast<const float2*>(A.twid);
    const float2* __restrict__ ubtab = reinterpret_cast<const float2*>(A.ubtab);
    const float2* __restrict__ vown = reinterpret_cast<const float2*>(A.vown);
    const float2* __restrict__ fbtab = reinterpret_cast<const float2*>(A.fbtab);
    bool fbin = FWD && A.fbin != 0;

    // step-A twiddles w_L^{t k1}, k1 = 1..15: fixed per lane (they depend on L only)
    // (T >= 64: in shared memory instead, written here and first read after the barriers
    // that open every tile)
    constexpr bool TW_SMEM = S::TWS > 0;
    Cx<float> twA[TW_SMEM ? 1 : 16];
    if constexpr (TW_SMEM) {
        // [b][t] = w_L^{t 2^b}, then the step-B twiddles [4 T + b][h] = w_L^{16 h 2^b}, b < 4
        for (int i = threadIdx.x; i < 4 * T; i += S::THREADS) {
            const int k1 = 1 << (i / T), tt = i % T;
            twS[i] = __ldg(tw + ((tt * k1) & (L - 1)));
        }
        for (int i = threadIdx.x; i < 4 * S::R; i += S::THREADS) {
            const int k2 = 1 << (i / S::R), hh = i % S::R;
            twS[4 * T + i] = __ldg(tw + ((16 * hh * k2) & (L - 1)));
        }
    } else {
#pragma unroll
        for (int k1 = 1; k1 < 16; ++k1) twA[k1] = cx(__ldg(tw + ((t * k1) & (L - 1))));
    }
    // Per-lane constants of one job.  Forward: padded gather-buffer index of each owned point,
    // two 16-bit fields a word.  Adjoint: whether one of the lane's bins holds more than two points.
    constexpr int NPK = FWD ? 8 : 2;
    unsigned pk[NPK];
    bool sorted = false;
    auto load_job_constants = [&]() {
        n = A.n;
        nu0 = A.nu0;
        rank = A.rank;
        vtab = reinterpret_cast<const float2*>(A.vtab);
        utab = reinterpret_cast<const float2*>(A.utab);
        vblk = reinterpret_cast<const float*>(A.vblk);
        ubtab = reinterpret_cast<const float2*>(A.ubtab);
        vown = reinterpret_cast<const float2*>(A.vown);
        fbtab = reinterpret_cast<const float2*>(A.fbtab);
        fbin = FWD && A.fbin != 0;
#pragma unroll
        for (int i = 0; i < NPK; ++i) {
            if constexpr (FWD) {
                unsigned v[2] = {0u, 0u};
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int j = t + T * (2 * i + h);
                    if (j < n) v[h] = (unsigned)S::ypad(__ldg(A.mtab + j));
                }
                pk[i] = fbin ? 0u : (v[0] | (v[1] << 16));
            } else {
                pk[i] = (unsigned)__ldg(A.ovftab + 2 * t + i);
            }
        }
        sorted = A.sorted != 0;
    };
    int cur_job = -1;
    if constexpr (!BATCHED) load_job_constants();

    const long long ntiles = BATCHED ? total_tiles : (nfib + FT - 1) / FT;
    // rank split over the CTAs of a cluster (jt_axis.cuh); every CTA of a cluster walks the
    // same tiles, so all of them meet the same cluster barriers
    const unsigned csize = SPLIT ? cluster_size() : 1u, crank = SPLIT ? cluster_rank() : 0u;
    const long long cfirst = SPLIT ? (long long)cluster_index() : (long long)blockIdx.x;
    const long long cstep = SPLIT ? (long long)cluster_count() : (long long)gridDim.x;

    // Batched launches: the job of global tile gt (jobs are ordered by tile_begin and a CTA's
    // tiles increase, so a hint from an earlier tile only moves forward).
    auto find_job = [&](long long gt, int hint) -> int {
        int j = hint;
        if (j < 0) {
            int lo = 0, hi = njobs - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (jobs[mid].tile_begin <= gt) lo = mid; else hi = mid - 1;
            }
            j = lo;
        }
        while (j + 1 < njobs && jobs[j + 1].tile_begin <= gt) ++j;
        return j;
    };
    // Strided axes: stage the input of global tile gt into dst ([FT][TROW]) with asynchronous
    // copies, so that the next tile's input arrives while this tile's rank terms run; thread
    // (ql, r0) walks rows r0, r0 + RSTEP, .. of fibre ql.
    int pf_job = -1;
    auto stage_tile = [&](long long gt, float* dst) {
        const float* src = in;
        long long nf = nfib, inr = inner, ti = gt;
        int nn = n;
        if constexpr (BATCHED) {
            pf_job = find_job(gt, pf_job);
            const BatchJob& J = jobs[pf_job];
            src = ptrs.in[J.slot];
            nf = J.nfib;
            inr = J.inner;
            nn = J.A.n;
            ti = gt - J.tile_begin;
        }
        const long long g0 = ti * FT;
        if constexpr (STRIDED) {
            const int ql = threadIdx.x % FT;
            const long long ff = g0 + ql;
            constexpr int RSTEP = S::THREADS / FT;
            const int r0 = threadIdx.x / FT;
            float* trow = dst + ql * S::TROW;
            if (ff < nf) {
                const float* p = src + fibre_offset(ff, nn, inr) + (long long)r0 * inr;
                const long long step = (long long)RSTEP * inr;
#pragma unroll 4
                for (int row = r0; row < nn; row += RSTEP, p += step) cp_async4(trow + row, p, true);
            } else {
                for (int row = r0; row < nn; row += RSTEP) cp_async4(trow + row, src, false);
            }
        }
        cp_async_commit();
    };

    // rank terms of this CTA (a rank-split cluster gives each CTA its share); batched launches
    // recompute them per job in the tile loop
    int kb = (int)(((long long)rank * crank) / csize);
    int ke = (int)(((long long)rank * (crank + 1)) / csize);
    // Streamed tables: slice i (the i-th term this CTA applies, over all its tiles) goes to
    // buffer i & 1 and completes the ((i >> 1) + 1)-th phase of that buffer's mbarrier.
    unsigned long long nslices = 0, slice = 0;
    auto issue_slice = [&](unsigned long long i) {
        const int k = kb + (int)(i % (unsigned long long)(ke - kb));
        float2* dst = tstream + (i & 1) * SL;
        unsigned long long* bar = tbar + (i & 1);
        // the buffer was last read by the generic proxy (every thread passed a barrier since)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if constexpr (FWD) {
            const unsigned vb = 8u * L, ub = fbin ? 8u * 18 * T : 0u;
            mbar_expect_tx(bar, vb + ub);
            if (A.skip_copy) return;
            bulk_g2s(dst, vtab + (size_t)k * L, vb, bar);
            if (fbin) bulk_g2s(dst + L, fbtab + (size_t)k * 18 * T, ub, bar);
        } else {
            mbar_expect_tx(bar, 8u * 34 * T);
            if (A.skip_copy) return;
            bulk_g2s(dst, ubtab + (size_t)k * 18 * T, 8u * 18 * T, bar);
            bulk_g2s(dst + 18 * T, vown + (size_t)k * 16 * T, 8u * 16 * T, bar);
        }
    };
    if constexpr (STREAM) {
        if (cfirst < ntiles && ke > kb)
            nslices = (unsigned long long)((ntiles - cfirst + cstep - 1) / cstep) * (unsigned long long)(ke - kb);
        if (threadIdx.x == 0) {
            mbar_init(tbar, 1);
            mbar_init(tbar + 1, 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
        if (threadIdx.x == 0 && nslices > 0) issue_slice(0);
    }

    constexpr int NSTAGE = warp_nstage<LOG2L, STRIDED>();
    int cur = 0;
    if (NSTAGE == 2 && cfirst < ntiles) stage_tile(cfirst, stage);
    for (long long g_tile = cfirst; g_tile < ntiles; g_tile += cstep, cur ^= (NSTAGE - 1)) {
        long long tile_i = g_tile;
        if constexpr (BATCHED) {
            const int j = find_job(g_tile, cur_job);
            if (j != cur_job) {
                A = jobs[j].A;
                in = ptrs.in[jobs[j].slot];
                out = ptrs.out[jobs[j].slot];
                nfib = jobs[j].nfib;
                inner = jobs[j].inner;
                load_job_constants();
                cur_job = j;
            }
            tile_i = g_tile - jobs[j].tile_begin;
        }
        const long long f0 = tile_i * FT;
        const long long f = f0 + fl;
        const bool valid = f < nfib;
        float* tile = stage + cur * (FT * S::TROW);
        float val[16];
        if constexpr (STRIDED) {
            if constexpr (NSTAGE == 1) {
                __syncthreads();  // the previous tile's output transpose is done
                stage_tile(g_tile, tile);
            }
            cp_async_wait_all();
            __syncthreads();  // rows staged by other threads
#pragma unroll
            for (int s2 = 0; s2 < 16; ++s2) {
                const int p = t + T * s2;
                val[s2] = (p < n) ? tile[fl * S::TROW + p] : 0.0f;
            }
            // the other buffer was last read by the previous tile (input and output
            // transpose), before the barrier above
            if (NSTAGE == 2 && g_tile + cstep < ntiles) stage_tile(g_tile + cstep, stage + (cur ^ 1) * (FT * S::TROW));
        } else {
            const long long base = f * (long long)n;
#pragma unroll
            for (int s2 = 0; s2 < 16; ++s2) {
                const int p = t + T * s2;
                val[s2] = (valid && p < n) ? in[base + p] : 0.0f;
            }
        }

        // forward with fbin: 18 partial sums in bin order (slot c, point i at 2c + i); otherwise
        // 16 in natural order (point t + T e at e)
        float acc[18];
        acc[16] = acc[17] = 0.0f;
        __syncthreads();  // the previous tile is done with aux and the exchange region
        if constexpr (FWD) {
            // lengths L >= 1024 keep the whole fibre here instead of in registers (it is
            // re-read by every rank term), which leaves room for the two-level step B
#pragma unroll
            for (int s = 0; s < 16; ++s) {
                int p = t + T * s;
                if (VAL_SMEM || p < nu0) aux[p] = val[s];
            }
        } else {
            // all L points, zero beyond n: the dense block multiplies the zero-padded table
            // rows by every entry, so none may be left unwritten
#pragma unroll
            for (int s = 0; s < 16; ++s) aux[S::apad(t + T * s)] = val[s];
        }
        __syncthreads();
        // Dense low-degree block for the whole tile at once, so that each row of the table
        // (vblk[c][0..L), zero beyond n) is read once per tile rather than once per fibre.
        // The exchange region is free until the rank loop and holds the results meanwhile.
        float* vres = reinterpret_cast<float*>(smem_raw);
        const float* __restrict__ auxbase =
            aux0;
        if (SPLIT && crank != 0) {
            // rank-split partners: the dense block belongs to the first CTA of the cluster
#pragma unroll
            for (int e = 0; e < 18; ++e) acc[e] = 0.0f;
        } else if constexpr (FWD) {
            // FT x L outputs, 16 per thread: JPT points x FPT fibres
            constexpr int JPT = (L > 256) ? L / 256 : 1;
            constexpr int FPT = 16 / JPT;
            constexpr int FSTEP = (L >= 256) ? 1 : 256 / L;
            const int j0 = threadIdx.x % (L < 256 ? L : 256);
            const int fb = (L >= 256) ? 0 : threadIdx.x / L;
            float part[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) part[i] = 0.0f;
#pragma unroll 4
            for (int c = 0; c < nu0; ++c) {
                float vj[JPT];
#pragma unroll
                for (int jj = 0; jj < JPT; ++jj) vj[jj] = __ldg(vblk + (size_t)c * L + j0 + 256 * jj);
#pragma unroll
                for (int ff = 0; ff < FPT; ++ff) {
                    const float a = auxbase[(size_t)(fb + FSTEP * ff) * S::AUX + c];
#pragma unroll
                    for (int jj = 0; jj < JPT; ++jj) part[ff * JPT + jj] = fmaf(vj[jj], a, part[ff * JPT + jj]);
                }
            }
#pragma unroll
            for (int ff = 0; ff < FPT; ++ff)
#pragma unroll
                for (int jj = 0; jj < JPT; ++jj) vres[(fb + FSTEP * ff) * L + j0 + 256 * jj] = part[ff * JPT + jj];
            __syncthreads();
            if (fbin) {
#pragma unroll
                for (int q = 0; q < 18; ++q) {
                    const int j = __ldg(A.bjf + q * T + t);
                    acc[q] = (j >= 0) ? vres[fl * L + j] : 0.0f;
                }
            } else {
#pragma unroll
                for (int e = 0; e < 16; ++e) acc[e] = vres[fl * L + t + T * e];
            }
        } else if constexpr (FT <= 2) {
            // alpha_c(fibre) = sum_j vblk[c][j] g_j with one or two fibres a tile (L >= 2048):
            // every thread takes L/256 points of each fibre and all degrees, so that its table
            // loads are independent of one another; a transposing butterfly leaves lane l of
            // each warp with the warp's sum for degree l, and the warps' sums are added last.
            constexpr int JPT = L / 256;
            float* wpart = vres + 2 * FT * 32;  // [warp][FT][32]
            float gv[FT][JPT];
#pragma unroll
            for (int ff = 0; ff < FT; ++ff)
#pragma unroll
                for (int jj = 0; jj < JPT; ++jj) gv[ff][jj] = auxbase[(size_t)ff * S::AUX + S::apad(threadIdx.x + 256 * jj)];
            float part[FT][32];
#pragma unroll
            for (int c = 0; c < 32; ++c) {
                float v[JPT];
#pragma unroll
                for (int jj = 0; jj < JPT; ++jj) v[jj] = (c < nu0) ? __ldg(vblk + (size_t)c * L + threadIdx.x + 256 * jj) : 0.0f;
#pragma unroll
                for (int ff = 0; ff < FT; ++ff) {
                    float a = 0.0f;
#pragma unroll
                    for (int jj = 0; jj < JPT; ++jj) a = fmaf(v[jj], gv[ff][jj], a);
                    part[ff][c] = a;
                }
            }
#pragma unroll
            for (int ff = 0; ff < FT; ++ff) {
                int base = 0;
                transpose_reduce<16, 32>(part[ff], lane, base);
                wpart[(warp * FT + ff) * 32 + base] = part[ff][0];
            }
            __syncthreads();
            if (threadIdx.x < FT * 32) {
                const int ff = threadIdx.x >> 5, c = threadIdx.x & 31;
                float tot = 0.0f;
#pragma unroll
                for (int w = 0; w < S::WARPS; ++w) tot += wpart[(w * FT + ff) * 32 + c];
                vres[ff * 32 + c] = tot;
                vres[(FT + ff) * 32 + c] = 0.0f;
            }
            __syncthreads();
#pragma unroll
            for (int o = 0; o < 16; ++o) {
                const int nu = Own<LOG2L, FWD>::idx(t, o);
                acc[o] = (nu < nu0) ? vres[fl * 32 + nu] : 0.0f;
            }
        } else {
            // alpha_c(fibre) = sum_j vblk[c][j] g_j with FT >= 4 fibres a tile, as a register-
            // blocked product: block (cb, fb) = degrees 4 cb .. 4 cb + 3 x fibres FB fb ..
            // FB fb + FB - 1 is owned by TPB consecutive lanes, lane u taking the points
            // j = u + TPB q; a transposing butterfly then sums each output over the TPB lanes.
            constexpr int CB = 4;
            constexpr int FB = (FT >= 256) ? 8 : 4;
            constexpr int NV = CB * FB;
            constexpr int NBLK = (32 / CB) * (FT / FB);
            constexpr int TPB = S::THREADS / NBLK;  // 1 .. 32
            constexpr int JR = L / TPB;
            static_assert(TPB >= 1 && TPB <= 32 && NBLK * TPB == S::THREADS, "dense-block blocking");
            const int blk = threadIdx.x / TPB, u = threadIdx.x % TPB;
            const int cb = blk % (32 / CB), fb = blk / (32 / CB);
            float v[NV];
#pragma unroll
            for (int i = 0; i < NV; ++i) v[i] = 0.0f;
            bool crow[CB];
#pragma unroll
            for (int i = 0; i < CB; ++i) crow[i] = CB * cb + i < nu0;
#pragma unroll 8
            for (int q = 0; q < JR; ++q) {
                const int j = u + TPB * q;
                float vv[CB], gg[FB];
#pragma unroll
                for (int i = 0; i < CB; ++i) vv[i] = crow[i] ? __ldg(vblk + (size_t)(CB * cb + i) * L + j) : 0.0f;
#pragma unroll
                for (int f = 0; f < FB; ++f) gg[f] = auxbase[(size_t)(FB * fb + f) * S::AUX + S::apad(j)];
#pragma unroll
                for (int i = 0; i < CB; ++i)
#pragma unroll
                    for (int f = 0; f < FB; ++f) v[i * FB + f] = fmaf(vv[i], gg[f], v[i * FB + f]);
            }
            // lane u ends with outputs base .. base + NV/TPB - 1 (TPB > NV: duplicated on lanes
            // that differ in the low bits; the one with those bits clear stores)
            int base = 0;
            transpose_reduce<TPB / 2, NV>(v, u, base);
            constexpr int KEEP = (NV / TPB > 0) ? NV / TPB : 1;
            constexpr int DUP = (TPB > NV) ? TPB / NV - 1 : 0;
            if ((u & DUP) == 0) {
#pragma unroll
                for (int i = 0; i < KEEP; ++i) {
                    const int o = base + i;
                    vres[(FB * fb + o % FB) * 32 + CB * cb + o / FB] = v[i];
                }
            }
            __syncthreads();
#pragma unroll
            for (int o = 0; o < 16; ++o) {
                const int nu = Own<LOG2L, FWD>::idx(t, o);
                acc[o] = (nu < nu0) ? vres[fl * 32 + nu] : 0.0f;
            }
        }
        __syncthreads();  // results read before the rank loop reuses the exchange region

        // adjoint: g at the first two points of each owned bin (s <= 8), zero where there is none
        float gb[FWD ? 1 : 18];
        if constexpr (!FWD) {
#pragma unroll
            for (int q = 0; q < 18; ++q) {
                const int j = __ldg(A.bjtab + q * T + t);
                gb[q] = (j >= 0) ? aux[S::apad(j)] : 0.0f;
            }
        }

        if constexpr (BATCHED) {
            kb = (int)(((long long)rank * crank) / csize);
            ke = (int)(((long long)rank * (crank + 1)) / csize);
        }
        for (int k = kb; k < ke; ++k) {
            // streamed tables: wait for this term's slice (bounded), then, with every thread
            // past the barrier and so done with the previous slice, fetch the next one into it
            const float2* tsv = nullptr;  // forward v_k (L) / adjoint bin-ordered u_k (18 T)
            const float2* tsu = nullptr;  // forward bin-ordered u_k (18 T) / adjoint lane-ordered v_k (16 T)
            if constexpr (STREAM) {
                const bool ok = mbar_wait(tbar + (slice & 1), (unsigned)((slice >> 1) & 1));
                if (__syncthreads_or(!ok)) {
                    if (threadIdx.x == 0) atomicOr(A.status, 1u);
                    return;  // every thread: nothing of this CTA is in flight but the late copy
                }
                if (threadIdx.x == 0 && slice + 1 < nslices) issue_slice(slice + 1);
                tsv = tstream + (slice & 1) * SL;
                tsu = FWD ? tsv + L : tsv + 18 * T;
                ++slice;
            }
            Cx<float> x[16];
            if constexpr (FWD) {
                const float2* vk = vtab + (size_t)k * L;
#pragma unroll
                for (int s = 0; s < 16; ++s) {
                    float2 v = STREAM ? tsv[t + T * s] : __ldg(vk + t + T * s);
                    const float a = VAL_SMEM ? aux[t + T * s] : val[s];
                    x[s] = Cx<float>{v.x * a, v.y * a};
                }
            } else {
                // z[m] = sum_{j : m_j = m} u_k[j] g_j for the owned bins m = t + T s; only
                // m <= L/2 (s <= 8) can hold points.  The first two points of every bin come
                // from the bin-ordered tables (u_k contiguous across lanes, g in registers);
                // lanes with a larger bin add the remaining points from the CSR lists.
                const float2* ubk = ubtab + (size_t)k * (18 * T);
#pragma unroll
                for (int s = 0; s < 16; ++s) {
                    Cx<float> z{0.0f, 0.0f};
                    if (s <= 8) {
                        const float2 u0 = STREAM ? tsv[(2 * s) * T + t] : __ldg(ubk + (2 * s) * T + t);
                        const float2 u1 = STREAM ? tsv[(2 * s + 1) * T + t] : __ldg(ubk + (2 * s + 1) * T + t);
                        z.re = fmaf(u1.x, gb[2 * s + 1], u0.x * gb[2 * s]);
                        z.im = fmaf(u1.y, gb[2 * s + 1], u0.y * gb[2 * s]);
                    }
                    x[s] = z;
                }
                if (A.ovmode == 1) {
                    // The lane's extra points in one flat loop (a warp runs as many iterations
                    // as its busiest lane has points), their bin slot s packed with the point
                    // index and u_k lane-interleaved, so no load waits on another.  The sums
                    // go to the lane's own column of the exchange buffer, free until step A
                    // once every lane of the fibre is past the previous term's step B.
                    gsync<T, FT>(fl);
                    const int cnt = (int)pk[0];
                    if (cnt) {
#pragma unroll
                        for (int s = 0; s <= 8; ++s) buf[s * T + t] = make_float2(0.0f, 0.0f);
                        const float2* ouk = reinterpret_cast<const float2*>(A.ovu) + (size_t)k * A.ovmax * T;
                        for (int i = 0; i < cnt; ++i) {
                            const int e = __ldg(A.ovj + i * T + t);
                            const float2 u = __ldg(ouk + i * T + t);
                            const int j = e & 0xfffff, s = e >> 20;
                            const float g = aux[S::apad(j)];
                            float2 z = buf[s * T + t];
                            z.x = fmaf(u.x, g, z.x);
                            z.y = fmaf(u.y, g, z.y);
                            buf[s * T + t] = z;
                        }
#pragma unroll
                        for (int s = 0; s <= 8; ++s) {
                            const float2 z = buf[s * T + t];
                            x[s].re += z.x;
                            x[s].im += z.y;
                        }
                    }
                } else if (A.ovmode == 2 && pk[0]) {
                    const float2* uk = utab + (size_t)k * n;
#pragma unroll
                    for (int s = 0; s <= 8; ++s) {
                        const int m = t + T * s;
                        if (m > L / 2) continue;
                        const int p2 = __ldg(A.bin_ptr + m + 1);
                        for (int p = __ldg(A.bin_ptr + m) + 2; p < p2; ++p) {
                            const int j = sorted ? p : __ldg(A.bin_idx + p);
                            const float2 u = __ldg(uk + j);
                            const float g = aux[S::apad(j)];
                            x[s].re = fmaf(u.x, g, x[s].re);
                            x[s].im = fmaf(u.y, g, x[s].im);
                        }
                    }
                }
            }
            // step A: 16-point DFT over s, then the per-lane twiddles
            if constexpr (FWD)
                dft<16, float>(x);
            else
                dft16_low9<float>(x);
            if constexpr (TW_SMEM) {
                apply_powers15(x, twS + t, T);
            } else {
#pragma unroll
                for (int k1 = 1; k1 < 16; ++k1) x[k1] = cmul(x[k1], twA[k1]);
            }
            // exchange: buf[k1][t]
            gsync<T, FT>(fl);
#pragma unroll
            for (int k1 = 0; k1 < 16; ++k1) buf[k1 * S::XROW + t] = f2(x[k1]);
            // adjoint: the v_k values the end of this rank term needs, fetched while step B runs
            float2 post[FWD ? 1 : 16];
            if constexpr (!FWD) {
#pragma unroll
                for (int o = 0; o < 16; ++o) post[o] = STREAM ? tsu[o * T + t] : __ldg(vown + ((size_t)k * 16 + o) * T + t);
            }
            gsync<T, FT>(fl);
            Cx<float> y[16];  // step-B outputs in Own<> order
            if constexpr (T == 32) {
                const int k1 = t >> 1, h = t & 1;
                Cx<float> a[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) a[q] = cx(buf[k1 * S::XROW + 2 * q + h]);
                dft<16, float>(a);
                // odd lanes: twiddle w_32^{k2'}
                if (h) {
                    a[1] = twc<1, 32, float>(a[1]);
                    a[2] = twc<2, 32, float>(a[2]);
                    a[3] = twc<3, 32, float>(a[3]);
                    a[4] = twc<4, 32, float>(a[4]);
                    a[5] = twc<5, 32, float>(a[5]);
                    a[6] = twc<6, 32, float>(a[6]);
                    a[7] = twc<7, 32, float>(a[7]);
                    a[8] = twc<8, 32, float>(a[8]);
                    a[9] = twc<9, 32, float>(a[9]);
                    a[10] = twc<10, 32, float>(a[10]);
                    a[11] = twc<11, 32, float>(a[11]);
                    a[12] = twc<12, 32, float>(a[12]);
                    a[13] = twc<13, 32, float>(a[13]);
                    a[14] = twc<14, 32, float>(a[14]);
                    a[15] = twc<15, 32, float>(a[15]);
                }
                // radix-2 across the lane pair: lane h keeps k2' in [8h, 8h + 8)
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    Cx<float> send = h ? a[i] : a[8 + i];
                    Cx<float> own = h ? a[8 + i] : a[i];
                    Cx<float> recv{__shfl_xor_sync(0xffffffffu, send.re, 1), __shfl_xor_sync(0xffffffffu, send.im, 1)};
                    // B_0 + B_1 and B_0 - B_1 (own is B_h, recv is B_{1-h})
                    y[i] = own + recv;
                    Cx<float> d = own - recv;
                    y[8 + i] = h ? Cx<float>{-d.re, -d.im} : d;
                }
            } else if constexpr (T >= 64) {
                // problem k1 is split over R lanes h: a 16-point DFT over q of X1[R q + h][k1],
                // the twiddle w_T^{h k2'}, a second exchange, then R-point DFTs over h
                constexpr int R = S::R, QP = S::QP;
                const int k1 = t / R, h = t % R;
                Cx<float> a[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) a[q] = cx(buf[k1 * S::XROW + R * q + h]);
                dft<16, float>(a);
                apply_powers15(a, twS + 4 * T + h, R);
                gsync<T, FT>(fl);
#pragma unroll
                for (int k2 = 0; k2 < 16; ++k2) buf[S::x2idx(k1, k2, h)] = f2(a[k2]);
                gsync<T, FT>(fl);
#pragma unroll
                for (int i = 0; i < QP; ++i) {
                    const int k2 = h * QP + i;
                    Cx<float> b[R];
#pragma unroll
                    for (int hh = 0; hh < R; ++hh) b[hh] = cx(buf[S::x2idx(k1, k2, hh)]);
                    dft<R, float>(b);
#pragma unroll
                    for (int g2 = 0; g2 < R; ++g2) y[i * R + g2] = b[g2];
                }
            } else {
                constexpr int P = 16 / T;
#pragma unroll
                for (int q = 0; q < P; ++q) {
                    Cx<float> a[T];
                    const int k1 = t * P + q;
#pragma unroll
                    for (int tt = 0; tt < T; ++tt) a[tt] = cx(buf[k1 * S::XROW + tt]);
                    dft<T, float>(a);
#pragma unroll
                    for (int k2 = 0; k2 < T; ++k2) y[q * T + k2] = a[k2];
                }
            }
            if (fbin) {
                // acc at the points of the lane's own bins += Re(u_k y), u_k in bin order
                const float2* fbk = fbtab + (size_t)k * (18 * T);
#pragma unroll
                for (int c = 0; c < 9; ++c) {
                    const Cx<float> yc = y[fslot<LOG2L>(c)];
                    const float2 u0 = STREAM ? tsu[(2 * c) * T + t] : __ldg(fbk + (2 * c) * T + t);
                    const float2 u1 = STREAM ? tsu[(2 * c + 1) * T + t] : __ldg(fbk + (2 * c + 1) * T + t);
                    acc[2 * c] = fmaf(u0.x, yc.re, fmaf(-u0.y, yc.im, acc[2 * c]));
                    acc[2 * c + 1] = fmaf(u1.x, yc.re, fmaf(-u1.y, yc.im, acc[2 * c + 1]));
                }
            } else if constexpr (FWD) {
                // Y[m] for m <= L/2 into the gather buffer, then acc_j += Re(u_k[j] Y[m_j])
                gsync<T, FT>(fl);
#pragma unroll
                for (int o = 0; o < 16; ++o) {
                    int m = Own<LOG2L, FWD>::idx(t, o);
                    if (m <= L / 2) buf[S::ypad(m)] = f2(y[o]);
                }
                gsync<T, FT>(fl);
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    int j = t + T * e;
                    if (j < n) {
                        const unsigned ym = (e & 1) ? (pk[e >> 1] >> 16) : (pk[e >> 1] & 0xffffu);
                        float2 yy = buf[ym];
                        const float2 u = __ldg(utab + (size_t)k * n + j);
                        acc[e] = fmaf(u.x, yy.x, fmaf(-u.y, yy.y, acc[e]));
                    }
                }
            } else {
#pragma unroll
                for (int o = 0; o < 16; ++o) {
                    const float2 v = post[o];
                    acc[o] = fmaf(v.x, y[o].re, fmaf(-v.y, y[o].im, acc[o]));
                }
            }
        }

        if (fbin) {
            // bin order back to natural order through the exchange region
            float* nat = reinterpret_cast<float*>(smem_raw);
            __syncthreads();  // every group is done with the exchange region
#pragma unroll
            for (int q = 0; q < 18; ++q) {
                const int j = __ldg(A.bjf + q * T + t);
                if (j >= 0) nat[fl * L + j] = acc[q];
            }
            __syncthreads();
#pragma unroll
            for (int e = 0; e < 16; ++e) acc[e] = nat[fl * L + t + T * e];
        }

        // store
        if (SPLIT && csize > 1) {
            // partial sums of the cluster's CTAs, [FT][L + 1] over the exchange region; CTA
            // crank adds up and stores its share of the tile's FT x L = 4096 elements
            constexpr int LP = L + 1;
            float* red = reinterpret_cast<float*>(smem_raw);
            __syncthreads();  // every group is done with the exchange region
            if constexpr (FWD) {
#pragma unroll
                for (int e = 0; e < 16; ++e) red[fl * LP + t + T * e] = acc[e];
            } else {
#pragma unroll
                for (int o = 0; o < 16; ++o) red[fl * LP + Own<LOG2L, FWD>::idx(t, o)] = acc[o];
            }
            cluster_sync();
            const int per = (FT * L) / (int)csize;
            for (int i = threadIdx.x; i < per; i += S::THREADS) {
                const int el = (int)crank * per + i;
                // strided axes: fibres fastest, so that neighbouring threads store neighbours
                const int fib = STRIDED ? el % FT : el / L;
                const int j = STRIDED ? el / FT : el % L;
                const long long ff = f0 + fib;
                if (j < n && ff < nfib) {
                    float v = 0.0f;
                    for (unsigned r = 0; r < csize; ++r) v += ld_cluster(red + fib * LP + j, r);
                    out[fibre_offset(ff, n, inner) + (long long)j * inner] = v;
                }
            }
            cluster_sync();  // the peers are done reading before the region is reused
        } else if constexpr (STRIDED) {
            __syncthreads();
            if constexpr (FWD) {
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    int j = t + T * e;
                    if (j < n) tile[fl * S::TROW + j] = acc[e];
                }
            } else {
#pragma unroll
                for (int o = 0; o < 16; ++o) {
                    int nu = Own<LOG2L, FWD>::idx(t, o);
                    if (nu < n) tile[fl * S::TROW + nu] = acc[o];
                }
            }
            __syncthreads();
            {
                const int ql = threadIdx.x % FT;
                const long long ff = f0 + ql;
                if (ff < nfib) {
                    constexpr int RSTEP = S::THREADS / FT;
                    const int r0 = threadIdx.x / FT;
                    const float* trow = tile + ql * S::TROW;
                    float* p = out + fibre_offset(ff, n, inner) + (long long)r0 * inner;
                    const long long step = (long long)RSTEP * inner;
#pragma unroll 4
                    for (int row = r0; row < n; row += RSTEP, p += step) *p = trow[row];
                }
            }
        } else if (valid) {
            const long long base = f * (long long)n;
            if constexpr (FWD) {
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    int j = t + T * e;
                    if (j < n) out[base + j] = acc[e];
                }
            } else {
#pragma unroll
                for (int o = 0; o < 16; ++o) {
                    int nu = Own<LOG2L, FWD>::idx(t, o);
                    if (nu < n) out[base + nu] = acc[o];
                }
            }
        }
    }
}

}  // namespace dev
}  // namespace jt
