// Plans and the transform entry points of the C ABI (include/jt.h).
//
// jt_plan_create runs the host setup of every axis (jt_setup.cpp), converts the tables to
// the working precision, uploads them once, and keeps them for the lifetime of the plan.
// jt_forward / jt_adjoint sweep the axes one at a time (Sec. 3.2--3.3, Eqs. eq:TJ, eq:TJ3,
// eq:invTJ, eq:invTJ3): the first sweep reads the caller's input and writes the caller's
// output, every later sweep works in place on the output, fibre by fibre, so no scratch
// array is needed.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <mutex>
#include <cstring>
#include <new>
#include <thread>
#include <type_traits>
#include <vector>

#include "jt.h"
#include "jt_internal.hpp"
#include "jt_launch.hpp"
#include "jt_plain.hpp"

namespace {

using jt::dev::AxisDev;
using jt::dev::Cx;
using jt::dev::dw;

struct DeviceAxis {
    jt::AxisTables host;
    AxisDev dev{};
    jt::dev::BigAxisDev big{};  // double-word axes of length 2^14 only
    int log2L = 0;
    std::vector<void*> allocs;
};

}  // namespace

struct jt_plan {
    int d = 0;
    int prec = JT_FP32;
    bool all_uniform = true;
    int64_t n[3] = {1, 1, 1};
    std::vector<DeviceAxis> axes;
    jt::PlainPlan* plain = nullptr;  // JT_FP64_PLAIN resources
    // Schedules of the fused sweeps: the rank split (CTAs per tile) of each (axis, direction).
    // A measured choice for a sweep of that many fibres (jt_plan_tune) comes first, then a
    // fixed one (jt_plan_set_ksplit), then the occupancy rule of the launchers.
    int ksplit_fixed[3][2] = {{0, 0}, {0, 0}, {0, 0}};
    bool autotune = false;  // jt_batch_create measures the splits of this plan's sweeps
    int kind = JT_FIRST_KIND;
    struct Tuned {
        int axis, fwd;
        long long nfib;
        int ksplit;
    };
    std::vector<Tuned> tuned;
    // host-array transforms (jt_transform_host): three streams and their events, made on first use
    static constexpr int PIPES = 3;
    std::mutex pipe_mu;
    cudaStream_t pipe[PIPES] = {nullptr, nullptr, nullptr};
    cudaEvent_t pipe_fork = nullptr, pipe_done[PIPES] = {nullptr, nullptr, nullptr};
};

namespace {

template <class T>
jt_status upload(DeviceAxis& ax, const std::vector<T>& host, const void** dst, cudaStream_t s) {
    if (host.empty()) {
        *dst = nullptr;
        return JT_OK;
    }
    void* p = nullptr;
    if (cudaMalloc(&p, sizeof(T) * host.size()) != cudaSuccess) {
        cudaGetLastError();
        return JT_ENOMEM;
    }
    ax.allocs.push_back(p);
    if (cudaMemcpyAsync(p, host.data(), sizeof(T) * host.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return JT_ECUDA;
    *dst = p;
    return JT_OK;
}

inline float to_r(double v, float*) { return (float)v; }
inline dw to_r(double v, dw*) {
    float h = (float)v;
    return dw{h, (float)(v - (double)h)};
}

// Build and upload the device tables of one axis in precision R.
// Output slot o of lane t in the four-step adjoint (jt_warp.cuh, Own<>) for FFT length 2^lg.
template <int LG>
int own_index(int lg, int t, int o) {
    if (lg == LG) return jt::dev::Own<LG, false>::idx(t, o);
    if constexpr (LG > jt::F32_WARP_MIN_LOG2L) return own_index<LG - 1>(lg, t, o);
    return 0;
}

// Forward output slot c of the four-step kernel (jt_warp.cuh, fslot<>) for FFT length 2^lg.
template <int LG>
int fslot_index(int lg, int c) {
    if (lg == LG) return jt::dev::fslot<LG>(c);
    if constexpr (LG > jt::F32_WARP_MIN_LOG2L) return fslot_index<LG - 1>(lg, c);
    return 0;
}

template <class R>
jt_status build_device_axis(DeviceAxis& ax, cudaStream_t s) {
    const jt::AxisTables& T = ax.host;
    const int64_t n = T.n, L = T.L, r = T.rank, nu0 = T.nu0, N = T.N;
    R* tag = nullptr;
    std::vector<Cx<R>> vtab((size_t)r * L, Cx<R>{to_r(0.0, tag), to_r(0.0, tag)});
    for (int64_t k = 0; k < r; ++k)
        for (int64_t c = 0; c < N; ++c) {
            const jt::cd v = T.V[(size_t)k * N + c];
            vtab[(size_t)k * L + nu0 + c] = Cx<R>{to_r(v.real(), tag), to_r(v.imag(), tag)};
        }
    // second kind: Im(u y) = Re((-i u) y), so the kernels take -i u_k and stay unchanged
    std::vector<Cx<R>> utab((size_t)r * n);
    const bool second = T.kind == JT_SECOND_KIND;
    for (size_t i = 0; i < utab.size(); ++i) {
        const double ur = second ? T.U[i].imag() : T.U[i].real();
        const double ui = second ? -T.U[i].real() : T.U[i].imag();
        utab[i] = Cx<R>{to_r(ur, tag), to_r(ui, tag)};
    }
    std::vector<R> vblk;
    if (std::is_same<R, float>::value && jt::f32_warp_path(ax.log2L)) {
        // rows padded to L with zeros (warp kernel)
        vblk.assign((size_t)nu0 * L, to_r(0.0, tag));
        for (int64_t j = 0; j < n; ++j)
            for (int64_t c = 0; c < nu0; ++c) vblk[(size_t)c * L + j] = to_r(T.Vblk[(size_t)j * nu0 + c], tag);
    } else {
        vblk.assign((size_t)nu0 * n, to_r(0.0, tag));
        for (int64_t j = 0; j < n; ++j)
            for (int64_t c = 0; c < nu0; ++c) vblk[(size_t)c * n + j] = to_r(T.Vblk[(size_t)j * nu0 + c], tag);
    }
    std::vector<Cx<R>> twid(L);
    const double twopi = 6.283185307179586476925286766559;
    if (std::is_same<R, float>::value && ax.log2L > jt::F32_WARP_MAX_LOG2L) {
        // FP32 Stockham axes longer than 4096: the twiddles in pass order, pass of span NS
        // (R0, 16 R0, 256 R0) at [NS - R0 + (r - 1) NS + k] = e^{2 pi i r k / (16 NS)}, r = 1..15,
        // k < NS, so that the lanes of a pass read consecutive entries
        const int P = (ax.log2L + 3) / 4;
        const int64_t R0 = (int64_t)1 << (ax.log2L - 4 * (P - 1));
        for (int64_t ns = R0; ns < L; ns *= 16)
            for (int64_t i = 0; i < 15 * ns; ++i) {
                const int64_t r = 1 + i / ns, k = i % ns;
                double ang = twopi * (double)(r * k) / (double)(16 * ns);
                twid[ns - R0 + i] = Cx<R>{to_r(std::cos(ang), tag), to_r(std::sin(ang), tag)};
            }
    } else {
        for (int64_t q = 0; q < L; ++q) {
            double ang = twopi * (double)q / (double)L;
            twid[q] = Cx<R>{to_r(std::cos(ang), tag), to_r(std::sin(ang), tag)};
        }
    }
    // bins: points of bin m are bin_idx[bin_ptr[m] .. bin_ptr[m+1]), m = 0..L/2
    std::vector<int> bin_ptr(L / 2 + 2, 0), bin_idx(n);
    for (int64_t j = 0; j < n; ++j) bin_ptr[T.m[j] + 1]++;
    for (int64_t m = 0; m <= L / 2; ++m) bin_ptr[m + 1] += bin_ptr[m];
    {
        std::vector<int> fill(bin_ptr.begin(), bin_ptr.end() - 1);
        for (int64_t j = 0; j < n; ++j) bin_idx[fill[T.m[j]]++] = (int)j;
    }
    std::vector<int> mtab(T.m.begin(), T.m.end());
    // bin-ordered copy of u_k for the FP32 warp kernel: [k][(s * 2 + i) * TT + t] = u_k at the
    // i-th point of bin m = t + TT s (s <= 8, i < 2), zero where the bin has fewer points
    std::vector<Cx<R>> ubtab, ovu, vown, fbtab;
    std::vector<int> bjtab, ovftab, ovj, bjf;
    int ovmode = 0, ovmax = 0, fbin = 0;
    // u_k at the first two points of the bins m = t + TT s of slots s < nsl: [k][(s * 2 + i) * TT + t]
    auto fill_ubtab = [&](int64_t TT, int64_t nsl) {
        ubtab.assign((size_t)r * 2 * nsl * TT, Cx<R>{to_r(0.0, tag), to_r(0.0, tag)});
        for (int64_t k = 0; k < r; ++k)
            for (int64_t s2 = 0; s2 < nsl; ++s2)
                for (int64_t t = 0; t < TT; ++t) {
                    const int64_t m = t + TT * s2;
                    if (m > L / 2) continue;
                    for (int i = 0; i < 2; ++i) {
                        const int64_t p = bin_ptr[m] + i;
                        if (p >= bin_ptr[m + 1]) break;
                        const int64_t j = bin_idx[p];
                        ubtab[(size_t)k * 2 * nsl * TT + (s2 * 2 + i) * TT + t] = utab[(size_t)k * n + j];
                    }
                }
    };
    if (std::is_same<R, float>::value && jt::f32_warp_path(ax.log2L)) {
        const int64_t TT = L / 16;
        // v_k in the adjoint's output order: [k][o][t] = v_k[Own(t, o)], coalesced per slot
        vown.resize((size_t)r * 16 * TT);
        for (int64_t k = 0; k < r; ++k)
            for (int o = 0; o < 16; ++o)
                for (int64_t t = 0; t < TT; ++t)
                    vown[((size_t)k * 16 + o) * TT + t] =
                        vtab[(size_t)k * L + own_index<jt::F32_WARP_MAX_LOG2L>(ax.log2L, (int)t, o)];
        bjtab.assign((size_t)18 * TT, -1);
        ovftab.assign((size_t)2 * TT, 0);
        int most = 0;  // largest number of extra points in one bin
        for (int64_t m = 0; m <= L / 2; ++m) most = std::max(most, bin_ptr[m + 1] - bin_ptr[m] - 2);
        ovmode = most <= 0 ? 0 : (most <= 15 ? 1 : 2);
        std::vector<std::vector<int>> lists((size_t)TT);
        for (int64_t s2 = 0; s2 <= 8; ++s2)
            for (int64_t t = 0; t < TT; ++t) {
                const int64_t m = t + TT * s2;
                if (m > L / 2) continue;
                for (int i = 0; i < 2; ++i)
                    if (bin_ptr[m] + i < bin_ptr[m + 1]) bjtab[(s2 * 2 + i) * TT + t] = bin_idx[bin_ptr[m] + i];
                const int extra = std::max(0, bin_ptr[m + 1] - bin_ptr[m] - 2);
                if (ovmode == 1) {
                    for (int p = bin_ptr[m] + 2; p < bin_ptr[m + 1]; ++p) lists[t].push_back(bin_idx[p]);
                    ovftab[2 * t] += extra;
                } else if (ovmode == 2 && extra > 0) {
                    ovftab[2 * t] = 1;
                }
            }
        if (ovmode == 1) {
            for (const auto& l : lists) ovmax = std::max(ovmax, (int)l.size());
            ovj.assign((size_t)ovmax * TT, 0);
            ovu.assign((size_t)r * ovmax * TT, Cx<R>{to_r(0.0, tag), to_r(0.0, tag)});
            for (int64_t t = 0; t < TT; ++t)
                for (size_t i = 0; i < lists[t].size(); ++i) {
                    const int j = lists[t][i];
                    const int s2 = (int)((T.m[j] - t) / TT);  // the lane's bin slot of point j
                    ovj[i * TT + t] = j | (s2 << 20);
                    for (int64_t k = 0; k < r; ++k) ovu[((size_t)k * ovmax + i) * TT + t] = utab[(size_t)k * n + j];
                }
        }
        // forward in bin order (no bin with more than two points): the points of the output
        // bins each lane keeps after step B, and u_k there; every point must appear once
        if (ovmode == 0) {
            bjf.assign((size_t)18 * TT, -1);
            std::vector<int> seen(n, 0);
            for (int64_t t = 0; t < TT; ++t)
                for (int c = 0; c < 9; ++c) {
                    if (c == 8 && t != 0) continue;
                    const int64_t m = own_index<jt::F32_WARP_MAX_LOG2L>(ax.log2L, (int)t,
                                                                        fslot_index<jt::F32_WARP_MAX_LOG2L>(ax.log2L, c));
                    if (m > L / 2) continue;
                    for (int i = 0; i < 2 && bin_ptr[m] + i < bin_ptr[m + 1]; ++i) {
                        const int j = bin_idx[bin_ptr[m] + i];
                        bjf[(size_t)(2 * c + i) * TT + t] = j;
                        seen[j]++;
                    }
                }
            fbin = 1;
            for (int64_t j = 0; j < n; ++j)
                if (seen[j] != 1) fbin = 0;
            if (fbin) {
                fbtab.assign((size_t)r * 18 * TT, Cx<R>{to_r(0.0, tag), to_r(0.0, tag)});
                for (int64_t k = 0; k < r; ++k)
                    for (size_t q = 0; q < bjf.size(); ++q)
                        if (bjf[q] >= 0) fbtab[(size_t)k * 18 * TT + q] = utab[(size_t)k * n + bjf[q]];
            } else {
                bjf.clear();
            }
        }
        fill_ubtab(TT, 9);
    } else if (std::is_same<R, float>::value && ax.log2L > jt::F32_WARP_MAX_LOG2L) {
        // FP32 Stockham axes longer than 4096 (threads of T = L / 16, bins m = t + T e): the
        // adjoint's bin-ordered tables, and per thread a flag for a bin with more than two points
        const int64_t TT = L / 16;
        bjtab.assign((size_t)18 * TT, -1);
        ovftab.assign((size_t)2 * TT, 0);
        for (int64_t s2 = 0; s2 <= 8; ++s2)
            for (int64_t t = 0; t < TT; ++t) {
                const int64_t m = t + TT * s2;
                if (m > L / 2) continue;
                for (int i = 0; i < 2; ++i)
                    if (bin_ptr[m] + i < bin_ptr[m + 1]) bjtab[(s2 * 2 + i) * TT + t] = bin_idx[bin_ptr[m] + i];
                if (bin_ptr[m + 1] - bin_ptr[m] > 2) ovftab[2 * t] = 1;
            }
        fill_ubtab(TT, 9);
    } else if (std::is_same<R, dw>::value && ax.log2L <= jt::DW_SMEM_MAX_LOG2L) {
        // Double-word Stockham axes (E = min(L, 8) elements a thread, TT = L / E threads, bins
        // m = t + TT e): the adjoint's bin-ordered tables for the slots e < E / 2, so that
        // u_k of one rank term takes L entries like v_k; bin L/2 (thread 0, slot E / 2) and the
        // points past the first two of a bin are walked, on the threads flagged here
        const int64_t E = std::min<int64_t>(L, 8), TT = L / E, nsl = E / 2;
        bjtab.assign((size_t)2 * nsl * TT, -1);
        ovftab.assign((size_t)2 * TT, 0);
        for (int64_t s2 = 0; s2 < nsl; ++s2)
            for (int64_t t = 0; t < TT; ++t) {
                const int64_t m = t + TT * s2;
                for (int i = 0; i < 2; ++i)
                    if (bin_ptr[m] + i < bin_ptr[m + 1]) bjtab[(s2 * 2 + i) * TT + t] = bin_idx[bin_ptr[m] + i];
                if (bin_ptr[m + 1] - bin_ptr[m] > 2) ovftab[2 * t] = 1;
            }
        if (bin_ptr[L / 2 + 1] > bin_ptr[L / 2]) ovftab[0] = 1;
        fill_ubtab(TT, nsl);
    }
    AxisDev& A = ax.dev;
    A.n = (int)n;
    A.L = (int)L;
    A.nu0 = (int)nu0;
    A.rank = (int)r;
    A.sorted = 1;
    for (int64_t j = 1; j < n; ++j)
        if (T.m[j] < T.m[j - 1]) A.sorted = 0;
    jt_status st;
    const void* p;
    if ((st = upload(ax, vtab, &A.vtab, s)) != JT_OK) return st;
    if ((st = upload(ax, utab, &A.utab, s)) != JT_OK) return st;
    if ((st = upload(ax, mtab, &p, s)) != JT_OK) return st;
    A.mtab = (const int*)p;
    if ((st = upload(ax, vblk, &A.vblk, s)) != JT_OK) return st;
    if ((st = upload(ax, twid, &A.twid, s)) != JT_OK) return st;
    if ((st = upload(ax, bin_ptr, &p, s)) != JT_OK) return st;
    A.bin_ptr = (const int*)p;
    if ((st = upload(ax, bin_idx, &p, s)) != JT_OK) return st;
    A.bin_idx = (const int*)p;
    if ((st = upload(ax, ubtab, &A.ubtab, s)) != JT_OK) return st;
    if ((st = upload(ax, bjtab, &p, s)) != JT_OK) return st;
    A.bjtab = (const int*)p;
    if ((st = upload(ax, vown, &A.vown, s)) != JT_OK) return st;
    if ((st = upload(ax, ovftab, &p, s)) != JT_OK) return st;
    A.ovftab = (const int*)p;
    if ((st = upload(ax, ovj, &p, s)) != JT_OK) return st;
    A.ovj = (const int*)p;
    if ((st = upload(ax, ovu, &A.ovu, s)) != JT_OK) return st;
    A.ovmax = ovmax;
    A.ovmode = ovmode;
    if ((st = upload(ax, fbtab, &A.fbtab, s)) != JT_OK) return st;
    if ((st = upload(ax, bjf, &p, s)) != JT_OK) return st;
    A.bjf = (const int*)p;
    A.fbin = fbin;
    // status word of the bounded waits (cleared by jt_plan_check)
    const std::vector<unsigned> status0(1, 0u);
    if ((st = upload(ax, status0, &p, s)) != JT_OK) return st;
    A.status = (unsigned*)p;
    A.skip_copy = 0;
    // Double-word axes of length 2^14: the tables of the two half-length transforms
    // (jt_axis_dw_big.cu): u_k e^{2 pi i m_j / L}, bins m_j mod L/2 and their CSR, the
    // half-length twiddles, and the partial-sum buffer of one launch.
    std::vector<Cx<R>> utab1, tw2;
    std::vector<int> mtab2, bin_ptr2, bin_idx2;
    if (std::is_same<R, dw>::value && ax.log2L == jt::MAX_LOG2L_DW) {
        const int64_t Lh = L / 2;
        utab1.resize((size_t)r * n);
        for (int64_t k = 0; k < r; ++k)
            for (int64_t j = 0; j < n; ++j) {
                const size_t i = (size_t)k * n + j;
                const jt::cd u = second ? jt::cd(T.U[i].imag(), -T.U[i].real()) : T.U[i];
                const double ang = twopi * (double)T.m[j] / (double)L;
                const jt::cd v = u * jt::cd(std::cos(ang), std::sin(ang));
                utab1[i] = Cx<R>{to_r(v.real(), tag), to_r(v.imag(), tag)};
            }
        tw2.resize(Lh);
        for (int64_t q = 0; q < Lh; ++q) {
            const double ang = twopi * (double)q / (double)Lh;
            tw2[q] = Cx<R>{to_r(std::cos(ang), tag), to_r(std::sin(ang), tag)};
        }
        mtab2.resize(n);
        bin_ptr2.assign(Lh + 1, 0);
        bin_idx2.resize(n);
        for (int64_t j = 0; j < n; ++j) {
            mtab2[j] = (int)(T.m[j] % Lh);
            bin_ptr2[mtab2[j] + 1]++;
        }
        for (int64_t m = 0; m < Lh; ++m) bin_ptr2[m + 1] += bin_ptr2[m];
        std::vector<int> fill(bin_ptr2.begin(), bin_ptr2.end() - 1);
        for (int64_t j = 0; j < n; ++j) bin_idx2[fill[mtab2[j]]++] = (int)j;
        jt::dev::BigAxisDev& Bg = ax.big;
        Bg.n = (int)n;
        Bg.nu0 = (int)nu0;
        Bg.rank = (int)r;
        Bg.vtab = reinterpret_cast<const Cx<dw>*>(A.vtab);
        Bg.utab = reinterpret_cast<const Cx<dw>*>(A.utab);
        Bg.vblk = reinterpret_cast<const dw*>(A.vblk);
        if ((st = upload(ax, utab1, &p, s)) != JT_OK) return st;
        Bg.utab1 = reinterpret_cast<const Cx<dw>*>(p);
        if ((st = upload(ax, tw2, &p, s)) != JT_OK) return st;
        Bg.tw2 = reinterpret_cast<const Cx<dw>*>(p);
        if ((st = upload(ax, mtab2, &p, s)) != JT_OK) return st;
        Bg.mtab2 = (const int*)p;
        if ((st = upload(ax, bin_ptr2, &p, s)) != JT_OK) return st;
        Bg.bin_ptr2 = (const int*)p;
        if ((st = upload(ax, bin_idx2, &p, s)) != JT_OK) return st;
        Bg.bin_idx2 = (const int*)p;
        int dev_id = 0, sms = 0;
        if (cudaGetDevice(&dev_id) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev_id) != cudaSuccess)
            return JT_ECUDA;
        Bg.max_ctas = std::max(1, sms);
        void* part = nullptr;
        if (cudaMalloc(&part, sizeof(dw) * (size_t)Bg.max_ctas * (size_t)n) != cudaSuccess) {
            cudaGetLastError();
            return JT_ENOMEM;
        }
        ax.allocs.push_back(part);
        Bg.part = reinterpret_cast<dw*>(part);
        if (jt::dw_big_init() != cudaSuccess) return JT_ECUDA;
    }
    // keep the host vectors alive until the copies are done
    if (cudaStreamSynchronize(s) != cudaSuccess) return JT_ECUDA;
    return JT_OK;
}

void free_axis(DeviceAxis& ax) {
    for (void* p : ax.allocs) cudaFree(p);
    ax.allocs.clear();
}

// Rank split of the sweep of axis ax over nfib fibres.
int sweep_ksplit(const jt_plan* plan, int ax, bool fwd, long long nfib, bool strided) {
    for (const auto& t : plan->tuned)
        if (t.axis == ax && t.fwd == (int)fwd && t.nfib == nfib) return t.ksplit;
    const int fixed = plan->ksplit_fixed[ax][fwd ? 0 : 1];
    if (fixed > 0) return fixed;
    const DeviceAxis& A = plan->axes[ax];
    if (plan->prec == JT_FP32) return jt::auto_ksplit_f32(A.log2L, fwd, strided, nfib, A.dev.rank);
    return jt::auto_ksplit_dw(A.log2L, fwd, nfib, A.dev.rank);
}

cudaError_t launch_sweep(const jt_plan* plan, int ax, bool fwd, const void* src, void* dst, long long nfib,
                         long long inner, int ksplit, cudaStream_t s) {
    const DeviceAxis& A = plan->axes[ax];
    if (plan->prec == JT_FP32)
        return jt::launch_axis_f32(A.dev, A.log2L, fwd, (const float*)src, (float*)dst, nfib, inner, ksplit, s);
    if (A.log2L > jt::DW_SMEM_MAX_LOG2L)
        return jt::launch_axis_dw_big(A.big, fwd, (const double*)src, (double*)dst, nfib, inner, s);
    return jt::launch_axis_dw(A.dev, A.log2L, fwd, (const double*)src, (double*)dst, nfib, inner, ksplit, s);
}

// Sweep every axis (last axis first).  Sweep 0 maps in -> out; later sweeps run in place.
template <class IO>
jt_status sweep(jt_plan* plan, const IO* in, IO* out, int64_t nrhs, bool fwd, cudaStream_t s) {
    const int d = plan->d;
    int64_t total = nrhs;
    for (int i = 0; i < d; ++i) total *= plan->n[i];
    const IO* src = in;
    for (int ax = d - 1; ax >= 0; --ax) {
        int64_t inner = 1;
        for (int i = ax + 1; i < d; ++i) inner *= plan->n[i];
        const int64_t nfib = total / plan->n[ax];
        const int ks = sweep_ksplit(plan, ax, fwd, nfib, inner > 1);
        if (launch_sweep(plan, ax, fwd, src, out, nfib, inner, ks, s) != cudaSuccess) return JT_ECUDA;
        src = out;
    }
    return JT_OK;
}

jt_status apply(jt_plan* plan, const void* in, void* out, int64_t nrhs, bool fwd, cudaStream_t s) {
    if (!plan || !in || !out || nrhs < 1) return JT_EINVAL;
    int64_t total = nrhs;
    for (int i = 0; i < plan->d; ++i) {
        if (total > (int64_t(1) << 40) / plan->n[i]) return JT_EINVAL;
        total *= plan->n[i];
    }
    try {
        if (plan->prec == JT_FP32) return sweep<float>(plan, (const float*)in, (float*)out, nrhs, fwd, s);
        if (plan->prec == JT_SPLIT) return sweep<double>(plan, (const double*)in, (double*)out, nrhs, fwd, s);
        if (plan->prec == JT_FP64_PLAIN)
            return jt::plain_apply(plan->plain, (const double*)in, (double*)out, nrhs, fwd, s);
    } catch (...) {
        return JT_ENOMEM;
    }
    return JT_EINVAL;
}

}  // namespace

// Total elements of nrhs right-hand sides, or -1 past the addressing limit.
int64_t plan_elements(const jt_plan* plan, int64_t nrhs) {
    int64_t total = nrhs;
    for (int i = 0; i < plan->d; ++i) {
        if (total > (int64_t(1) << 40) / plan->n[i]) return -1;
        total *= plan->n[i];
    }
    return total;
}

// Measure the rank splits of every sweep of `plan` for nrhs right-hand sides (see
// jt_plan_tune) and record the fastest of each.
jt_status tune_plan(jt_plan* plan, int64_t nrhs, cudaStream_t s) {
    const int64_t total = plan_elements(plan, nrhs);
    if (total < 1) return JT_EINVAL;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return JT_ECUDA;
    if (cap != cudaStreamCaptureStatusNone) return JT_EINVAL;
    const size_t bytes = (size_t)total * (plan->prec == JT_FP32 ? 4 : 8);
    void *x = nullptr, *y = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    jt_status st = JT_OK;
    if (cudaMalloc(&x, bytes) != cudaSuccess || cudaMalloc(&y, bytes) != cudaSuccess) {
        cudaGetLastError();
        st = JT_ENOMEM;
    } else if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
               cudaMemsetAsync(x, 0, bytes, s) != cudaSuccess) {
        st = JT_ECUDA;
    }
    for (int ax = plan->d - 1; st == JT_OK && ax >= 0; --ax) {
        long long inner = 1;
        for (int i = ax + 1; i < plan->d; ++i) inner *= plan->n[i];
        const long long nfib = total / plan->n[ax];
        const int rank = plan->axes[ax].dev.rank;
        for (int dir = 0; st == JT_OK && dir < 2; ++dir) {
            const bool fwd = dir == 0;
            int best = 1;
            float best_ms = 0.0f;
            for (int ks = 1; ks <= 8 && (ks == 1 || ks <= rank); ks *= 2) {
                float ms = 0.0f;
                if (launch_sweep(plan, ax, fwd, x, y, nfib, inner, ks, s) != cudaSuccess ||
                    cudaEventRecord(e0, s) != cudaSuccess) {
                    st = JT_ECUDA;
                    break;
                }
                for (int rep = 0; rep < 3 && st == JT_OK; ++rep)
                    if (launch_sweep(plan, ax, fwd, x, y, nfib, inner, ks, s) != cudaSuccess) st = JT_ECUDA;
                if (st != JT_OK || cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                    cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                    st = JT_ECUDA;
                    break;
                }
                if (ks == 1 || ms < best_ms) {
                    best = ks;
                    best_ms = ms;
                }
            }
            if (st != JT_OK) break;
            auto& tv = plan->tuned;
            tv.erase(std::remove_if(tv.begin(), tv.end(),
                                    [&](const jt_plan::Tuned& t) { return t.axis == ax && t.fwd == (int)fwd && t.nfib == nfib; }),
                     tv.end());
            tv.push_back({ax, (int)fwd, nfib, best});
        }
    }
    if (st == JT_OK && cudaStreamSynchronize(s) != cudaSuccess) st = JT_ECUDA;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (x) cudaFree(x);
    if (y) cudaFree(y);
    return st;
}

// A batch: the axis sweeps of several plans, grouped by stage (the s-th sweep of every
// transform) and, inside a stage, by FFT length, stride kind and rank split.  FP32 sweeps of
// length 16..4096 run as one launch per group (at most BATCH_MAX_JOBS jobs a launch); every
// other sweep is launched on its own.  The launches of a stage are spread over a few worker
// streams (forked from and joined back to the caller's stream, with a barrier between
// stages), so that small launches run side by side.  First-stage launches of one-dimensional
// transforms only (nothing later waits for them) go to two more streams of the highest
// priority that take no part in the stage barriers: those are mostly long axes with few
// fibres, whose few CTAs then start at once and run beside the large groups instead of
// holding up the next stage.  Nothing is allocated or copied at execution, so an execution
// can be captured in a CUDA graph.
struct jt_batch {
    static constexpr int WORKERS = 4, FREE = 2, STREAMS = WORKERS + FREE;
    int count = 0;
    int prec = JT_FP32;
    std::vector<jt_plan*> plans;
    std::vector<int64_t> nrhs;
    struct Launch {
        bool fused = false;
        bool free = false;  // on a free stream (index WORKERS + f): no stage barrier
        int stage = 0, log2L = 0, ksplit = 1, worker = 0;
        bool strided = false;
        // fused: device jobs [job_off, job_off + njobs), slot -> transform index
        int job_off = 0, njobs = 0;
        long long total_tiles = 0;
        std::vector<int> slot_transform;
        // single: transform index and axis
        int transform = 0, axis = 0;
        long long nfib = 0, inner = 1;
        double cost = 0;  // relative work, for spreading a stage over the workers
    };
    std::vector<Launch> launches[2];  // [0] forward, [1] adjoint; ordered by stage
    jt::dev::BatchJob* d_jobs = nullptr;
    cudaStream_t work[STREAMS] = {};
    cudaEvent_t ev_fork = nullptr, ev_stage[WORKERS] = {}, ev_join[STREAMS] = {};
};

namespace {

struct SweepJob {
    int transform, axis, stage, log2L, ksplit;
    bool strided, fused;
    long long nfib, inner;
    double cost;
};

jt_status batch_run(jt_batch* b, const void* const* in, void* const* out, bool fwd, cudaStream_t s) {
    if (!b || !in || !out) return JT_EINVAL;
    for (int i = 0; i < b->count; ++i)
        if (!in[i] || !out[i]) return JT_EINVAL;
    constexpr int W = jt_batch::WORKERS, NS = jt_batch::STREAMS;
    if (cudaEventRecord(b->ev_fork, s) != cudaSuccess) return JT_ECUDA;
    for (int w = 0; w < NS; ++w)
        if (cudaStreamWaitEvent(b->work[w], b->ev_fork, 0) != cudaSuccess) return JT_ECUDA;
    int stage = 0;
    for (const auto& L : b->launches[fwd ? 0 : 1]) {
        if (L.stage != stage) {
            // stage barrier: every worker waits for the previous stage on all workers
            for (int w = 0; w < W; ++w)
                if (cudaEventRecord(b->ev_stage[w], b->work[w]) != cudaSuccess) return JT_ECUDA;
            for (int w = 0; w < W; ++w)
                for (int v = 0; v < W; ++v)
                    if (v != w && cudaStreamWaitEvent(b->work[w], b->ev_stage[v], 0) != cudaSuccess) return JT_ECUDA;
            stage = L.stage;
        }
        cudaStream_t ws = b->work[L.worker];
        cudaError_t e = cudaSuccess;
        if (L.fused) {
            jt::dev::BatchPtrs ptrs;
            for (size_t q = 0; q < L.slot_transform.size(); ++q) {
                const int i = L.slot_transform[q];
                ptrs.in[q] = (const float*)(L.stage == 0 ? in[i] : out[i]);
                ptrs.out[q] = (float*)out[i];
            }
            e = jt::launch_axis_f32_batched(L.log2L, fwd, L.strided, b->d_jobs + L.job_off, L.njobs, L.total_tiles,
                                            ptrs, L.ksplit, ws);
        } else {
            const void* src = (L.stage == 0) ? in[L.transform] : out[L.transform];
            e = launch_sweep(b->plans[L.transform], L.axis, fwd, src, out[L.transform], L.nfib, L.inner, L.ksplit, ws);
        }
        if (e != cudaSuccess) return JT_ECUDA;
    }
    for (int w = 0; w < NS; ++w) {
        if (cudaEventRecord(b->ev_join[w], b->work[w]) != cudaSuccess) return JT_ECUDA;
        if (cudaStreamWaitEvent(s, b->ev_join[w], 0) != cudaSuccess) return JT_ECUDA;
    }
    return JT_OK;
}

// Launch lists of one direction: groups per stage, then the stage's launches spread over the
// workers, largest first, each to the least loaded worker (first-stage launches of 1-D
// transforms only over the free streams the same way).
void batch_plan_launches(jt_batch* b, bool fwd, const std::vector<SweepJob>& sweeps, int max_stage,
                         std::vector<jt::dev::BatchJob>& hjobs) {
    auto& out = b->launches[fwd ? 0 : 1];
    for (int st = 0; st <= max_stage; ++st) {
        std::vector<jt_batch::Launch> ls;
        // fused groups: (log2L, strided, ksplit) -> jobs
        for (int lg = jt::F32_WARP_MIN_LOG2L; lg <= jt::F32_WARP_MAX_LOG2L; ++lg)
            for (int sk = 0; sk < 2; ++sk)
                for (int ks = 1; ks <= 8; ks *= 2) {
                    std::vector<const SweepJob*> grp;
                    for (const auto& j : sweeps)
                        if (j.fused && j.stage == st && j.log2L == lg && (int)j.strided == sk && j.ksplit == ks)
                            grp.push_back(&j);
                    for (size_t c0 = 0; c0 < grp.size(); c0 += jt::dev::BATCH_MAX_JOBS) {
                        jt_batch::Launch L;
                        L.fused = true;
                        L.stage = st;
                        L.log2L = lg;
                        L.strided = sk != 0;
                        L.ksplit = ks;
                        L.job_off = (int)hjobs.size();
                        const int ft = jt::f32_warp_tile_fibres(lg);
                        for (size_t q = c0; q < std::min(grp.size(), c0 + jt::dev::BATCH_MAX_JOBS); ++q) {
                            const SweepJob& j = *grp[q];
                            jt::dev::BatchJob bj{};
                            bj.A = b->plans[j.transform]->axes[j.axis].dev;
                            bj.nfib = j.nfib;
                            bj.inner = j.inner;
                            bj.tile_begin = L.total_tiles;
                            bj.slot = (int)L.slot_transform.size();
                            L.slot_transform.push_back(j.transform);
                            L.total_tiles += (j.nfib + ft - 1) / ft;
                            L.cost += j.cost;
                            hjobs.push_back(bj);
                        }
                        L.njobs = (int)hjobs.size() - L.job_off;
                        ls.push_back(L);
                    }
                }
        for (const auto& j : sweeps) {
            if (j.fused || j.stage != st) continue;
            jt_batch::Launch L;
            L.stage = st;
            L.transform = j.transform;
            L.axis = j.axis;
            L.nfib = j.nfib;
            L.inner = j.inner;
            L.ksplit = j.ksplit;
            L.cost = j.cost;
            ls.push_back(L);
        }
        std::stable_sort(ls.begin(), ls.end(), [](const jt_batch::Launch& x, const jt_batch::Launch& y) { return x.cost > y.cost; });
        double load[jt_batch::STREAMS] = {};
        for (auto& L : ls) {
            if (st == 0) {
                L.free = true;
                if (L.fused) {
                    for (int i : L.slot_transform) L.free = L.free && b->plans[i]->d == 1;
                } else {
                    L.free = b->plans[L.transform]->d == 1;
                }
            }
            const int w0 = L.free ? jt_batch::WORKERS : 0, w1 = L.free ? jt_batch::STREAMS : jt_batch::WORKERS;
            int w = w0;
            for (int v = w0 + 1; v < w1; ++v)
                if (load[v] < load[w]) w = v;
            L.worker = w;
            load[w] += L.cost;
            out.push_back(std::move(L));
        }
    }
}

}  // namespace

extern "C" {

jt_status jt_batch_create(jt_batch** out, int count, jt_plan* const* plans, const int64_t* nrhs, jt_stream_t stream) {
    if (!out) return JT_EINVAL;
    *out = nullptr;
    if (count < 1 || !plans || !nrhs) return JT_EINVAL;
    const int prec = plans[0] ? plans[0]->prec : -1;
    if (prec != JT_FP32 && prec != JT_SPLIT) return (prec == JT_FP64_PLAIN) ? JT_ENOTSUP : JT_EINVAL;
    for (int i = 0; i < count; ++i) {
        if (!plans[i] || nrhs[i] < 1) return JT_EINVAL;
        if (plans[i]->prec != prec) return JT_EINVAL;
    }
    // a plan whose sweeps use a work buffer of its own (double-word axes of length 2^14) may
    // appear once: the workers would otherwise run two of its sweeps on that buffer at once
    for (int i = 0; i < count; ++i) {
        bool own_work = false;
        for (const auto& ax : plans[i]->axes) own_work = own_work || (prec == JT_SPLIT && ax.log2L > jt::DW_SMEM_MAX_LOG2L);
        if (!own_work) continue;
        for (int k = 0; k < i; ++k)
            if (plans[k] == plans[i]) return JT_EINVAL;
    }
    jt_batch* b = nullptr;
    try {
        b = new jt_batch();
        b->count = count;
        b->prec = prec;
        b->plans.assign(plans, plans + count);
        b->nrhs.assign(nrhs, nrhs + count);
        int prio_low = 0, prio_high = 0;
        if (cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high) != cudaSuccess) {
            cudaGetLastError();
            prio_high = prio_low = 0;
        }
        for (int w = 0; w < jt_batch::STREAMS; ++w) {
            const int prio = (w < jt_batch::WORKERS) ? prio_low : prio_high;
            if (cudaStreamCreateWithPriority(&b->work[w], cudaStreamNonBlocking, prio) != cudaSuccess ||
                (w < jt_batch::WORKERS && cudaEventCreateWithFlags(&b->ev_stage[w], cudaEventDisableTiming) != cudaSuccess) ||
                cudaEventCreateWithFlags(&b->ev_join[w], cudaEventDisableTiming) != cudaSuccess) {
                cudaGetLastError();
                jt_batch_destroy(b);
                return JT_ECUDA;
            }
        }
        if (cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            jt_batch_destroy(b);
            return JT_ECUDA;
        }
        for (int i = 0; i < count; ++i) {
            if (!plans[i]->autotune) continue;
            const jt_status st = tune_plan(plans[i], nrhs[i], (cudaStream_t)stream);
            if (st != JT_OK) {
                jt_batch_destroy(b);
                return st;
            }
        }
        std::vector<jt::dev::BatchJob> hjobs;  // both directions, offsets global
        for (int dir = 0; dir < 2; ++dir) {
            const bool fwd = dir == 0;
            // sweeps of every transform, last axis first (the order of jt_forward)
            std::vector<SweepJob> sweeps;
            int max_stage = 0;
            for (int i = 0; i < count; ++i) {
                const jt_plan* p = plans[i];
                int64_t total = nrhs[i];
                for (int a = 0; a < p->d; ++a) total *= p->n[a];
                for (int a = p->d - 1, st = 0; a >= 0; --a, ++st) {
                    long long inner = 1;
                    for (int q = a + 1; q < p->d; ++q) inner *= p->n[q];
                    SweepJob j;
                    j.transform = i;
                    j.axis = a;
                    j.stage = st;
                    j.log2L = p->axes[a].log2L;
                    j.strided = inner > 1;
                    j.fused = (prec == JT_FP32) && jt::f32_warp_path(j.log2L);
                    j.nfib = total / p->n[a];
                    j.inner = inner;
                    j.ksplit = sweep_ksplit(p, a, fwd, j.nfib, j.strided);
                    j.cost = (double)j.nfib * (double)std::max(1, p->axes[a].dev.rank) * (double)(int64_t(1) << j.log2L) *
                             (double)std::max(1, j.log2L);
                    sweeps.push_back(j);
                    max_stage = std::max(max_stage, st);
                }
            }
            batch_plan_launches(b, fwd, sweeps, max_stage, hjobs);
        }
        // first use of each kernel instance (attributes, occupancy) here rather than at the
        // first execution, which may be under stream capture: launches of zero tiles
        for (int dir = 0; dir < 2; ++dir)
            for (const auto& L : b->launches[dir]) {
                cudaError_t e;
                if (L.fused) {
                    const jt::dev::BatchPtrs none{};
                    e = jt::launch_axis_f32_batched(L.log2L, dir == 0, L.strided, nullptr, 0, 0, none, L.ksplit,
                                                    (cudaStream_t)stream);
                } else {
                    e = launch_sweep(b->plans[L.transform], L.axis, dir == 0, nullptr, nullptr, 0, L.inner, L.ksplit,
                                     (cudaStream_t)stream);
                }
                if (e != cudaSuccess) {
                    jt_batch_destroy(b);
                    return JT_ECUDA;
                }
            }
        if (!hjobs.empty()) {
            static_assert(std::is_trivially_copyable<jt::dev::BatchJob>::value, "jobs are copied as bytes");
            if (cudaMalloc((void**)&b->d_jobs, sizeof(jt::dev::BatchJob) * hjobs.size()) != cudaSuccess) {
                cudaGetLastError();
                jt_batch_destroy(b);
                return JT_ENOMEM;
            }
            cudaStream_t s = (cudaStream_t)stream;
            if (cudaMemcpyAsync(b->d_jobs, hjobs.data(), sizeof(jt::dev::BatchJob) * hjobs.size(),
                                cudaMemcpyHostToDevice, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess) {
                jt_batch_destroy(b);
                return JT_ECUDA;
            }
        }
    } catch (const std::bad_alloc&) {
        jt_batch_destroy(b);
        return JT_ENOMEM;
    } catch (...) {
        jt_batch_destroy(b);
        return JT_EINVAL;
    }
    *out = b;
    return JT_OK;
}

jt_status jt_batch_forward(jt_batch* batch, const void* const* in, void* const* out, jt_stream_t stream) {
    return batch_run(batch, in, out, true, (cudaStream_t)stream);
}

jt_status jt_batch_adjoint(jt_batch* batch, const void* const* in, void* const* out, jt_stream_t stream) {
    return batch_run(batch, in, out, false, (cudaStream_t)stream);
}

void jt_batch_destroy(jt_batch* batch) {
    if (!batch) return;
    if (batch->d_jobs) cudaFree(batch->d_jobs);
    for (int w = 0; w < jt_batch::STREAMS; ++w) {
        if (batch->work[w]) cudaStreamDestroy(batch->work[w]);
        if (w < jt_batch::WORKERS && batch->ev_stage[w]) cudaEventDestroy(batch->ev_stage[w]);
        if (batch->ev_join[w]) cudaEventDestroy(batch->ev_join[w]);
    }
    if (batch->ev_fork) cudaEventDestroy(batch->ev_fork);
    delete batch;
}

}  // extern "C"

namespace {

// Argument checks of jt_plan_create (JT_OK or the status to return).
jt_status check_plan_args(int d, const int64_t* n, const double* a, const double* b, double eps, const jt_options& o) {
    if (d < 1 || d > 3 || !n || !a || !b) return JT_EINVAL;
    if (o.prec != JT_FP32 && o.prec != JT_SPLIT && o.prec != JT_FP64_PLAIN) return JT_EINVAL;
    if (o.kind != JT_FIRST_KIND && o.kind != JT_SECOND_KIND) return JT_EINVAL;
    if (o.kind == JT_SECOND_KIND && o.prec == JT_FP64_PLAIN) return JT_ENOTSUP;
    const int64_t nmax = (o.prec == JT_SPLIT) ? (int64_t(1) << jt::MAX_LOG2L_DW) : (int64_t(1) << jt::MAX_LOG2L_F32);
    for (int i = 0; i < d; ++i) {
        if (n[i] < 1 || !jt::valid_parameter(a[i]) || !jt::valid_parameter(b[i])) return JT_EINVAL;
        if (n[i] > nmax) return JT_ENOTSUP;
    }
    if (!(eps > 0.0 && eps < 1.0)) return JT_EINVAL;
    return JT_OK;
}

int log2_of(int64_t L) {
    int lg = 0;
    while ((int64_t(1) << lg) < L) ++lg;
    return lg;
}

// Host phase of plan creation: the setup of every axis (no GPU).
jt_status plan_host_setup(jt_plan* plan, int d, const int64_t* n, const double* a, const double* b,
                          const double* const* points, double eps, const jt_options& o) {
    plan->d = d;
    plan->prec = o.prec;
    plan->autotune = o.autotune != 0;
    plan->kind = o.kind;
    plan->axes.resize(d);
    for (int i = 0; i < d; ++i) {
        plan->n[i] = n[i];
        const double* pts = points ? points[i] : nullptr;
        if (pts) plan->all_uniform = false;
        jt_status st = jt::axis_setup(plan->axes[i].host, n[i], a[i], b[i], pts, eps, o);
        if (st != JT_OK) return st;
        plan->axes[i].log2L = log2_of(plan->axes[i].host.L);
    }
    return JT_OK;
}

// Device phase: upload the working-precision tables (or build the plain FP64 resources).
jt_status plan_device_setup(jt_plan* plan, cudaStream_t s) {
    for (auto& ax : plan->axes) {
        jt_status st = JT_OK;
        if (plan->prec == JT_FP32)
            st = build_device_axis<float>(ax, s);
        else if (plan->prec == JT_SPLIT)
            st = build_device_axis<dw>(ax, s);
        if (st != JT_OK) return st;
    }
    if (plan->prec == JT_FP64_PLAIN) {
        std::vector<const jt::AxisTables*> tabs;
        for (auto& ax : plan->axes) tabs.push_back(&ax.host);
        return jt::plain_create(&plan->plain, tabs, s);
    }
    return JT_OK;
}

// Serialised plan: magic, version, plan fields, the tables of each axis, FNV-1a checksum.
const unsigned char PLAN_MAGIC[8] = {'J', 'T', 'P', 'L', 'A', 'N', 0, 1};
constexpr uint32_t PLAN_VERSION = 1;

uint64_t fnv1a(const unsigned char* p, size_t n) {
    uint64_t h = 1469598103934665603ull;
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

template <class T>
void put_raw(std::vector<unsigned char>& out, const T& v) {
    const unsigned char* p = reinterpret_cast<const unsigned char*>(&v);
    out.insert(out.end(), p, p + sizeof(T));
}
template <class T>
bool get_raw(const unsigned char*& p, const unsigned char* end, T& v) {
    if ((size_t)(end - p) < sizeof(T)) return false;
    std::memcpy(&v, p, sizeof(T));
    p += sizeof(T);
    return true;
}

void serialize_plan(const jt_plan* plan, std::vector<unsigned char>& out) {
    out.insert(out.end(), PLAN_MAGIC, PLAN_MAGIC + 8);
    put_raw<uint32_t>(out, PLAN_VERSION);
    put_raw<int32_t>(out, plan->d);
    put_raw<int32_t>(out, plan->prec);
    put_raw<int32_t>(out, plan->kind);
    put_raw<int32_t>(out, plan->autotune ? 1 : 0);
    put_raw<int32_t>(out, plan->all_uniform ? 1 : 0);
    for (int i = 0; i < 3; ++i) put_raw<int64_t>(out, plan->n[i]);
    for (int i = 0; i < plan->d; ++i) jt::serialize_tables(plan->axes[i].host, out);
    put_raw<uint64_t>(out, fnv1a(out.data(), out.size()));
}

// Parse and check a serialised plan into the host fields of *plan (no GPU).
jt_status deserialize_plan(const unsigned char* buf, size_t size, jt_plan* plan) {
    if (!buf || size < 8 + 4 + 8) return JT_EINVAL;
    if (std::memcmp(buf, PLAN_MAGIC, 8) != 0) return JT_EINVAL;
    uint64_t sum = 0;
    std::memcpy(&sum, buf + size - 8, 8);
    if (sum != fnv1a(buf, size - 8)) return JT_EINVAL;
    const unsigned char* p = buf + 8;
    const unsigned char* end = buf + size - 8;
    uint32_t version = 0;
    int32_t d = 0, prec = 0, kind = 0, autotune = 0, uni = 0;
    if (!get_raw(p, end, version) || version != PLAN_VERSION || !get_raw(p, end, d) || !get_raw(p, end, prec) ||
        !get_raw(p, end, kind) || !get_raw(p, end, autotune) || !get_raw(p, end, uni))
        return JT_EINVAL;
    if (d < 1 || d > 3 || (prec != JT_FP32 && prec != JT_SPLIT && prec != JT_FP64_PLAIN)) return JT_EINVAL;
    if ((kind != JT_FIRST_KIND && kind != JT_SECOND_KIND) || (kind == JT_SECOND_KIND && prec == JT_FP64_PLAIN))
        return JT_EINVAL;
    plan->d = d;
    plan->prec = prec;
    plan->kind = kind;
    plan->autotune = autotune != 0;
    plan->all_uniform = uni != 0;
    for (int i = 0; i < 3; ++i)
        if (!get_raw(p, end, plan->n[i])) return JT_EINVAL;
    const int64_t nmax = (prec == JT_SPLIT) ? (int64_t(1) << jt::MAX_LOG2L_DW) : (int64_t(1) << jt::MAX_LOG2L_F32);
    plan->axes.resize(d);
    bool all_uni = true;
    for (int i = 0; i < d; ++i) {
        jt::AxisTables& T = plan->axes[i].host;
        if (!jt::deserialize_tables(p, end, T, nmax)) return JT_EINVAL;
        if (T.n != plan->n[i] || T.kind != kind) return JT_EINVAL;
        all_uni = all_uni && T.uniform;
        plan->axes[i].log2L = log2_of(T.L);
    }
    if (p != end || all_uni != plan->all_uniform) return JT_EINVAL;
    return JT_OK;
}

}  // namespace

extern "C" {

jt_status jt_plan_create(jt_plan** out, int d, const int64_t* n, const double* a, const double* b,
                         const double* const* points, double eps, const jt_options* opt, jt_stream_t stream) {
    if (!out) return JT_EINVAL;
    *out = nullptr;
    jt_options o;
    jt_options_default(&o);
    if (opt) o = *opt;
    jt_status st = check_plan_args(d, n, a, b, eps, o);
    if (st != JT_OK) return st;
    jt_plan* plan = nullptr;
    try {
        plan = new jt_plan();
        st = plan_host_setup(plan, d, n, a, b, points, eps, o);
        if (st == JT_OK) st = plan_device_setup(plan, (cudaStream_t)stream);
    } catch (const std::bad_alloc&) {
        st = JT_ENOMEM;
    } catch (...) {
        st = JT_EINVAL;
    }
    if (st != JT_OK) {
        jt_destroy(plan);
        return st;
    }
    *out = plan;
    return JT_OK;
}

jt_status jt_plan_create_many(int count, jt_plan** out, const jt_plan_desc* descs, jt_stream_t stream) {
    if (count < 0 || (count > 0 && (!out || !descs))) return JT_EINVAL;
    for (int i = 0; i < count; ++i) out[i] = nullptr;
    std::vector<jt_options> opts(count);
    for (int i = 0; i < count; ++i) {
        jt_options_default(&opts[i]);
        if (descs[i].opt) opts[i] = *descs[i].opt;
        const jt_status st = check_plan_args(descs[i].d, descs[i].n, descs[i].a, descs[i].b, descs[i].eps, opts[i]);
        if (st != JT_OK) return st;
    }
    std::vector<jt_plan*> plans(count, nullptr);
    std::vector<jt_status> status(count, JT_OK);
    try {
        for (int i = 0; i < count; ++i) plans[i] = new jt_plan();
        // host setups side by side: W workers, each plan's own setup with hw / W threads
        const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
        const int workers = (int)std::min<unsigned>((unsigned)std::max(count, 1), std::min(hw, 16u));
        const int inner = std::max(1, (int)std::min(hw, 16u) / std::max(workers, 1));
        std::atomic_int next(0);
        auto work = [&]() {
            jt::set_setup_threads(inner);
            for (int i = next.fetch_add(1); i < count; i = next.fetch_add(1)) {
                try {
                    const jt_plan_desc& D = descs[i];
                    const double* const* pts = D.points[0] || D.points[1] || D.points[2] ? D.points : nullptr;
                    status[i] = plan_host_setup(plans[i], D.d, D.n, D.a, D.b, pts, D.eps, opts[i]);
                } catch (const std::bad_alloc&) {
                    status[i] = JT_ENOMEM;
                } catch (...) {
                    status[i] = JT_EINVAL;
                }
            }
        };
        std::vector<std::thread> th;
        for (int w = 1; w < workers; ++w) th.emplace_back(work);
        work();
        for (auto& t : th) t.join();
        for (int i = 0; i < count; ++i)
            if (status[i] == JT_OK) status[i] = plan_device_setup(plans[i], (cudaStream_t)stream);
    } catch (const std::bad_alloc&) {
        for (auto* p : plans) jt_destroy(p);
        return JT_ENOMEM;
    } catch (...) {
        for (auto* p : plans) jt_destroy(p);
        return JT_EINVAL;
    }
    for (int i = 0; i < count; ++i)
        if (status[i] != JT_OK) {
            const jt_status st = status[i];
            for (auto* p : plans) jt_destroy(p);
            return st;
        }
    for (int i = 0; i < count; ++i) out[i] = plans[i];
    return JT_OK;
}

jt_status jt_plan_save(const jt_plan* plan, void* buf, size_t* size) {
    if (!plan || !size) return JT_EINVAL;
    try {
        std::vector<unsigned char> bytes;
        serialize_plan(plan, bytes);
        if (!buf) {
            *size = bytes.size();
            return JT_OK;
        }
        if (*size < bytes.size()) {
            *size = bytes.size();
            return JT_EINVAL;
        }
        std::memcpy(buf, bytes.data(), bytes.size());
        *size = bytes.size();
        return JT_OK;
    } catch (...) {
        return JT_ENOMEM;
    }
}

jt_status jt_plan_load(jt_plan** out, const void* buf, size_t size, jt_stream_t stream) {
    if (!out) return JT_EINVAL;
    *out = nullptr;
    jt_plan* plan = nullptr;
    jt_status st;
    try {
        plan = new jt_plan();
        st = deserialize_plan(static_cast<const unsigned char*>(buf), size, plan);
        if (st == JT_OK) st = plan_device_setup(plan, (cudaStream_t)stream);
    } catch (const std::bad_alloc&) {
        st = JT_ENOMEM;
    } catch (...) {
        st = JT_EINVAL;
    }
    if (st != JT_OK) {
        jt_destroy(plan);
        return st;
    }
    *out = plan;
    return JT_OK;
}

jt_status jt_forward(jt_plan* plan, const void* alpha, void* f, int64_t nrhs, jt_stream_t stream) {
    return apply(plan, alpha, f, nrhs, true, (cudaStream_t)stream);
}

jt_status jt_adjoint(jt_plan* plan, const void* g, void* alpha, int64_t nrhs, jt_stream_t stream) {
    return apply(plan, g, alpha, nrhs, false, (cudaStream_t)stream);
}

jt_status jt_inverse(jt_plan* plan, const void* g, void* alpha, int64_t nrhs, jt_stream_t stream) {
    if (!plan) return JT_EINVAL;
    if (!plan->all_uniform || plan->kind != JT_FIRST_KIND) return JT_ENOTSUP;
    return apply(plan, g, alpha, nrhs, false, (cudaStream_t)stream);
}

jt_status jt_forward_plain_noalloc(jt_plan* plan, const void* alpha, void* f, int64_t nrhs, jt_stream_t stream) {
    if (!plan || !alpha || !f || nrhs < 1) return JT_EINVAL;
    if (plan->prec != JT_FP64_PLAIN) return JT_ENOTSUP;
    if (plan_elements(plan, nrhs) < 1) return JT_EINVAL;
    return jt::plain_apply_static(plan->plain, (const double*)alpha, (double*)f, nrhs, true, (cudaStream_t)stream);
}

jt_status jt_plan_check(jt_plan* plan, jt_stream_t stream) {
    if (!plan) return JT_EINVAL;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return JT_ECUDA;
    bool timed_out = false;
    for (auto& ax : plan->axes) {
        if (!ax.dev.status) continue;
        unsigned w = 0;
        if (cudaMemcpy(&w, ax.dev.status, sizeof(w), cudaMemcpyDeviceToHost) != cudaSuccess) return JT_ECUDA;
        if (w) {
            timed_out = true;
            const unsigned zero = 0;
            if (cudaMemcpy(ax.dev.status, &zero, sizeof(zero), cudaMemcpyHostToDevice) != cudaSuccess) return JT_ECUDA;
        }
    }
    return timed_out ? JT_ETIMEOUT : JT_OK;
}

jt_status jt_plan_inject_wait_timeout(jt_plan* plan, int on) {
    if (!plan) return JT_EINVAL;
    if (plan->prec != JT_FP32) return JT_ENOTSUP;
    for (auto& ax : plan->axes) ax.dev.skip_copy = on ? 1 : 0;
    return JT_OK;
}

jt_status jt_plan_info(const jt_plan* plan, int axis, int* rank, int64_t* fft_len, double* t_out, double* w_out) {
    if (!plan || axis < 0 || axis >= plan->d) return JT_EINVAL;
    const jt::AxisTables& T = plan->axes[axis].host;
    if (rank) *rank = T.rank;
    if (fft_len) *fft_len = T.L;
    if (t_out) std::memcpy(t_out, T.t.data(), sizeof(double) * T.n);
    if (w_out) std::memcpy(w_out, T.w.data(), sizeof(double) * T.n);
    return JT_OK;
}

jt_status jt_plan_set_ksplit(jt_plan* plan, int axis, int direction, int ksplit) {
    if (!plan || axis < -1 || axis >= plan->d || direction < -1 || direction > 1) return JT_EINVAL;
    if (ksplit != 0 && ksplit != 1 && ksplit != 2 && ksplit != 4 && ksplit != 8) return JT_EINVAL;
    if (plan->prec == JT_FP64_PLAIN) return JT_ENOTSUP;
    for (int ax = 0; ax < plan->d; ++ax) {
        if (axis >= 0 && ax != axis) continue;
        for (int dir = 0; dir < 2; ++dir) {
            if (direction >= 0 && dir != direction) continue;
            plan->ksplit_fixed[ax][dir] = ksplit;
            auto& tv = plan->tuned;
            tv.erase(std::remove_if(tv.begin(), tv.end(),
                                    [&](const jt_plan::Tuned& t) { return t.axis == ax && t.fwd == (dir == 0 ? 1 : 0); }),
                     tv.end());
        }
    }
    return JT_OK;
}

jt_status jt_plan_tune(jt_plan* plan, int64_t nrhs, jt_stream_t stream) {
    if (!plan || nrhs < 1) return JT_EINVAL;
    if (plan->prec == JT_FP64_PLAIN) return JT_ENOTSUP;
    try {
        return tune_plan(plan, nrhs, (cudaStream_t)stream);
    } catch (...) {
        return JT_ENOMEM;
    }
}

jt_status jt_plan_schedule(const jt_plan* plan, int axis, int direction, int64_t nrhs, int* ksplit) {
    if (!plan || !ksplit || axis < 0 || axis >= plan->d || direction < 0 || direction > 1 || nrhs < 1) return JT_EINVAL;
    if (plan->prec == JT_FP64_PLAIN) return JT_ENOTSUP;
    const int64_t total = plan_elements(plan, nrhs);
    if (total < 1) return JT_EINVAL;
    long long inner = 1;
    for (int i = axis + 1; i < plan->d; ++i) inner *= plan->n[i];
    *ksplit = sweep_ksplit(plan, axis, direction == 0, total / plan->n[axis], inner > 1);
    return JT_OK;
}

jt_status jt_plan_shape(const jt_plan* plan, int* d, int64_t* n, int* prec, int* kind, int* all_uniform) {
    if (!plan) return JT_EINVAL;
    if (d) *d = plan->d;
    if (n)
        for (int i = 0; i < 3; ++i) n[i] = (i < plan->d) ? plan->n[i] : 1;
    if (prec) *prec = plan->prec;
    if (kind) *kind = plan->kind;
    if (all_uniform) *all_uniform = plan->all_uniform ? 1 : 0;
    return JT_OK;
}

jt_status jt_transform_host(jt_plan* plan, int direction, const void* in_host, void* out_host, int64_t nrhs,
                            void* dev_buf, size_t dev_bytes, jt_stream_t stream) {
    if (!plan || !in_host || !out_host || nrhs < 1 || !dev_buf || direction < 0 || direction > 2) return JT_EINVAL;
    if (plan->prec == JT_FP64_PLAIN) return JT_ENOTSUP;
    if (direction == 2 && (!plan->all_uniform || plan->kind != JT_FIRST_KIND)) return JT_ENOTSUP;
    const int64_t per_elems = plan_elements(plan, 1);
    if (per_elems < 1 || plan_elements(plan, nrhs) < 1) return JT_EINVAL;
    const size_t esz = plan->prec == JT_FP32 ? 4 : 8;
    const size_t per = (size_t)per_elems * esz;
    const int64_t cap = (int64_t)(dev_bytes / per);  // right-hand sides the work area holds
    if (cap < 1) return JT_EINVAL;
    const bool fwd = direction == 0;
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned char* src = static_cast<const unsigned char*>(in_host);
    unsigned char* dst = static_cast<unsigned char*>(out_host);
    unsigned char* buf = static_cast<unsigned char*>(dev_buf);
    auto run_chunk = [&](int64_t r0, int64_t rc, unsigned char* b, cudaStream_t cs) -> jt_status {
        const size_t bytes = (size_t)rc * per;
        if (cudaMemcpyAsync(b, src + (size_t)r0 * per, bytes, cudaMemcpyHostToDevice, cs) != cudaSuccess)
            return JT_ECUDA;
        jt_status st = apply(plan, b, b, rc, fwd, cs);
        if (st != JT_OK) return st;
        if (cudaMemcpyAsync(dst + (size_t)r0 * per, b, bytes, cudaMemcpyDeviceToHost, cs) != cudaSuccess) return JT_ECUDA;
        return JT_OK;
    };
    if (cap < 2) {  // one buffer: chunks one after another on the caller's stream
        for (int64_t r0 = 0; r0 < nrhs; ++r0) {
            jt_status st = run_chunk(r0, 1, buf, s);
            if (st != JT_OK) return st;
        }
        return JT_OK;
    }
    constexpr int P = jt_plan::PIPES;
    const int np = (int)std::min<int64_t>(P, cap);  // streams (and buffers) in use
    {
        std::lock_guard<std::mutex> lock(plan->pipe_mu);
        for (int w = 0; w < P; ++w) {
            if (!plan->pipe[w] && cudaStreamCreateWithFlags(&plan->pipe[w], cudaStreamNonBlocking) != cudaSuccess)
                return JT_ECUDA;
            if (!plan->pipe_done[w] && cudaEventCreateWithFlags(&plan->pipe_done[w], cudaEventDisableTiming) != cudaSuccess)
                return JT_ECUDA;
        }
        if (!plan->pipe_fork && cudaEventCreateWithFlags(&plan->pipe_fork, cudaEventDisableTiming) != cudaSuccess)
            return JT_ECUDA;
    }
    // chunks of at most cap/np right-hand sides, at least 2 np of them when nrhs allows: chunk c
    // runs on stream c % np with its own buffer, so that one chunk's copy in, another's
    // transform and a third's copy out proceed together
    const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(cap / np, (nrhs + 2 * np - 1) / (2 * np)));
    if (cudaEventRecord(plan->pipe_fork, s) != cudaSuccess) return JT_ECUDA;
    for (int w = 0; w < np; ++w)
        if (cudaStreamWaitEvent(plan->pipe[w], plan->pipe_fork, 0) != cudaSuccess) return JT_ECUDA;
    int64_t c = 0;
    for (int64_t r0 = 0; r0 < nrhs; r0 += chunk, ++c) {
        const int w = (int)(c % np);
        jt_status st = run_chunk(r0, std::min(chunk, nrhs - r0), buf + (size_t)w * (size_t)chunk * per, plan->pipe[w]);
        if (st != JT_OK) return st;
    }
    for (int w = 0; w < np; ++w) {
        if (cudaEventRecord(plan->pipe_done[w], plan->pipe[w]) != cudaSuccess) return JT_ECUDA;
        if (cudaStreamWaitEvent(s, plan->pipe_done[w], 0) != cudaSuccess) return JT_ECUDA;
    }
    return JT_OK;
}

void jt_destroy(jt_plan* plan) {
    if (!plan) return;
    for (int w = 0; w < jt_plan::PIPES; ++w) {
        if (plan->pipe[w]) cudaStreamDestroy(plan->pipe[w]);
        if (plan->pipe_done[w]) cudaEventDestroy(plan->pipe_done[w]);
    }
    if (plan->pipe_fork) cudaEventDestroy(plan->pipe_fork);
    for (auto& ax : plan->axes) free_axis(ax);
    if (plan->plain) jt::plain_destroy(plan->plain);
    delete plan;
}

}  // extern "C"
