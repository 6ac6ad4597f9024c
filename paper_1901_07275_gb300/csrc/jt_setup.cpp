// Host setup of one transform axis (FP64): Gauss--Jacobi nodes and weights, the
// values of the modified Jacobi functions of both kinds at the points, the bins
// m_j, and the randomised low-rank factorisation of the matrix B (Sec. 2.1,
// Algorithm 2.1; Sec. 3.1, Eqs. eq:B, eq:approxA).
//
// Phase and amplitude.  The paper writes the high-degree block of J as
// Re(B o F) with B_{j,nu} = M(t_j,nu) exp(i(psi(t_j,nu) - 2 pi m_j nu / L)) and
// P~ = M cos(psi), Q~ = M sin(psi) (Eqs. eq:jacnonosci, eq:jacnonosci2).  We never
// need psi or M separately: B_{j,nu} = (P~_nu(t_j) + i Q~_nu(t_j)) e^{-2 pi i m_j nu / L},
// so only P~ and the second-kind Q~ at the points are required.  With p_nu the
// orthonormal Jacobi polynomials and
//     h_nu(x) = PV int_{-1}^{1} w(s) p_nu(s) / (x - s) ds,   w(s) = (1-s)^a (1+s)^b,
// the function h_nu / w solves Jacobi's equation on (-1,1) and h_nu obeys the same
// three-term recurrence as p_nu for nu >= 1, started from h_0 = p_0 S(x),
// S(x) = PV int w(s)/(x-s) ds, and h_1 = ((x - beta_0) h_0 - mu0^{1/2}) / sg_1.
// Q~_nu = kappa 2^{(a+b+1)/2} sin(t/2)^{a+1/2} cos(t/2)^{b+1/2} h_nu(cos t) / w(cos t)
// with kappa = -1/pi gives P~ + i Q~ a non-oscillatory modulus (at a = b = -1/2 it is
// exactly sqrt(2/pi) e^{i nu t}).  Because Re(B o F) equals the high-degree block of J
// for any choice of the imaginary part, the transform stays exact; Q~ only controls
// how low the rank of B is.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <stdexcept>
#include <thread>
#include <vector>

#include "jt_internal.hpp"
#include "jt_linalg.hpp"

// Precision.  Near the ends of (0, pi) the orthonormal recurrence in FP64 loses
// about eps * n / sin(t) relative accuracy, which at n ~ 1e4 exceeds the accuracy
// of the factorisation.  Points with min(t, pi - t) < NEAR_END therefore run every
// recurrence in double-word arithmetic (a pair of doubles: Dekker 1971; Joldes,
// Muller and Popescu, ACM TOMS 2017, "Tight and rigorous error bounds for basic
// building blocks of double-word arithmetic"), with x = cos t formed as 1 - 2 sin^2(t/2)
// or 2 cos^2(t/2) - 1 exactly, and with the recurrence coefficients in double-word.

namespace jt {

static const double PI = 3.14159265358979323846264338327950288;
static const double NEAR_END = 0.35;

bool valid_parameter(double v) { return std::isfinite(v) && v > -1.0 && v < 1.0; }

// ------------------------------------------------------------ double-word numbers
namespace {

struct DD {
    double hi, lo;
};
inline DD two_sum(double a, double b) {
    double s = a + b;
    double bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
inline DD fast_two_sum(double a, double b) {
    double s = a + b;
    return {s, b - (s - a)};
}
inline DD two_prod(double a, double b) {
    double p = a * b;
    return {p, std::fma(a, b, -p)};
}
inline DD operator+(DD a, DD b) {
    DD s = two_sum(a.hi, b.hi);
    DD t = two_sum(a.lo, b.lo);
    DD v = fast_two_sum(s.hi, s.lo + t.hi);
    return fast_two_sum(v.hi, t.lo + v.lo);
}
inline DD operator-(DD a) { return {-a.hi, -a.lo}; }
inline DD operator-(DD a, DD b) { return a + (-b); }
inline DD operator*(DD a, DD b) {
    DD p = two_prod(a.hi, b.hi);
    double t = std::fma(a.hi, b.lo, a.lo * b.hi);
    return fast_two_sum(p.hi, p.lo + t);
}
inline DD operator*(DD a, double b) {
    DD p = two_prod(a.hi, b);
    return fast_two_sum(p.hi, std::fma(a.lo, b, p.lo));
}
inline DD dd(double v) { return {v, 0.0}; }
inline DD operator+(DD a, double b) { return a + dd(b); }
inline DD recip(DD b) {
    double q1 = 1.0 / b.hi;
    DD r = dd(1.0) - b * q1;
    double q2 = r.hi / b.hi;
    r = r - b * q2;
    double q3 = r.hi / b.hi;
    return fast_two_sum(q1, q2) + dd(q3);
}
inline DD dsqrt(DD a) {
    double s = std::sqrt(a.hi);
    DD e = a - two_prod(s, s);
    return fast_two_sum(s, e.hi / (2.0 * s));
}
inline double todouble(double v) { return v; }
inline double todouble(DD v) { return v.hi + v.lo; }

// Recurrence coefficients x p_j = sg[j+1] p_{j+1} + beta[j] p_j + sg[j] p_{j-1} in both
// precisions; isg = 1/sg.  At j = 1 the factor (1+a+b) is cancelled analytically.
struct Coefs {
    std::vector<double> beta, sg, isg;
    std::vector<DD> betaD, sgD, isgD;
    double p0 = 0, sqrt_mu0 = 0;
    Coefs(double a, double b, int64_t n) {
        beta.resize(n + 2);
        sg.assign(n + 2, 0.0);
        isg.assign(n + 2, 0.0);
        betaD.resize(n + 2);
        sgD.assign(n + 2, dd(0));
        isgD.assign(n + 2, dd(0));
        DD A = dd(a), B = dd(b);
        betaD[0] = (B - A) * recip(A + B + dd(2.0));
        for (int64_t j = 1; j <= n + 1; ++j) {
            DD s = two_sum(2.0 * (double)j, a) + B;
            DD num = two_prod(b, b) - two_prod(a, a);
            betaD[j] = num * recip(s * (s + dd(2.0)));
        }
        for (int64_t j = 1; j <= n + 1; ++j) {
            DD q;
            if (j == 1) {
                DD ab2 = A + B + dd(2.0);
                DD num = (dd(1.0) + A) * (dd(1.0) + B) * 4.0;
                q = num * recip(ab2 * ab2 * (A + B + dd(3.0)));
            } else {
                double jj = (double)j;
                DD s = two_sum(2.0 * jj, a) + B;
                DD num = dd(jj) * two_sum(jj, a) * two_sum(jj, b) * (two_sum(jj, a) + B) * 4.0;
                DD den = s * s * (s - dd(1.0)) * (s + dd(1.0));
                q = num * recip(den);
            }
            sgD[j] = dsqrt(q);
            isgD[j] = recip(sgD[j]);
        }
        for (int64_t j = 0; j <= n + 1; ++j) {
            beta[j] = todouble(betaD[j]);
            sg[j] = todouble(sgD[j]);
            isg[j] = (j > 0) ? todouble(isgD[j]) : 0.0;
        }
        double lmu = (a + b + 1.0) * std::log(2.0) + std::lgamma(a + 1.0) + std::lgamma(b + 1.0) -
                     std::lgamma(a + b + 2.0);
        sqrt_mu0 = std::exp(0.5 * lmu);
        p0 = 1.0 / sqrt_mu0;
    }
    const double* b_(double) const { return beta.data(); }
    const DD* b_(DD) const { return betaD.data(); }
    const double* s_(double) const { return sg.data(); }
    const DD* s_(DD) const { return sgD.data(); }
    const double* i_(double) const { return isg.data(); }
    const DD* i_(DD) const { return isgD.data(); }
};

inline bool near_end(double t) { return std::min(t, PI - t) < NEAR_END; }

inline void make_x(double t, double& x) { x = std::cos(t); }
inline void make_x(double t, DD& x) {
    if (t <= 0.5 * PI) {
        double s = std::sin(0.5 * t);
        x = dd(1.0) - two_prod(s, s) * 2.0;
    } else {
        double c = std::cos(0.5 * t);
        x = two_prod(c, c) * 2.0 - dd(1.0);
    }
}

thread_local int g_setup_threads = 16;

template <class F>
void parallel_for(int64_t count, F&& fn) {
    if (count <= 0) return;
    unsigned hw = std::thread::hardware_concurrency();
    int64_t nt = std::max<int64_t>(1, std::min<int64_t>({(int64_t)(hw ? hw : 1), (int64_t)g_setup_threads, count}));
    if (nt == 1) {
        for (int64_t i = 0; i < count; ++i) fn(i);
        return;
    }
    std::vector<std::thread> th;
    std::atomic_int64_t next(0);
    for (int64_t w = 0; w < nt; ++w)
        th.emplace_back([&]() {
            for (int64_t i = next.fetch_add(1); i < count; i = next.fetch_add(1)) fn(i);
        });
    for (auto& t : th) t.join();
}

// p_n, p_n' and sum_{j<n} p_j^2 for a block of points, in lockstep over the points.
template <class R>
void pn_block(const Coefs& C, int64_t n, const R* x, int nb, R* p, double* dp, R* ssq) {
    const R* be = C.b_(R());
    const R* sg = C.s_(R());
    const R* is = C.i_(R());
    const R zero = R(), p0 = R() + C.p0 * 1.0;
    std::vector<R> pm(nb, zero), pc(nb, p0), s(nb, zero);
    std::vector<double> dm(nb, 0.0), dc(nb, 0.0);
    for (int64_t j = 0; j < n; ++j) {
        const R bj = be[j], sj = sg[j], ij = is[j + 1];
        const double bjd = todouble(bj), sjd = todouble(sj), ijd = todouble(ij);
        for (int k = 0; k < nb; ++k) {
            s[k] = s[k] + pc[k] * pc[k];
            R xb = x[k] - bj;
            R pn = (xb * pc[k] - sj * pm[k]) * ij;
            double dn = ((todouble(x[k]) - bjd) * dc[k] + todouble(pc[k]) - sjd * dm[k]) * ijd;
            pm[k] = pc[k];
            pc[k] = pn;
            dm[k] = dc[k];
            dc[k] = dn;
        }
    }
    for (int k = 0; k < nb; ++k) {
        p[k] = pc[k];
        dp[k] = dc[k];
        ssq[k] = s[k];
    }
}

// Newton in t for a block of zeros of p_n(cos t).  The iteration runs in FP64; points near
// the ends (`dw`) then take two more steps with double-word evaluations, the second of
// which also gives the Christoffel number.  FP64 alone converges to within the accuracy of
// its own evaluation, so those two steps are enough to reach a root of the exact polynomial.
void newton_block(const Coefs& C, int64_t n, double maxstep, double* t, double* omega, int nb, bool dw) {
    std::vector<int> act(nb);
    std::iota(act.begin(), act.end(), 0);
    std::vector<double> x(nb), p(nb), s(nb), dp(nb);
    const double tol = dw ? 1e-13 : 2e-16;
    for (int it = 0; it < 40 && !act.empty(); ++it) {
        int na = (int)act.size();
        for (int q = 0; q < na; ++q) make_x(t[act[q]], x[q]);
        pn_block<double>(C, n, x.data(), na, p.data(), dp.data(), s.data());
        std::vector<int> still;
        for (int q = 0; q < na; ++q) {
            int k = act[q];
            double dt = p[q] / (std::sin(t[k]) * dp[q]);
            if (!std::isfinite(dt)) dt = 0.0;
            dt = std::max(-maxstep, std::min(maxstep, dt));
            t[k] += dt;
            if (std::abs(dt) > tol * std::min(t[k], PI - t[k])) still.push_back(k);
        }
        act.swap(still);
    }
    if (!dw) {
        for (int k = 0; k < nb; ++k) make_x(t[k], x[k]);
        pn_block<double>(C, n, x.data(), nb, p.data(), dp.data(), s.data());
        for (int k = 0; k < nb; ++k) omega[k] = 1.0 / s[k];
        return;
    }
    std::vector<DD> xd(nb), pd(nb), sd(nb);
    for (int step = 0; step < 2; ++step) {
        for (int k = 0; k < nb; ++k) make_x(t[k], xd[k]);
        pn_block<DD>(C, n, xd.data(), nb, pd.data(), dp.data(), sd.data());
        for (int k = 0; k < nb; ++k) {
            double dt = todouble(pd[k]) / (std::sin(t[k]) * dp[k]);
            if (step == 0 && std::isfinite(dt) && std::abs(dt) < maxstep) t[k] += dt;
            if (step == 1) omega[k] = 1.0 / todouble(sd[k]);
        }
    }
}

// Serial FP64 evaluation for the bracketing fallback.
void pn_eval(const Coefs& C, int64_t n, double x, double& p, double& dp, double& ssq) {
    double pm = 0, dm = 0, pc = C.p0, dc = 0, s = 0;
    for (int64_t j = 0; j < n; ++j) {
        s += pc * pc;
        double pn = ((x - C.beta[j]) * pc - C.sg[j] * pm) * C.isg[j + 1];
        double dn = ((x - C.beta[j]) * dc + pc - C.sg[j] * dm) * C.isg[j + 1];
        pm = pc;
        pc = pn;
        dm = dc;
        dc = dn;
    }
    p = pc;
    dp = dc;
    ssq = s;
}

// McMahon's expansion of the k-th positive zero of the Bessel function J_nu.
double bessel_zero(double nu, int k) {
    double beta = (k + 0.5 * nu - 0.25) * PI;
    double mu = 4.0 * nu * nu;
    double e8 = 8.0 * beta;
    return beta - (mu - 1.0) / e8 - 4.0 * (mu - 1.0) * (7.0 * mu - 31.0) / (3.0 * e8 * e8 * e8);
}

// Initial angle of the k-th zero of p_n(cos t) (k = 1.., counted from t = 0): a Bessel-type
// estimate near the endpoint, the interior asymptotic phase (Szego 8.21.10) otherwise.
double zero_guess(int64_t n, double a, double b, int64_t k) {
    double rho = n + 0.5 * (a + b + 1.0);
    if (k <= 12) {
        double nu_eff = std::sqrt(rho * rho + (1.0 - a * a - 3.0 * b * b) / 12.0);
        return bessel_zero(a, (int)k) / nu_eff;
    }
    return (k + 0.5 * a - 0.25) * PI / rho;
}

SetupRec flatten(const Coefs& C) {
    SetupRec H;
    H.beta = C.beta;
    H.sg = C.sg;
    H.isg = C.isg;
    for (size_t j = 0; j < C.betaD.size(); ++j) {
        H.betaD.push_back(C.betaD[j].hi);
        H.betaD.push_back(C.betaD[j].lo);
        H.sgD.push_back(C.sgD[j].hi);
        H.sgD.push_back(C.sgD[j].lo);
        H.isgD.push_back(C.isgD[j].hi);
        H.isgD.push_back(C.isgD[j].lo);
    }
    H.p0 = C.p0;
    H.sqrt_mu0 = C.sqrt_mu0;
    return H;
}

bool nodes_newton(const Coefs& C, double a, double b, int64_t n, std::vector<double>& t, std::vector<double>& omega,
                  const SetupRec* gpu, jt_status& gpu_err) {
    const double rho = n + 0.5 * (a + b + 1.0);
    const double maxstep = 0.3 * PI / rho;
    t.resize(n);
    omega.assign(n, 0.0);
    for (int64_t k = 1; k <= n; ++k) {
        if (2 * k <= n + 1)
            t[k - 1] = zero_guess(n, a, b, k);
        else
            t[k - 1] = PI - zero_guess(n, b, a, n + 1 - k);
    }
    if (gpu) {
        gpu_err = gpu_newton_nodes(*gpu, n, maxstep, t.data(), omega.data());
        return gpu_err == JT_OK;
    }
    // blocks of consecutive nodes; end blocks in double-word
    const int BS = 32;
    int64_t nblk = (n + BS - 1) / BS;
    parallel_for(nblk, [&](int64_t ib) {
        int64_t lo = ib * BS, hi = std::min<int64_t>(n, lo + BS);
        bool nearb = false;
        for (int64_t k = lo; k < hi; ++k) nearb = nearb || near_end(t[k]);
        newton_block(C, n, maxstep, &t[lo], &omega[lo], (int)(hi - lo), nearb);
    });
    return true;
}

bool nodes_valid(const Coefs& C, int64_t n, const std::vector<double>& t, const std::vector<double>& omega) {
    double sum = 0;
    for (int64_t k = 0; k < n; ++k) {
        if (!(t[k] > 0.0 && t[k] < PI) || !std::isfinite(omega[k]) || omega[k] <= 0) return false;
        if (k > 0 && !(t[k] > t[k - 1])) return false;
        sum += omega[k];
    }
    return std::abs(sum / (C.sqrt_mu0 * C.sqrt_mu0) - 1.0) < 1e-10;
}

// Robust fallback: bracket sign changes of p_n(cos t) on a grid that is uniform in the
// interior and geometric toward both endpoints, bisect, then polish like the main path.
bool nodes_scan(const Coefs& C, double a, double b, int64_t n, std::vector<double>& t, std::vector<double>& omega) {
    const double rho = n + 0.5 * (a + b + 1.0);
    std::vector<double> grid;
    double h = PI / (16.0 * rho);
    for (double e = h; e > 1e-6 * h; e *= 0.5) grid.push_back(e);
    for (double s = 2 * h; s < PI - 2 * h; s += h) grid.push_back(s);
    for (double e = h; e > 1e-6 * h; e *= 0.5) grid.push_back(PI - e);
    std::sort(grid.begin(), grid.end());
    t.clear();
    double p, dp, ssq, pprev = 0, tprev = 0;
    for (size_t i = 0; i < grid.size(); ++i) {
        pn_eval(C, n, std::cos(grid[i]), p, dp, ssq);
        if (i > 0 && ((p > 0) != (pprev > 0))) {
            double lo = tprev, hi = grid[i], plo = pprev;
            for (int it = 0; it < 200 && hi - lo > 1e-17 * hi; ++it) {
                double mid = 0.5 * (lo + hi), pm;
                pn_eval(C, n, std::cos(mid), pm, dp, ssq);
                if ((pm > 0) == (plo > 0)) {
                    lo = mid;
                    plo = pm;
                } else {
                    hi = mid;
                }
            }
            t.push_back(0.5 * (lo + hi));
        }
        pprev = p;
        tprev = grid[i];
    }
    if ((int64_t)t.size() != n) return false;
    omega.assign(n, 0.0);
    const double maxstep = 1e-3 * h;
    for (int64_t k = 0; k < n; ++k) {
        newton_block(C, n, maxstep, &t[k], &omega[k], 1, near_end(t[k]));
    }
    return true;
}

// -------------------------------------------------------------- Stieltjes values
// S(x) = PV int_{-1}^{1} (1-s)^a (1+s)^b / (x - s) ds
//      = int_{-1}^{1} (w(s) - w(x)) / (x - s) ds + w(x) log((1+x)/(1-x)),
// the remaining integral by the tanh-sinh rule (Takahasi and Mori 1974) on pieces
// whose lengths grow geometrically away from x, so that the branch point of w next
// to x is never closer to a piece than the piece is long.
struct TanhSinh {
    static const int K = 64;  // nodes tau = i h, |i| <= K
    double h = 1.0 / 8.0;
    double e2[2 * K + 1], wgt[2 * K + 1];
    bool pos[2 * K + 1];
    TanhSinh() {
        for (int i = -K; i <= K; ++i) {
            double tau = i * h;
            double u = 0.5 * PI * std::sinh(tau);
            double e = std::exp(-2.0 * std::abs(u));
            e2[i + K] = e;
            pos[i + K] = (u >= 0);
            wgt[i + K] = 0.5 * PI * std::cosh(tau) * 2.0 * e / ((1.0 + e) * (1.0 + e));
        }
    }
    // int over one piece [c, d] of (w(s) - w(x)) / (x - s) ds; the piece is given by its
    // length L = d - c and the exactly formed complements omd = 1 - d, opc = 1 + c and
    // xmd = x - d, so that 1 - s, 1 + s and x - s never suffer cancellation.
    double piece(double L, double omd, double opc, double xmd, double a, double b, double wx) const {
        double sum = 0;
        for (int i = 0; i <= 2 * K; ++i) {
            double e = e2[i];
            double wg = L * wgt[i];
            if (wg == 0.0) continue;
            double smc = pos[i] ? L / (1.0 + e) : L * e / (1.0 + e);  // s - c
            double dms = pos[i] ? L * e / (1.0 + e) : L / (1.0 + e);  // d - s
            double oms = omd + dms, ops = opc + smc, xms = xmd + dms;
            if (oms <= 0 || ops <= 0 || xms == 0) continue;
            double g = (std::exp(a * std::log(oms) + b * std::log(ops)) - wx) / xms * wg;
            if (std::isfinite(g)) sum += g;
        }
        return h * sum;
    }
    // omx = 1 - x and opx = 1 + x, both accurate (x itself is never used).
    double stieltjes(double omx, double opx, double a, double b) const {
        const double wx = std::exp(a * std::log(omx) + b * std::log(opx));
        double tot = 0;
        if (omx <= opx) {
            // x near +1: the side [-1, x] sees the branch point s = 1 at distance 1 - x from
            // its right end, so it is cut into pieces that double in length away from x.
            tot += piece(omx, 0.0, opx, -omx, a, b, wx);  // [x, 1]
            double ylo = omx, step = omx;                 // current piece: 1 - d = ylo
            while (ylo + step < 2.0 - step) {
                tot += piece(step, ylo, 2.0 - (ylo + step), ylo - omx, a, b, wx);
                ylo += step;
                step *= 2.0;
            }
            tot += piece(2.0 - ylo, ylo, 0.0, ylo - omx, a, b, wx);  // [-1, 1 - ylo]
        } else {
            tot += piece(opx, omx, 0.0, 0.0, a, b, wx);  // [-1, x]
            double zlo = opx, step = opx;                // current piece: 1 + c = zlo
            while (zlo + step < 2.0 - step) {
                tot += piece(step, 2.0 - (zlo + step), zlo, opx - (zlo + step), a, b, wx);
                zlo += step;
                step *= 2.0;
            }
            tot += piece(2.0 - zlo, 0.0, zlo, -omx, a, b, wx);  // [-1 + zlo, 1]
        }
        return tot + wx * std::log(opx / omx);
    }
};

// ------------------------------------------------------------ entries of Z = W B
struct Sampler {  // SplitMix64 (Steele, Lea and Flood, OOPSLA 2014)
    uint64_t s;
    uint64_t next() {
        uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        return z ^ (z >> 31);
    }
    // `count` distinct indices of [0, total) not in `exclude`, ascending.
    std::vector<int> pick(int total, int count, const std::vector<int>& exclude) {
        std::vector<char> taken(total, 0);
        for (int e : exclude) taken[e] = 1;
        std::vector<int> pool;
        pool.reserve(total);
        for (int i = 0; i < total; ++i)
            if (!taken[i]) pool.push_back(i);
        count = std::min<int>(count, (int)pool.size());
        for (int i = 0; i < count; ++i) {
            int j = i + (int)(next() % (uint64_t)(pool.size() - i));
            std::swap(pool[i], pool[j]);
        }
        pool.resize(count);
        std::sort(pool.begin(), pool.end());
        return pool;
    }
};

// Entry (j, c) of Z = W B (Eq. eq:B with the row scale W):
//   (rowP_j p_nu(x_j) + i rowQ_j h_nu(x_j)) e^{-2 pi i m_j nu / L},   nu = nu0 + c.
struct Entries {
    const AxisTables& T;
    const Coefs& C;
    GpuColumns* gpu = nullptr;        // columns on the GPU (setup_device = 1)
    mutable jt_status gpu_err = JT_OK;
    std::vector<cd> phase;  // e^{-2 pi i r / L}
    Entries(const AxisTables& T_, const Coefs& C_) : T(T_), C(C_) {
        phase.resize(T.L);
        for (int64_t r = 0; r < T.L; ++r) {
            double ang = -2.0 * PI * (double)r / (double)T.L;
            phase[r] = cd(std::cos(ang), std::sin(ang));
        }
    }
    cd ph(int64_t j, int64_t nu) const { return phase[((int64_t)T.m[j] * nu) % T.L]; }

    // Walk nu = 0..last for the points js[0..nb) in lockstep; emit(k, nu, p, h) for nu >= nu0.
    template <class R, class Emit>
    void walk(const int64_t* js, int nb, int64_t last, Emit&& emit) const {
        const R* be = C.b_(R());
        const R* sg = C.s_(R());
        const R* is = C.i_(R());
        std::vector<R> x(nb), pm(nb), pc(nb), hm(nb), hc(nb);
        const R p0 = R() + C.p0 * 1.0;
        for (int k = 0; k < nb; ++k) {
            make_x(T.t[js[k]], x[k]);
            pm[k] = R();
            pc[k] = p0;
            hm[k] = R();
            hc[k] = R() + C.p0 * T.S[js[k]];
        }
        const R sm = R() + C.sqrt_mu0;
        for (int64_t nu = 0; nu <= last; ++nu) {
            if (nu >= T.nu0)
                for (int k = 0; k < nb; ++k) emit(k, nu, todouble(pc[k]), todouble(hc[k]));
            if (nu == last) break;
            const R bt = be[nu], s0 = sg[nu], i1 = is[nu + 1];
            for (int k = 0; k < nb; ++k) {
                R xb = x[k] - bt;
                R pn, hn;
                if (nu == 0) {
                    pn = xb * pc[k] * i1;
                    hn = (xb * hc[k] - sm) * i1;
                } else {
                    pn = (xb * pc[k] - s0 * pm[k]) * i1;
                    hn = (xb * hc[k] - s0 * hm[k]) * i1;
                }
                pm[k] = pc[k];
                pc[k] = pn;
                hm[k] = hc[k];
                hc[k] = hn;
            }
        }
    }

    // full rows: out[i*N + c]
    void rows(const int64_t* idx, int64_t nr, cd* out) const {
        const int64_t N = T.N;
        parallel_for(nr, [&](int64_t i) {
            int64_t j = idx[i];
            cd* o = out + i * N;
            auto emit = [&](int, int64_t nu, double p, double h) {
                o[nu - T.nu0] = cd(T.rowP[j] * p, T.rowQ[j] * h) * ph(j, nu);
            };
            if (near_end(T.t[j]))
                walk<DD>(&j, 1, T.n - 1, emit);
            else
                walk<double>(&j, 1, T.n - 1, emit);
        });
    }

    // columns with ascending indices cl: out is n x |cl| column-major
    void cols(const std::vector<int>& cl, cd* out) const {
        const int64_t n = T.n;
        if (cl.empty()) return;
        if (gpu) {
            const jt_status st = gpu_columns(gpu, cl, out);
            if (st != JT_OK) gpu_err = st;
            return;
        }
        std::vector<int> slot(T.N, -1);
        for (size_t q = 0; q < cl.size(); ++q) slot[cl[q]] = (int)q;
        const int64_t last = T.nu0 + cl.back();
        const int BS = 64;
        int64_t nblk = (n + BS - 1) / BS;
        parallel_for(nblk, [&](int64_t ib) {
            int64_t lo = ib * BS, hi = std::min<int64_t>(n, lo + BS);
            std::vector<int64_t> js;
            bool nearb = false;
            for (int64_t j = lo; j < hi; ++j) {
                js.push_back(j);
                nearb = nearb || near_end(T.t[j]);
            }
            auto emit = [&](int k, int64_t nu, double p, double h) {
                int q = slot[nu - T.nu0];
                if (q < 0) return;
                int64_t j = js[k];
                out[j + (size_t)q * n] = cd(T.rowP[j] * p, T.rowQ[j] * h) * ph(j, nu);
            };
            if (nearb)
                walk<DD>(js.data(), (int)js.size(), last, emit);
            else
                walk<double>(js.data(), (int)js.size(), last, emit);
        });
    }
};

std::vector<int> unite(std::vector<int> a, const std::vector<int>& b) {
    a.insert(a.end(), b.begin(), b.end());
    std::sort(a.begin(), a.end());
    a.erase(std::unique(a.begin(), a.end()), a.end());
    return a;
}

// Algorithm 2.1 (Sec. 2.1) with rank parameter r and oversampling q.  Returns u_k (rows of
// Uk, length n) and v_k (rows of Vk, length N) with Z ~ sum_k u_k v_k^T: u_k = sqrt(s_k) U0[:,k],
// v_k = sqrt(s_k) V0^*[k,:] (Eq. eq:approxA), keeping s_k > eps * s_1.
void randomized_svd(const AxisTables& T, const Entries& E, int r, int q, Sampler& rng, double eps,
                    std::vector<cd>& Uk, std::vector<cd>& Vk, std::vector<double>& sig, bool& saturated) {
    const int n = (int)T.n, N = (int)T.N;
    const int nr = std::min(n, r * q), ncs = std::min(N, r * q);
    std::vector<int> Prow, Pcol, J;
    std::vector<cd> Cm;
    for (int it = 0; it < 2; ++it) {  // steps 2-3, iterated twice
        std::vector<int> I = unite(rng.pick(n, nr, Prow), Prow);
        std::vector<int64_t> I64(I.begin(), I.end());
        std::vector<cd> rowsI((size_t)I.size() * N);
        E.rows(I64.data(), (int64_t)I.size(), rowsI.data());
        if (E.gpu) {
            // on the GPU of the setup: Z_{I,:} as it comes, row by row
            const jt_status st = gpu_qrcp_pivots(E.gpu, rowsI.data(), (int)I.size(), N, std::min(r, (int)I.size()), Pcol);
            if (st != JT_OK) E.gpu_err = st;
        } else {
            std::vector<cd> A((size_t)I.size() * N);  // Z_{I,:}, |I| x N
            for (size_t i = 0; i < I.size(); ++i)
                for (int c = 0; c < N; ++c) A[i + (size_t)c * I.size()] = rowsI[i * (size_t)N + c];
            Pcol = la::qrcp_pivots(std::move(A), (int)I.size(), N, std::min(r, (int)I.size()), g_setup_threads);
        }
        J = unite(rng.pick(N, ncs, Pcol), Pcol);
        Cm.assign((size_t)n * J.size(), cd());
        E.cols(J, Cm.data());
        // Z_{:,J}^H: pivoted LQ of Z_{:,J}
        if (E.gpu) {
            std::vector<cd> Chr((size_t)J.size() * n);  // row c: conj(Z_{:,J[c]})
            for (size_t q = 0; q < Chr.size(); ++q) Chr[q] = std::conj(Cm[q]);
            const jt_status st = gpu_qrcp_pivots(E.gpu, Chr.data(), (int)J.size(), n, std::min(r, (int)J.size()), Prow);
            if (st != JT_OK) E.gpu_err = st;
        } else {
            std::vector<cd> Ch((size_t)J.size() * n);
            for (int j = 0; j < n; ++j)
                for (size_t c = 0; c < J.size(); ++c) Ch[c + (size_t)j * J.size()] = std::conj(Cm[j + c * (size_t)n]);
            Prow = la::qrcp_pivots(std::move(Ch), (int)J.size(), n, std::min(r, (int)J.size()), g_setup_threads);
        }
    }
    // step 5: orthonormal bases of Z_{:,Pcol} and Z_{Prow,:}^* (only the directions these
    // samples really have: kc <= |Pcol|, kr <= |Prow|)
    const int pc = (int)Pcol.size(), pr = (int)Prow.size();
    std::vector<cd> Zc((size_t)n * pc);
    for (int c = 0; c < pc; ++c) {
        size_t pos = std::lower_bound(J.begin(), J.end(), Pcol[c]) - J.begin();
        std::copy(Cm.begin() + pos * n, Cm.begin() + (pos + 1) * n, Zc.begin() + (size_t)c * n);
    }
    // directions below this fraction of the largest sampled column are rounding noise
    const double drop = std::max(1e-15, std::min(1e-13, 1e-2 * eps));
    int kc = 0, kr = 0;
    std::vector<cd> Qcol = la::orth(Zc, n, pc, kc, drop);
    std::vector<int64_t> Pr64(Prow.begin(), Prow.end());
    std::vector<cd> rowsP((size_t)pr * N);
    E.rows(Pr64.data(), pr, rowsP.data());
    std::vector<cd> Zrh((size_t)N * pr);
    for (int i = 0; i < pr; ++i)
        for (int c = 0; c < N; ++c) Zrh[c + (size_t)i * N] = std::conj(rowsP[(size_t)i * N + c]);
    std::vector<cd> Qrow = la::orth(Zrh, N, pr, kr, drop);
    if (kc == 0 || kr == 0) {  // Z vanishes on every sample: nothing to keep
        saturated = false;
        sig.clear();
        Uk.clear();
        Vk.clear();
        return;
    }
    // step 6: middle matrix by least squares on fresh samples
    std::vector<int> I2 = unite(rng.pick(n, nr, Prow), Prow);
    std::vector<int> J2 = unite(rng.pick(N, ncs, Pcol), Pcol);
    std::vector<int64_t> I264(I2.begin(), I2.end());
    std::vector<cd> rowsI2((size_t)I2.size() * N);
    E.rows(I264.data(), (int64_t)I2.size(), rowsI2.data());
    const int mi = (int)I2.size(), mj = (int)J2.size();
    std::vector<cd> ZIJ((size_t)mi * mj);
    for (int i = 0; i < mi; ++i)
        for (int c = 0; c < mj; ++c) ZIJ[i + (size_t)c * mi] = rowsI2[(size_t)i * N + J2[c]];
    std::vector<cd> QcI((size_t)mi * kc);
    for (int c = 0; c < kc; ++c)
        for (int i = 0; i < mi; ++i) QcI[i + (size_t)c * mi] = Qcol[I2[i] + (size_t)c * n];
    std::vector<cd> QrJh((size_t)kr * mj);
    for (int c = 0; c < mj; ++c)
        for (int k = 0; k < kr; ++k) QrJh[k + (size_t)c * kr] = std::conj(Qrow[J2[c] + (size_t)k * N]);
    std::vector<cd> P1 = la::pinv(QcI, mi, kc);   // kc x mi
    std::vector<cd> P2 = la::pinv(QrJh, kr, mj);  // mj x kr
    std::vector<cd> M = la::matmul(la::matmul(P1, ZIJ, kc, mi, mj), P2, kc, mj, kr);  // kc x kr
    // step 7: SVD of the middle matrix
    std::vector<cd> Um, Vm;  // M = Um S Vm^H, Um kc x kmin, Vm kr x kmin
    std::vector<double> s;
    const int kmin = std::min(kc, kr);
    if (kc >= kr) {
        la::svd_jacobi(M, kc, kr, Um, s, Vm);
    } else {
        std::vector<cd> Mh((size_t)kr * kc);
        for (int i = 0; i < kc; ++i)
            for (int j = 0; j < kr; ++j) Mh[j + (size_t)i * kr] = std::conj(M[i + (size_t)j * kc]);
        la::svd_jacobi(Mh, kr, kc, Vm, s, Um);
    }
    int keep = 0;
    while (keep < kmin && s[keep] > eps * s[0] && s[keep] > 0) ++keep;
    // every sampled direction kept although none was left out as noise: the rank may exceed r
    // (a full-rank Z is exact, not saturated)
    saturated = (keep == kmin) && kc == pc && kr == pr && kmin < std::min(n, N);
    sig.assign(s.begin(), s.begin() + keep);
    Uk.assign((size_t)keep * n, cd());
    Vk.assign((size_t)keep * N, cd());
    for (int k = 0; k < keep; ++k) {
        double rs = std::sqrt(s[k]);
        for (int i = 0; i < n; ++i) {
            cd acc = 0;
            for (int l = 0; l < kc; ++l) acc += Qcol[i + (size_t)l * n] * Um[l + (size_t)k * kc];
            Uk[(size_t)k * n + i] = acc * rs;
        }
        for (int c = 0; c < N; ++c) {
            cd acc = 0;
            for (int l = 0; l < kr; ++l) acc += Qrow[c + (size_t)l * N] * Vm[l + (size_t)k * kr];
            Vk[(size_t)k * N + c] = std::conj(acc) * rs;
        }
    }
}

}  // namespace

void axis_b_rows(const AxisTables& T, const int64_t* rows, int64_t nrows, cd* out) {
    Coefs C(T.a, T.b, T.n);
    Entries E(T, C);
    E.rows(rows, nrows, out);
}

jt_status axis_setup(AxisTables& T, int64_t n, double a, double b, const double* points, double eps,
                     const jt_options& opt) {
    if (n < 1 || n > 65536 || !valid_parameter(a) || !valid_parameter(b)) return JT_EINVAL;
    if (!(eps > 0.0 && eps < 1.0)) return JT_EINVAL;
    if (opt.nu0 < 0 || opt.nu0 > 32 || opt.oversample_q < 1 || opt.rank_cap < 0 || opt.fft_len_policy != 0 || opt.autotune < 0 || opt.autotune > 1 ||
        (opt.kind != JT_FIRST_KIND && opt.kind != JT_SECOND_KIND) || opt.setup_device < 0 || opt.setup_device > 1)
        return JT_EINVAL;
    if (points)
        for (int64_t k = 0; k < n; ++k)
            if (!(std::isfinite(points[k]) && points[k] > 0.0 && points[k] < PI)) return JT_EINVAL;
    T = AxisTables();
    T.n = n;
    T.a = a;
    T.b = b;
    T.eps = eps;
    T.uniform = (points == nullptr);
    T.L = 1;
    while (T.L < n) T.L <<= 1;
    T.nu0 = (int)std::min<int64_t>(opt.nu0, n);
    T.N = n - T.nu0;
    Coefs C(a, b, n);
    SetupRec gpu_flat;
    const SetupRec* gpu_rec = nullptr;
    if (opt.setup_device == 1) {
        gpu_flat = flatten(C);
        gpu_rec = &gpu_flat;
    }
    T.beta = C.beta;
    T.sg = C.sg;
    T.p0 = C.p0;
    T.sqrt_mu0 = C.sqrt_mu0;

    // points and weights
    std::vector<double> omega;
    if (T.uniform) {
        if (n == 1) {
            T.t.assign(1, std::acos(C.beta[0]));
            omega.assign(1, C.sqrt_mu0 * C.sqrt_mu0);
        } else {
            jt_status gerr = JT_OK;
            bool ok = nodes_newton(C, a, b, n, T.t, omega, gpu_rec, gerr) && nodes_valid(C, n, T.t, omega);
            if (gerr != JT_OK) return gerr;
            if (!ok) ok = nodes_scan(C, a, b, n, T.t, omega) && nodes_valid(C, n, T.t, omega);
            if (!ok) return JT_ENOCONV;
        }
    } else {
        T.t.assign(points, points + n);
    }
    T.x.resize(n);
    T.w.resize(n);
    T.rowP.resize(n);
    T.rowQ.resize(n);
    T.m.resize(n);
    const double kappa = -1.0 / PI;
    for (int64_t j = 0; j < n; ++j) {
        double t = T.t[j];
        double s2 = std::sin(0.5 * t), c2 = std::cos(0.5 * t);
        T.x[j] = std::cos(t);
        double lw = a * std::log(2.0 * s2 * s2) + b * std::log(2.0 * c2 * c2);  // log w(x)
        if (T.uniform) {
            T.w[j] = omega[j] * std::exp(-(a + b + 1.0) * std::log(2.0) - (2.0 * a + 1.0) * std::log(s2) -
                                         (2.0 * b + 1.0) * std::log(c2));
            T.rowP[j] = std::sqrt(omega[j]);  // sqrt(w_j) P~_nu(t_j) = sqrt(omega_j) p_nu(x_j)
        } else {
            T.w[j] = 1.0;
            T.rowP[j] = std::exp(0.5 * (a + b + 1.0) * std::log(2.0) + (a + 0.5) * std::log(s2) +
                                 (b + 0.5) * std::log(c2));
        }
        T.rowQ[j] = kappa * T.rowP[j] * std::exp(-lw);
        int64_t mj = std::llround(t * (double)T.L / (2.0 * PI));
        T.m[j] = (int32_t)std::max<int64_t>(0, std::min<int64_t>(mj, T.L / 2));
    }
    T.kind = opt.kind;
    // Stieltjes values for h_0 = p_0 S (the imaginary part of B, and the second-kind block)
    if (T.N > 0 || T.kind == JT_SECOND_KIND) {
        T.S.resize(n);
        TanhSinh ts;
        parallel_for(n, [&](int64_t j) {
            double s2 = std::sin(0.5 * T.t[j]), c2 = std::cos(0.5 * T.t[j]);
            T.S[j] = ts.stieltjes(2.0 * s2 * s2, 2.0 * c2 * c2, a, b);
        });
    }
    // dense low-degree block W V (Eq. tf:jn), by the same recurrence: rowP p_c (first kind)
    // or rowQ h_c, with h_1 = ((x - beta_0) h_0 - mu0^{1/2}) / sg_1 (second kind)
    T.Vblk.assign((size_t)n * T.nu0, 0.0);
    if (T.nu0 > 0)
        parallel_for(n, [&](int64_t j) {
            DD x;
            make_x(T.t[j], x);
            const bool second = T.kind == JT_SECOND_KIND;
            DD pm = dd(0), pc = second ? dd(C.p0) * T.S[j] : dd(C.p0);
            const double row = second ? T.rowQ[j] : T.rowP[j];
            for (int c = 0; c < T.nu0; ++c) {
                T.Vblk[(size_t)j * T.nu0 + c] = row * todouble(pc);
                DD pn = (x - C.betaD[c]) * pc - C.sgD[c] * pm;
                if (second && c == 0) pn = pn - dd(C.sqrt_mu0);
                pn = pn * C.isgD[c + 1];
                pm = pc;
                pc = pn;
            }
        });
    if (T.N == 0) {
        T.rank = 0;
        return JT_OK;
    }

    Entries E(T, C);
    struct ColsGuard {
        GpuColumns* g = nullptr;
        ~ColsGuard() { gpu_columns_destroy(g); }
    } cols_guard;
    if (gpu_rec) {
        cols_guard.g = gpu_columns_create(*gpu_rec, T);
        if (!cols_guard.g) return JT_ECUDA;
        E.gpu = cols_guard.g;
    }
    int cap = opt.rank_cap;
    if (cap <= 0) cap = std::max<int>(64, (int)std::ceil(2.0 * std::log2((double)n)));
    cap = (int)std::min<int64_t>(cap, std::min<int64_t>(n, T.N));
    int r = std::min(cap, eps >= 1e-9 ? 24 : 40);
    Sampler rng{opt.seed ^ 0x6a09e667f3bcc909ULL};
    const double tol = std::max(20.0 * eps, 1e-13);
    for (;;) {
        std::vector<cd> Uk, Vk;
        std::vector<double> sig;
        bool saturated = false;
        randomized_svd(T, E, r, opt.oversample_q, rng, eps, Uk, Vk, sig, saturated);
        if (E.gpu_err != JT_OK) return E.gpu_err;
        const int k = (int)sig.size();
        // relative error on fresh rows, always including both end rows
        std::vector<int> chk = unite(rng.pick((int)n, 24, {}), {0, (int)n - 1});
        std::vector<int64_t> c64(chk.begin(), chk.end());
        std::vector<cd> Z((size_t)chk.size() * T.N);
        E.rows(c64.data(), (int64_t)chk.size(), Z.data());
        double num = 0, den = 0;
        for (size_t i = 0; i < chk.size(); ++i)
            for (int64_t c = 0; c < T.N; ++c) {
                cd approx = 0;
                for (int l = 0; l < k; ++l) approx += Uk[(size_t)l * n + chk[i]] * Vk[(size_t)l * T.N + c];
                cd z = Z[i * (size_t)T.N + c];
                num += std::norm(z - approx);
                den += std::norm(z);
            }
        double err = (den > 0) ? std::sqrt(num / den) : 0.0;
        bool ok = !saturated && err <= tol;
        if (ok || r >= cap) {
            // at the cap, the sampled check decides: a rank that reaches eps on it is kept even
            // if every sampled direction was kept; one that misses it is not convergence
            if (!(err <= tol)) return JT_ENOCONV;
            T.rank = k;
            T.U.swap(Uk);
            T.V.swap(Vk);
            T.sigma.swap(sig);
            T.fact_err = err;
            return JT_OK;
        }
        r = std::min(cap, 2 * r);
    }
}

void set_setup_threads(int n) { g_setup_threads = n < 1 ? 1 : (n > 16 ? 16 : n); }

}  // namespace jt
