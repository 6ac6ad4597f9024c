// Small dense complex linear algebra for plan setup (host, FP64): column-pivoted
// Householder QR (pivots only), orthonormal bases by twice-iterated Gram--Schmidt,
// one-sided Jacobi SVD and the SVD-based pseudo-inverse.  These are the building
// blocks of the randomised SVD of Algorithm 2.1 (Sec. 2.1).  Matrices are
// column-major: element (i, j) of an m x n matrix A is A[i + j*m].
#pragma once

#include <algorithm>
#include <cmath>
#include <complex>
#include <numeric>
#include <thread>
#include <vector>

namespace jt {
namespace la {

using cd = std::complex<double>;

// Column indices chosen, in order, by the first k steps of Householder QR with column
// pivoting (Businger--Golub) of the m x n matrix A.  A is taken by value (a work copy).
// The reflection of the trailing columns at each step is split over `threads` host threads
// (the result does not depend on the split: each column is updated by one thread).
inline std::vector<int> qrcp_pivots(std::vector<cd> A, int m, int n, int k, int threads = 1) {
    std::vector<int> perm(n);
    std::iota(perm.begin(), perm.end(), 0);
    std::vector<double> norms(n, 0.0);
    for (int j = 0; j < n; ++j) {
        double s = 0;
        for (int i = 0; i < m; ++i) s += std::norm(A[i + (size_t)j * m]);
        norms[j] = s;
    }
    k = std::min(k, std::min(m, n));
    std::vector<cd> v(m);
    for (int s = 0; s < k; ++s) {
        int p = s;
        for (int j = s + 1; j < n; ++j)
            if (norms[j] > norms[p]) p = j;
        if (p != s) {
            for (int i = 0; i < m; ++i) std::swap(A[i + (size_t)s * m], A[i + (size_t)p * m]);
            std::swap(norms[s], norms[p]);
            std::swap(perm[s], perm[p]);
        }
        double xn = 0;
        for (int i = s; i < m; ++i) xn += std::norm(A[i + (size_t)s * m]);
        xn = std::sqrt(xn);
        if (xn == 0.0) break;
        cd x0 = A[s + (size_t)s * m];
        cd phase = (std::abs(x0) > 0) ? x0 / std::abs(x0) : cd(1.0, 0.0);
        cd alpha = -phase * xn;
        double vn = 0;
        for (int i = s; i < m; ++i) {
            v[i] = A[i + (size_t)s * m];
            if (i == s) v[i] -= alpha;
            vn += std::norm(v[i]);
        }
        if (vn == 0.0) continue;
        auto update = [&](int j0, int j1) {
            for (int j = j0; j < j1; ++j) {
                cd* col = &A[(size_t)j * m];
                cd w = 0;
                for (int i = s; i < m; ++i) w += std::conj(v[i]) * col[i];
                w *= 2.0 / vn;
                double nn = 0;
                for (int i = s; i < m; ++i) {
                    col[i] -= w * v[i];
                    if (i > s) nn += std::norm(col[i]);
                }
                norms[j] = nn;
            }
        };
        const int rest = n - (s + 1);
        const int nt = std::max(1, std::min(threads, rest / 512));
        if (nt <= 1) {
            update(s + 1, n);
        } else {
            std::vector<std::thread> th;
            for (int w = 0; w < nt; ++w)
                th.emplace_back(update, s + 1 + (int)((long long)rest * w / nt), s + 1 + (int)((long long)rest * (w + 1) / nt));
            for (auto& t : th) t.join();
        }
    }
    perm.resize(k);
    return perm;
}

// Orthonormal basis of the range of the m x n matrix A by classical Gram--Schmidt applied
// twice per column; a column whose remainder is at most `drop` times the largest column norm
// of A adds no direction and is left out.  Returns m x k, k <= n the number of columns kept.
// (Padding the basis with arbitrary unit vectors in place of such columns would give it
// directions concentrated on single rows, which a least-squares fit on sampled rows cannot
// see, and the fit would then drop those rows' content.)
inline std::vector<cd> orth(const std::vector<cd>& A, int m, int n, int& k, double drop = 1e-13) {
    double amax = 0;
    for (int j = 0; j < n; ++j) {
        double s = 0;
        for (int i = 0; i < m; ++i) s += std::norm(A[i + (size_t)j * m]);
        amax = std::max(amax, std::sqrt(s));
    }
    std::vector<cd> Q;
    Q.reserve(A.size());
    k = 0;
    std::vector<cd> q(m);
    for (int j = 0; j < n; ++j) {
        for (int i = 0; i < m; ++i) q[i] = A[i + (size_t)j * m];
        for (int pass = 0; pass < 2; ++pass) {
            for (int l = 0; l < k; ++l) {
                const cd* ql = &Q[(size_t)l * m];
                cd d = 0;
                for (int i = 0; i < m; ++i) d += std::conj(ql[i]) * q[i];
                for (int i = 0; i < m; ++i) q[i] -= d * ql[i];
            }
        }
        double nn = 0;
        for (int i = 0; i < m; ++i) nn += std::norm(q[i]);
        nn = std::sqrt(nn);
        if (!(nn > drop * amax) || nn <= 1e-300) continue;
        for (int i = 0; i < m; ++i) Q.push_back(q[i] / nn);
        ++k;
    }
    return Q;
}

// A = U diag(s) V^H, U m x n with orthonormal columns, V n x n unitary,
// s descending.  Each step rotates a column pair so that it becomes orthogonal:
// with g = a_p^H a_q = |g| e^{i phi}, the pair (a_p, e^{-i phi} a_q) has the real
// Gram matrix [[alpha, |g|], [|g|, beta]], diagonalised by the rotation with
// t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), zeta = (beta - alpha) / (2 |g|).
inline void svd_jacobi(const std::vector<cd>& A, int m, int n, std::vector<cd>& U,
                       std::vector<double>& s, std::vector<cd>& V) {
    U = A;
    V.assign((size_t)n * n, cd(0.0, 0.0));
    for (int j = 0; j < n; ++j) V[j + (size_t)j * n] = 1.0;
    const double tol = 1e-15;
    for (int sweep = 0; sweep < 80; ++sweep) {
        bool rotated = false;
        for (int p = 0; p < n - 1; ++p) {
            for (int q = p + 1; q < n; ++q) {
                cd* ap = &U[(size_t)p * m];
                cd* aq = &U[(size_t)q * m];
                double alpha = 0, beta = 0;
                cd g = 0;
                for (int i = 0; i < m; ++i) {
                    alpha += std::norm(ap[i]);
                    beta += std::norm(aq[i]);
                    g += std::conj(ap[i]) * aq[i];
                }
                double ag = std::abs(g);
                if (ag == 0.0 || ag <= tol * std::sqrt(alpha * beta)) continue;
                rotated = true;
                cd ph = std::conj(g) / ag;  // e^{-i phi}
                double zeta = (beta - alpha) / (2.0 * ag);
                double t = (zeta >= 0 ? 1.0 : -1.0) / (std::abs(zeta) + std::sqrt(1.0 + zeta * zeta));
                double c = 1.0 / std::sqrt(1.0 + t * t);
                double sn = c * t;
                for (int i = 0; i < m; ++i) {
                    cd x = ap[i];
                    cd y = aq[i] * ph;
                    ap[i] = c * x - sn * y;
                    aq[i] = sn * x + c * y;
                }
                cd* vp = &V[(size_t)p * n];
                cd* vq = &V[(size_t)q * n];
                for (int i = 0; i < n; ++i) {
                    cd x = vp[i];
                    cd y = vq[i] * ph;
                    vp[i] = c * x - sn * y;
                    vq[i] = sn * x + c * y;
                }
            }
        }
        if (!rotated) break;
    }
    s.assign(n, 0.0);
    for (int j = 0; j < n; ++j) {
        double nn = 0;
        for (int i = 0; i < m; ++i) nn += std::norm(U[i + (size_t)j * m]);
        s[j] = std::sqrt(nn);
    }
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int i, int j) { return s[i] > s[j]; });
    std::vector<cd> U2((size_t)m * n), V2((size_t)n * n);
    std::vector<double> s2(n);
    for (int jj = 0; jj < n; ++jj) {
        int j = order[jj];
        s2[jj] = s[j];
        for (int i = 0; i < m; ++i)
            U2[i + (size_t)jj * m] = (s[j] > 0) ? U[i + (size_t)j * m] / s[j] : cd(0.0, 0.0);
        for (int i = 0; i < n; ++i) V2[i + (size_t)jj * n] = V[i + (size_t)j * n];
    }
    U.swap(U2);
    V.swap(V2);
    s.swap(s2);
}

// Moore--Penrose pseudo-inverse of the m x n matrix A (any shape) through its SVD;
// singular values below rcond * s_max are treated as zero.  Returns n x m.
inline std::vector<cd> pinv(const std::vector<cd>& A, int m, int n, double rcond = 1e-14) {
    bool tall = m >= n;
    std::vector<cd> B;
    int mm = m, nn = n;
    if (!tall) {  // work on A^H (n x m)
        B.assign((size_t)n * m, cd());
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < n; ++j) B[j + (size_t)i * n] = std::conj(A[i + (size_t)j * m]);
        mm = n;
        nn = m;
    } else {
        B = A;
    }
    std::vector<cd> U, V;
    std::vector<double> s;
    svd_jacobi(B, mm, nn, U, s, V);  // B = U S V^H, B^+ = V S^-1 U^H (nn x mm)
    double smax = s.empty() ? 0 : s[0];
    std::vector<cd> P((size_t)nn * mm, cd());
    for (int k = 0; k < nn; ++k) {
        if (s[k] <= rcond * smax || s[k] == 0) continue;
        double inv = 1.0 / s[k];
        for (int j = 0; j < mm; ++j) {
            cd uc = std::conj(U[j + (size_t)k * mm]) * inv;
            for (int i = 0; i < nn; ++i) P[i + (size_t)j * nn] += V[i + (size_t)k * nn] * uc;
        }
    }
    if (tall) return P;  // n x m
    // A^+ = ((A^H)^+)^H : P is m x n here (nn = m, mm = n); return its conjugate transpose
    std::vector<cd> R((size_t)n * m);
    for (int i = 0; i < nn; ++i)
        for (int j = 0; j < mm; ++j) R[j + (size_t)i * mm] = std::conj(P[i + (size_t)j * nn]);
    return R;
}

// C = A (m x k) * B (k x n), column-major.
inline std::vector<cd> matmul(const std::vector<cd>& A, const std::vector<cd>& B, int m, int k, int n) {
    std::vector<cd> C((size_t)m * n, cd());
    for (int j = 0; j < n; ++j)
        for (int l = 0; l < k; ++l) {
            cd bl = B[l + (size_t)j * k];
            if (bl == cd()) continue;
            const cd* a = &A[(size_t)l * m];
            cd* c = &C[(size_t)j * m];
            for (int i = 0; i < m; ++i) c[i] += a[i] * bl;
        }
    return C;
}

}  // namespace la
}  // namespace jt
