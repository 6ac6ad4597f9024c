// Internal declarations shared by the host setup (jt_setup.cpp) and the CUDA side
// (jt_api.cu) of libjt.  Not part of the public C ABI.
#pragma once

#include <complex>
#include <cstdint>
#include <vector>

#include "jt.h"

namespace jt {

using cd = std::complex<double>;

// Host tables of one transform axis (Sec. 3.1).  The plan factorises the row-scaled
// matrix Z = W B (Eq. eq:B; W = diag(sqrt(w_k)) on a uniform axis, I otherwise) as
// Z ~ sum_k u_k v_k^T (Eq. eq:approxA) and keeps the dense low-degree block
// Vblk = W V (Eq. tf:jn, degrees < nu0).
struct AxisTables {
    int64_t n = 0;      // points = degrees
    int64_t L = 0;      // FFT length (power of two >= n)
    int64_t N = 0;      // columns of B: n - nu0
    int nu0 = 0;        // effective split degree, min(nu0, n)
    int rank = 0;       // r
    bool uniform = true;
    int kind = JT_FIRST_KIND;  // second kind: Vblk holds W Q~ and the transform takes Im(B o F)
    double a = 0, b = 0, eps = 0;
    double fact_err = 0;  // sampled relative Frobenius error of sum u_k v_k^T vs Z

    std::vector<double> t, w;          // angles; trigonometric weights (1 if nonuniform)
    std::vector<double> x, rowP, rowQ; // cos t; row scales of p_nu and of h_nu (see jt_setup.cpp)
    std::vector<double> S;             // Stieltjes values PV int w(s)/(x-s) ds at the points
    std::vector<int32_t> m;            // FFT bin of each point
    std::vector<cd> U;                 // rank x n, row k = u_k
    std::vector<cd> V;                 // rank x N, row k = v_k
    std::vector<double> Vblk;          // n x nu0: W P~_c (first kind) or W Q~_c (second kind)
    std::vector<double> sigma;         // kept singular values

    // orthonormal Jacobi recurrence x p_j = sg[j+1] p_{j+1} + beta[j] p_j + sg[j] p_{j-1}
    std::vector<double> beta, sg;
    double p0 = 0;        // p_0 = mu0^{-1/2}
    double sqrt_mu0 = 0;  // mu0^{1/2}
};

// Build the tables of one axis.  points == nullptr selects Gauss--Jacobi nodes.
jt_status axis_setup(AxisTables& out, int64_t n, double a, double b, const double* points,
                     double eps, const jt_options& opt);

// Exact rows of Z = W B by recurrence: out is nrows x N row-major.
void axis_b_rows(const AxisTables& T, const int64_t* rows, int64_t nrows, cd* out);

// Validation shared by the C entry points.
bool valid_parameter(double v);

// Plan serialisation (jt_serialize.cpp): append the tables of one axis to out; read them
// back, checking every size and range (false on a malformed or truncated buffer).
void serialize_tables(const AxisTables& T, std::vector<unsigned char>& out);
bool deserialize_tables(const unsigned char*& p, const unsigned char* end, AxisTables& T, int64_t nmax);

// Recurrence coefficients of the orthonormal Jacobi polynomials, flattened for the GPU setup:
// beta[j], sg[j], isg[j] = 1/sg[j] for j = 0..n+1, and the same in double-word as (hi, lo).
struct SetupRec {
    std::vector<double> beta, sg, isg, betaD, sgD, isgD;
    double p0 = 0, sqrt_mu0 = 0;
};
// GPU versions of the O(n^2) setup steps (jt_setup_gpu.cu, jt_options.setup_device = 1):
// Newton for the Gauss--Jacobi nodes from the initial angles in t (in place) with the
// Christoffel numbers omega, and the sampled columns cl of Z = W B (n x |cl|, column-major).
jt_status gpu_newton_nodes(const SetupRec& H, int64_t n, double maxstep, double* t, double* omega);
struct GpuColumns;  // device copies of the tables the column walks read, made once per setup
GpuColumns* gpu_columns_create(const SetupRec& H, const AxisTables& T);  // nullptr on failure
jt_status gpu_columns(GpuColumns* g, const std::vector<int>& cl, cd* out);
void gpu_columns_destroy(GpuColumns* g);
// The first k pivot columns of Householder QR with column pivoting of the m x n matrix A, held
// row by row (A[i n + j]), on the GPU of that setup; the same steps and roundings as the host
// routine la::qrcp_pivots (which takes the matrix column by column).
jt_status gpu_qrcp_pivots(GpuColumns* g, const cd* A, int m, int n, int k, std::vector<int>& pivots);

// Upper bound on the setup threads of the calling thread (jt_plan_create_many lowers it in
// its workers so that plans set up side by side do not oversubscribe the host).
void set_setup_threads(int n);

}  // namespace jt
