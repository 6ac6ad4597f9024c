// Host-only C entry points of libjt: defaults, status strings and the inspection
// interface to the per-axis setup (no GPU is touched here).
#include <cstring>
#include <exception>
#include <new>

#include "jt_internal.hpp"

struct jt_axis_tables {
    jt::AxisTables T;
};

extern "C" {

void jt_options_default(jt_options* opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->prec = JT_FP32;
    opt->nu0 = 27;
    opt->rank_cap = 0;
    opt->oversample_q = 3;
    opt->seed = 0x1901072750ULL;
    opt->fft_len_policy = 0;
    opt->autotune = 0;
    opt->kind = JT_FIRST_KIND;
    opt->setup_device = 0;
}

const char* jt_status_string(jt_status s) {
    switch (s) {
        case JT_OK: return "JT_OK";
        case JT_EINVAL: return "JT_EINVAL: invalid argument";
        case JT_ENOMEM: return "JT_ENOMEM: allocation failed";
        case JT_ENOTSUP: return "JT_ENOTSUP: operation not supported for this plan";
        case JT_ECUDA: return "JT_ECUDA: CUDA call failed";
        case JT_ETIMEOUT: return "JT_ETIMEOUT: bounded device wait expired";
        case JT_ENOCONV: return "JT_ENOCONV: setup did not converge";
    }
    return "unknown jt_status";
}

jt_status jt_axis_tables_create(jt_axis_tables** out, int64_t n, double a, double b, const double* points,
                                double eps, const jt_options* opt) {
    if (!out) return JT_EINVAL;
    *out = nullptr;
    jt_options o;
    jt_options_default(&o);
    if (opt) o = *opt;
    try {
        jt_axis_tables* h = new jt_axis_tables();
        jt_status st = jt::axis_setup(h->T, n, a, b, points, eps, o);
        if (st != JT_OK) {
            delete h;
            return st;
        }
        *out = h;
        return JT_OK;
    } catch (const std::bad_alloc&) {
        return JT_ENOMEM;
    } catch (...) {
        return JT_EINVAL;
    }
}

jt_status jt_axis_tables_info(const jt_axis_tables* t, int* rank, int64_t* fft_len, int* nu0, double* fact_err) {
    if (!t) return JT_EINVAL;
    if (rank) *rank = t->T.rank;
    if (fft_len) *fft_len = t->T.L;
    if (nu0) *nu0 = t->T.nu0;
    if (fact_err) *fact_err = t->T.fact_err;
    return JT_OK;
}

jt_status jt_axis_tables_copy(const jt_axis_tables* h, double* tt, double* w, int32_t* m, double* u, double* v,
                              double* vblk) {
    if (!h) return JT_EINVAL;
    const jt::AxisTables& T = h->T;
    const int64_t n = T.n;
    if (tt) std::memcpy(tt, T.t.data(), sizeof(double) * n);
    if (w) std::memcpy(w, T.w.data(), sizeof(double) * n);
    if (m) std::memcpy(m, T.m.data(), sizeof(int32_t) * n);
    if (u)
        for (size_t i = 0; i < T.U.size(); ++i) {
            u[2 * i] = T.U[i].real();
            u[2 * i + 1] = T.U[i].imag();
        }
    if (v)
        for (size_t i = 0; i < T.V.size(); ++i) {
            v[2 * i] = T.V[i].real();
            v[2 * i + 1] = T.V[i].imag();
        }
    if (vblk && !T.Vblk.empty()) std::memcpy(vblk, T.Vblk.data(), sizeof(double) * T.Vblk.size());
    return JT_OK;
}

jt_status jt_axis_tables_b_rows(const jt_axis_tables* h, const int64_t* rows, int64_t nrows, double* out) {
    if (!h || (!rows && nrows > 0) || nrows < 0 || (!out && nrows > 0)) return JT_EINVAL;
    const jt::AxisTables& T = h->T;
    for (int64_t i = 0; i < nrows; ++i)
        if (rows[i] < 0 || rows[i] >= T.n) return JT_EINVAL;
    if (T.N == 0 || nrows == 0) return JT_OK;
    try {
        std::vector<jt::cd> buf((size_t)nrows * T.N);
        jt::axis_b_rows(T, rows, nrows, buf.data());
        for (size_t i = 0; i < buf.size(); ++i) {
            out[2 * i] = buf[i].real();
            out[2 * i + 1] = buf[i].imag();
        }
    } catch (...) {
        return JT_ENOMEM;
    }
    return JT_OK;
}

void jt_axis_tables_destroy(jt_axis_tables* t) { delete t; }

}  // extern "C"
