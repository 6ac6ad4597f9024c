// Byte layout of the host tables of one axis, for plan serialisation (jt_plan_save /
// jt_plan_load): everything the setup computed, so that a loaded plan needs no setup work
// and uploads exactly the same device tables.  Little-endian host order (x86-64 and
// aarch64 alike); every vector is a 64-bit element count followed by its raw elements.
#include <cstring>

#include "jt_internal.hpp"

namespace jt {
namespace {

template <class T>
void put(std::vector<unsigned char>& out, const T& v) {
    const unsigned char* p = reinterpret_cast<const unsigned char*>(&v);
    out.insert(out.end(), p, p + sizeof(T));
}
template <class T>
void put_vec(std::vector<unsigned char>& out, const std::vector<T>& v) {
    put<uint64_t>(out, (uint64_t)v.size());
    const unsigned char* p = reinterpret_cast<const unsigned char*>(v.data());
    out.insert(out.end(), p, p + sizeof(T) * v.size());
}
template <class T>
bool get(const unsigned char*& p, const unsigned char* end, T& v) {
    if ((size_t)(end - p) < sizeof(T)) return false;
    std::memcpy(&v, p, sizeof(T));
    p += sizeof(T);
    return true;
}
template <class T>
bool get_vec(const unsigned char*& p, const unsigned char* end, std::vector<T>& v, uint64_t max_count) {
    uint64_t c = 0;
    if (!get(p, end, c) || c > max_count || (uint64_t)(end - p) / sizeof(T) < c) return false;
    v.resize((size_t)c);
    std::memcpy(v.data(), p, sizeof(T) * (size_t)c);
    p += sizeof(T) * (size_t)c;
    return true;
}

}  // namespace

void serialize_tables(const AxisTables& T, std::vector<unsigned char>& out) {
    put<int64_t>(out, T.n);
    put<int64_t>(out, T.L);
    put<int64_t>(out, T.N);
    put<int32_t>(out, T.nu0);
    put<int32_t>(out, T.rank);
    put<int32_t>(out, T.uniform ? 1 : 0);
    put<int32_t>(out, T.kind);
    put<double>(out, T.a);
    put<double>(out, T.b);
    put<double>(out, T.eps);
    put<double>(out, T.fact_err);
    put<double>(out, T.p0);
    put<double>(out, T.sqrt_mu0);
    put_vec(out, T.t);
    put_vec(out, T.w);
    put_vec(out, T.x);
    put_vec(out, T.rowP);
    put_vec(out, T.rowQ);
    put_vec(out, T.S);
    put_vec(out, T.m);
    put_vec(out, T.U);
    put_vec(out, T.V);
    put_vec(out, T.Vblk);
    put_vec(out, T.sigma);
    put_vec(out, T.beta);
    put_vec(out, T.sg);
}

bool deserialize_tables(const unsigned char*& p, const unsigned char* end, AxisTables& T, int64_t nmax) {
    int32_t nu0 = 0, rank = 0, uni = 0, kind = 0;
    if (!get(p, end, T.n) || !get(p, end, T.L) || !get(p, end, T.N) || !get(p, end, nu0) || !get(p, end, rank) ||
        !get(p, end, uni) || !get(p, end, kind) || !get(p, end, T.a) || !get(p, end, T.b) || !get(p, end, T.eps) ||
        !get(p, end, T.fact_err) || !get(p, end, T.p0) || !get(p, end, T.sqrt_mu0))
        return false;
    T.nu0 = nu0;
    T.rank = rank;
    T.uniform = uni != 0;
    T.kind = kind;
    // shape checks before any vector is read
    const int64_t n = T.n;
    if (n < 1 || n > nmax || T.L < n || (T.L & (T.L - 1)) != 0 || T.L > 2 * nmax) return false;
    if (nu0 < 0 || nu0 > 32 || nu0 > n || T.N != n - nu0) return false;
    if (rank < 0 || rank > n || (uni != 0 && uni != 1) || (kind != JT_FIRST_KIND && kind != JT_SECOND_KIND)) return false;
    if (!valid_parameter(T.a) || !valid_parameter(T.b)) return false;
    const uint64_t un = (uint64_t)n, cap = un * un + 64;
    if (!get_vec(p, end, T.t, un) || !get_vec(p, end, T.w, un) || !get_vec(p, end, T.x, un) ||
        !get_vec(p, end, T.rowP, un) || !get_vec(p, end, T.rowQ, un) || !get_vec(p, end, T.S, un) ||
        !get_vec(p, end, T.m, un) || !get_vec(p, end, T.U, cap) || !get_vec(p, end, T.V, cap) ||
        !get_vec(p, end, T.Vblk, cap) || !get_vec(p, end, T.sigma, un) || !get_vec(p, end, T.beta, un + 2) ||
        !get_vec(p, end, T.sg, un + 3))
        return false;
    if ((int64_t)T.t.size() != n || (int64_t)T.w.size() != n || (int64_t)T.m.size() != n ||
        (int64_t)T.rowP.size() != n || (int64_t)T.rowQ.size() != n)
        return false;
    if ((int64_t)T.U.size() != (int64_t)rank * n || (int64_t)T.V.size() != (int64_t)rank * T.N ||
        (int64_t)T.Vblk.size() != n * nu0)
        return false;
    if (T.kind == JT_SECOND_KIND && (int64_t)T.S.size() != n) return false;
    for (int64_t j = 0; j < n; ++j) {
        if (T.m[j] < 0 || T.m[j] > T.L / 2) return false;
        if (!(T.t[j] > 0.0 && T.t[j] < 3.14159265358979323846)) return false;
    }
    return true;
}

}  // namespace jt
