"""Pins of the CPU oracle against facts it does not compute itself.

Each test ties one part of ``oracle/`` to a closed form, a library routine, brute
force in arbitrary precision or an identity the mathematics fixes, chosen so that
a dropped term, a wrong sign or index, a swapped (a, b) or a transposed operand
fails at least one of them.
"""

import math

import numpy as np
import pytest

import oracle
from oracle import jacobi as oj

mpmath = pytest.importorskip("mpmath")


# ---------------------------------------------------------------- closed forms
@pytest.mark.parametrize("n", [1, 2, 7, 64, 129])
def test_chebyshev_first_kind_is_orthonormal_dct3(n):
    """a = b = -1/2: nodes t_k = (2k-1)pi/(2n); W J is the orthonormal DCT-III,
    entries sqrt(2/n) cos(j t_k) and sqrt(1/n) in column 0."""
    Q = oracle.uniform_matrix(-0.5, -0.5, n)
    t = (2 * np.arange(1, n + 1) - 1) * np.pi / (2 * n)
    ref = np.sqrt(2.0 / n) * np.cos(np.outer(t, np.arange(n)))
    ref[:, 0] = np.sqrt(1.0 / n)
    assert np.abs(Q - ref).max() < 1e-14
    tt, _, _, _ = oracle.gauss_jacobi(-0.5, -0.5, n)
    assert np.abs(tt.astype(float) - t).max() < 1e-14


@pytest.mark.parametrize("n", [1, 3, 8, 100])
def test_chebyshev_second_kind_is_orthonormal_dst1(n):
    """a = b = 1/2: nodes t_k = k pi/(n+1); W J is the orthonormal DST-I,
    entries sqrt(2/(n+1)) sin((j+1) t_k)."""
    Q = oracle.uniform_matrix(0.5, 0.5, n)
    t = np.arange(1, n + 1) * np.pi / (n + 1)
    ref = np.sqrt(2.0 / (n + 1)) * np.sin(np.outer(t, np.arange(1, n + 1)))
    assert np.abs(Q - ref).max() < 1e-14


@pytest.mark.parametrize("n", [1, 5, 33])
def test_chebyshev_third_kind(n):
    """a = -1/2, b = 1/2 (weight sqrt((1+x)/(1-x))): p_j is proportional to
    V_j(cos t) = cos((j+1/2) t) / cos(t/2), so P~_j = sqrt(2/pi) cos((j+1/2) t);
    nodes t_k = (2k-1) pi / (2n+1) and W J = 2/sqrt(2n+1) cos((j+1/2) t_k)."""
    Q = oracle.uniform_matrix(-0.5, 0.5, n)
    t = (2 * np.arange(1, n + 1) - 1) * np.pi / (2 * n + 1)
    ref = 2 / np.sqrt(2 * n + 1) * np.cos(np.outer(t, np.arange(n) + 0.5))
    assert np.abs(Q - ref).max() < 1e-14
    tg = np.linspace(0.05, 3.0, 17)
    P = oracle.modified_jacobi(tg, -0.5, 0.5, 6).astype(float)
    assert np.abs(P - np.sqrt(2 / np.pi) * np.cos(np.outer(tg, np.arange(6) + 0.5))).max() < 1e-14


@pytest.mark.parametrize("n", [2, 9, 40])
def test_chebyshev_fourth_kind(n):
    """a = 1/2, b = -1/2: P~_j = sqrt(2/pi) sin((j+1/2) t); nodes t_k = 2k pi/(2n+1)."""
    Q = oracle.uniform_matrix(0.5, -0.5, n)
    t = 2 * np.arange(1, n + 1) * np.pi / (2 * n + 1)
    ref = 2 / np.sqrt(2 * n + 1) * np.sin(np.outer(t, np.arange(n) + 0.5))
    assert np.abs(Q - ref).max() < 1e-14


def test_legendre_textbook_values():
    """a = b = 0: p_j = sqrt((2j+1)/2) P_j with P_2 = (3x^2-1)/2, P_3 = (5x^3-3x)/2."""
    x = np.array([-0.7, 0.1, 0.95])
    P = oracle.orthonormal_jacobi(x, 0.0, 0.0, 4).astype(float)
    assert np.allclose(P[:, 0], np.sqrt(0.5), rtol=0, atol=1e-16)
    assert np.allclose(P[:, 1], np.sqrt(1.5) * x, rtol=0, atol=1e-15)
    assert np.allclose(P[:, 2], np.sqrt(2.5) * (3 * x**2 - 1) / 2, rtol=0, atol=1e-15)
    assert np.allclose(P[:, 3], np.sqrt(3.5) * (5 * x**3 - 3 * x) / 2, rtol=0, atol=1e-15)


def _read_golden(name):
    import os

    path = os.path.join(os.path.dirname(__file__), "golden", name)
    rows = []
    with open(path) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append([float(v) for v in line.split()])
    return np.array(rows)


def test_gauss_legendre_three_point_table():
    """Three-point Gauss--Legendre rule from the textbook table (golden fixture)."""
    g = _read_golden("gauss_legendre_3pt.txt")
    t, x, omega, _ = oracle.gauss_jacobi(0.0, 0.0, 3)
    assert np.abs(x.astype(float) - g[:, 0]).max() < 1e-15
    assert np.abs(omega.astype(float) - g[:, 1]).max() < 1e-15


# ----------------------------------------------------------- library routines
@pytest.mark.parametrize("a,b", [(-0.25, 0.5), (0.3, -0.4), (-0.5, 0.2), (0.9, -0.9), (-0.95, -0.6)])
@pytest.mark.parametrize("n", [4, 31, 200])
def test_nodes_match_scipy_roots_jacobi(a, b, n):
    from scipy.special import roots_jacobi

    xs, ws = roots_jacobi(n, a, b)
    _, x, omega, _ = oracle.gauss_jacobi(a, b, n)
    order = np.argsort(-xs)
    assert np.abs(x.astype(float) - xs[order]).max() < 5e-15
    # scipy's weights lose relative accuracy near the endpoints; the strict weight
    # pin is the moment test below.
    assert np.abs(omega.astype(float) / ws[order] - 1).max() < 1e-6


@pytest.mark.parametrize("a,b", [(-0.25, 0.5), (0.9, -0.9), (-0.95, -0.6)])
def test_selected_nodes_match_scipy_roots_jacobi(a, b):
    """A few nodes of a long rule (initial angles from single selected eigenvalues, then
    Newton) against scipy's nodes, including both ends of the rule."""
    from scipy.special import roots_jacobi

    n = 400
    idx = np.array([0, 1, 57, 200, 398, 399])
    xs, _ = roots_jacobi(n, a, b)
    ref = np.sort(xs)[::-1][idx]  # ascending t is descending x
    t, x, omega = oracle.gauss_jacobi_nodes_at(a, b, n, idx)
    assert np.abs(x.astype(float) - ref).max() < 5e-15
    _, xf, omf, _ = oracle.gauss_jacobi(a, b, n)
    assert np.abs(omega.astype(float) / omf[idx].astype(float) - 1).max() < 1e-13


@pytest.mark.parametrize("a,b", [(-0.25, 0.5), (0.7, 0.1)])
def test_nodes_match_golub_welsch_eigen(a, b):
    """Nodes are the eigenvalues of the Jacobi matrix (LAPACK dense eigensolver)."""
    n = 50
    beta, sg = oracle.recurrence_coefficients(a, b, n)
    T = np.diag(beta[:n].astype(float)) + np.diag(sg[1:n].astype(float), 1) + np.diag(sg[1:n].astype(float), -1)
    ev, vec = np.linalg.eigh(T)
    _, x, omega, _ = oracle.gauss_jacobi(a, b, n)
    assert np.abs(np.sort(x.astype(float)) - ev).max() < 1e-14
    # Golub--Welsch weights: mu0 * (first eigenvector component)^2
    mu0 = float(oj.mu0(a, b))
    gw = mu0 * vec[0, :] ** 2
    assert np.abs(np.sort(omega.astype(float))[::-1][:10] - np.sort(gw)[::-1][:10]).max() < 1e-13


# ------------------------------------------------------------- brute force
def _jacobi_explicit(nn, a, b, x):
    """DLMF 18.5.7: P_n(x) = sum_s C(n+a, n-s) C(n+b, s) ((x-1)/2)^s ((x+1)/2)^(n-s)."""
    tot = mpmath.mpf(0)
    for s in range(nn + 1):
        tot += (
            mpmath.binomial(nn + a, nn - s)
            * mpmath.binomial(nn + b, s)
            * ((x - 1) / 2) ** s
            * ((x + 1) / 2) ** (nn - s)
        )
    return tot


def _h(nn, a, b):
    """Squared norm of P_n^{(a,b)} (DLMF 18.3), with the n = 0 limit written out."""
    if nn == 0:
        return 2 ** (a + b + 1) * mpmath.gamma(a + 1) * mpmath.gamma(b + 1) / mpmath.gamma(a + b + 2)
    return (
        2 ** (a + b + 1)
        * mpmath.gamma(nn + a + 1)
        * mpmath.gamma(nn + b + 1)
        / ((2 * nn + a + b + 1) * mpmath.gamma(nn + a + b + 1) * mpmath.factorial(nn))
    )


@pytest.mark.parametrize("a,b", [(-0.25, 0.5), (0.3, -0.4), (-0.5, -0.5), (0.9, 0.8)])
def test_orthonormal_polys_match_explicit_sum(a, b):
    mpmath.mp.dps = 40
    a_m, b_m = mpmath.mpf(a), mpmath.mpf(b)
    xs = [-0.93, -0.2, 0.41, 0.999]
    n = 18
    P = oracle.orthonormal_jacobi(np.array(xs), a, b, n)
    for i, xv in enumerate(xs):
        for j in range(n):
            ref = _jacobi_explicit(j, a_m, b_m, mpmath.mpf(xv)) / mpmath.sqrt(_h(j, a_m, b_m))
            assert abs(float(P[i, j]) - float(ref)) <= 1e-14 * max(1.0, abs(float(ref)))


@pytest.mark.parametrize("a,b", [(-0.25, 0.5), (0.3, -0.4), (0.6, 0.6)])
def test_modified_function_uses_paper_normalisation(a, b):
    """P~_nu(t) = C_nu P_nu(cos t) sin(t/2)^{a+1/2} cos(t/2)^{b+1/2} with C_nu of Eq. (C)."""
    mpmath.mp.dps = 40
    a_m, b_m = mpmath.mpf(a), mpmath.mpf(b)
    ts = [0.01, 0.7, 1.9, 3.13]
    n = 12
    Pt = oracle.modified_jacobi(np.array(ts), a, b, n)
    for i, tv in enumerate(ts):
        t_m = mpmath.mpf(tv)
        for nu in range(n):
            C = mpmath.sqrt(
                (2 * nu + a_m + b_m + 1)
                * mpmath.gamma(1 + nu)
                * mpmath.gamma(1 + nu + a_m + b_m)
                / (mpmath.gamma(1 + nu + a_m) * mpmath.gamma(1 + nu + b_m))
            )
            ref = (
                C
                * _jacobi_explicit(nu, a_m, b_m, mpmath.cos(t_m))
                * mpmath.sin(t_m / 2) ** (a_m + mpmath.mpf(0.5))
                * mpmath.cos(t_m / 2) ** (b_m + mpmath.mpf(0.5))
            )
            assert abs(float(Pt[i, nu]) - float(ref)) <= 1e-14 * max(1.0, abs(float(ref)))


def _moment(m, a, b):
    """int_{-1}^{1} x^m (1-x)^a (1+x)^b dx via x = 2u-1 and Beta integrals."""
    tot = mpmath.mpf(0)
    for i in range(m + 1):
        tot += mpmath.binomial(m, i) * mpmath.mpf(2) ** i * (-1) ** (m - i) * mpmath.beta(b + i + 1, a + 1)
    return mpmath.mpf(2) ** (a + b + 1) * tot


@pytest.mark.parametrize("a,b", [(-0.25, 0.5), (0.9, -0.9), (-0.5, 0.2)])
@pytest.mark.parametrize("n", [1, 4, 11])
def test_rule_is_exact_to_degree_2n_minus_1(a, b, n):
    mpmath.mp.dps = 60
    _, x, omega, _ = oracle.gauss_jacobi(a, b, n)
    xm = [mpmath.mpf(str(v)) for v in x]
    wm = [mpmath.mpf(str(v)) for v in omega]
    for m in range(2 * n):
        quad = sum(w * xv**m for w, xv in zip(wm, xm))
        exact = _moment(m, mpmath.mpf(a), mpmath.mpf(b))
        assert abs(quad - exact) <= 1e-15 * max(1, abs(exact)) * 4


# --------------------------------------------------------------- invariants
@pytest.mark.parametrize("a,b", [(-0.25, 0.5), (0.3, -0.4), (0.8, 0.05), (-0.9, 0.9)])
def test_orthogonality_of_weighted_matrix(a, b):
    """W J is orthogonal in the uniform case (Sec. 3.1): Q^T Q = Q Q^T = I."""
    for n in (3, 27, 28, 150):
        Q = oracle.uniform_matrix(a, b, n)
        assert np.abs(Q.T @ Q - np.eye(n)).max() < 2e-14 * max(1, n / 50)
        assert np.abs(Q @ Q.T - np.eye(n)).max() < 2e-14 * max(1, n / 50)


@pytest.mark.parametrize("a,b", [(-0.25, 0.5), (0.3, -0.4)])
def test_modified_functions_solve_the_jacobi_ode(a, b):
    """P~_nu solves y'' + q_nu y = 0 with q_nu of Eq. ``jacobieq:coef``; a wrong
    prefactor exponent or normalisation breaks this."""
    h = 1e-3
    ts = np.array([0.3, 0.9, 1.6, 2.4, 2.9])
    nu = np.arange(10)
    Pm = oracle.modified_jacobi(ts - h, a, b, 10).astype(float)
    P0 = oracle.modified_jacobi(ts, a, b, 10).astype(float)
    Pp = oracle.modified_jacobi(ts + h, a, b, 10).astype(float)
    d2 = (Pp - 2 * P0 + Pm) / h**2
    q = (
        (nu[None, :] + (a + b + 1) / 2) ** 2
        + (0.25 - a * a) / (4 * np.sin(ts[:, None] / 2) ** 2)
        + (0.25 - b * b) / (4 * np.cos(ts[:, None] / 2) ** 2)
    )
    assert np.abs(d2 + q * P0).max() < 2e-4 * np.abs(q * P0).max()


@pytest.mark.parametrize("n", [5, 64])
def test_reflection_swaps_parameters(n):
    """P_n^{(a,b)}(-x) = (-1)^n P_n^{(b,a)}(x): the (a,b) nodes are pi minus the (b,a) nodes."""
    t1, _, om1, _ = oracle.gauss_jacobi(-0.25, 0.5, n)
    t2, _, om2, _ = oracle.gauss_jacobi(0.5, -0.25, n)
    assert np.abs(t1.astype(float) - (np.pi - t2.astype(float))[::-1]).max() < 1e-14
    assert np.abs(om1.astype(float) - om2.astype(float)[::-1]).max() < 1e-14


def test_christoffel_weights_sum_to_mass():
    for a, b in [(-0.25, 0.5), (0.99, -0.99)]:
        _, _, om, _ = oracle.gauss_jacobi(a, b, 300)
        assert abs(float(om.sum() / oj.mu0(a, b)) - 1) < 1e-14


def test_trig_weights_integrate_in_t():
    """The t-rule integrates sin^{2a+1}(t/2) cos^{2b+1}(t/2) exactly (Eq. introduction:modrule
    with f = 1): sum_k w_k s_k^{2a+1} c_k^{2b+1} = int_0^pi s^{2a+1} c^{2b+1} dt = B(a+1, b+1)."""
    a, b = -0.25, 0.5
    t, _, _, w = oracle.gauss_jacobi(a, b, 40)
    s, c = np.sin(t / 2), np.cos(t / 2)
    lhs = float((w * s ** np.longdouble(2 * a + 1) * c ** np.longdouble(2 * b + 1)).sum())
    rhs = math.gamma(a + 1) * math.gamma(b + 1) / math.gamma(a + b + 2)
    assert abs(lhs / rhs - 1) < 1e-14


def test_sampled_rows_match_full_matrix():
    a, b, n = 0.3, -0.4, 97
    Q = oracle.uniform_matrix(a, b, n)
    rows = np.array([0, 1, 48, 95, 96])
    assert np.abs(oracle.uniform_rows(a, b, n, rows) - Q[rows]).max() < 1e-15


# --------------------------------------------------------------- d-dim apply
def test_forward_2d_brute_force_nonsquare():
    rng = np.random.default_rng(0)
    M0 = rng.standard_normal((4, 3))
    M1 = rng.standard_normal((5, 2))
    al = rng.standard_normal((3, 2))
    f = oracle.forward(al, [M0, M1])
    for i in range(4):
        for j in range(5):
            ref = sum(M0[i, k] * M1[j, l] * al[k, l] for k in range(3) for l in range(2))
            assert abs(f[i, j] - ref) < 1e-13
    g = rng.standard_normal((4, 5))
    ad = oracle.adjoint(g, [M0, M1])
    for k in range(3):
        for l in range(2):
            ref = sum(M0[i, k] * M1[j, l] * g[i, j] for i in range(4) for j in range(5))
            assert abs(ad[k, l] - ref) < 1e-13


def test_forward_3d_brute_force_with_rhs():
    rng = np.random.default_rng(1)
    Ms = [rng.standard_normal((3, 2)), rng.standard_normal((2, 4)), rng.standard_normal((4, 3))]
    al = rng.standard_normal((2, 2, 4, 3))  # two right-hand sides
    f = oracle.forward(al, Ms)
    assert f.shape == (2, 3, 2, 4)
    for r in range(2):
        for i in range(3):
            for j in range(2):
                for k in range(4):
                    ref = sum(
                        Ms[0][i, h] * Ms[1][j, l] * Ms[2][k, m] * al[r, h, l, m]
                        for h in range(2)
                        for l in range(4)
                        for m in range(3)
                    )
                    assert abs(f[r, i, j, k] - ref) < 1e-12


def test_forward_sampled_matches_full():
    rng = np.random.default_rng(2)
    Ms = [rng.standard_normal((6, 6)), rng.standard_normal((5, 5)), rng.standard_normal((7, 7))]
    al = rng.standard_normal((6, 5, 7))
    full = oracle.forward(al, Ms)
    idx = np.stack([rng.integers(0, 6, 40), rng.integers(0, 5, 40), rng.integers(0, 7, 40)], axis=1)
    rows = [Ms[a][idx[:, a]] for a in range(3)]
    samp = oracle.forward_sampled(al, rows, idx)
    assert np.abs(samp - full[idx[:, 0], idx[:, 1], idx[:, 2]]).max() < 1e-12
    al2 = al[:, :, 0]
    full2 = oracle.forward(al2, Ms[:2])
    samp2 = oracle.forward_sampled(al2, rows[:2], idx[:, :2])
    assert np.abs(samp2 - full2[idx[:, 0], idx[:, 1]]).max() < 1e-12
