"""Pins of the second-kind oracle (oracle/second_kind.py) against what the mathematics fixes,
independently of how the oracle computes it:

* the Stieltjes transform of the weight, S(x) = PV int (1-s)^a (1+s)^b / (x - s) ds, at the
  three classical closed forms (a = b = 0: log((1+x)/(1-x)); a = b = -1/2: 0; a = b = 1/2:
  pi x), up to t = 1e-4 from the end points;
* h_nu = PV int w p_nu / (x - s) from the recurrence, against a direct evaluation by
  singularity subtraction (the polynomial divided difference under the weight);
* Q~ at a = b = -1/2 (sqrt(2/pi) sin(nu t)) and a = b = 1/2 (-sqrt(2/pi) cos((nu+1) t)), and
  at a = b = 0 against scipy's Ferrers functions of the second kind;
* the Wronskian of P~ and Q~ (both solve the same equation in t without a first-derivative
  term) equals (2 nu + a + b + 1) / pi at general (a, b), including a + b = -1 and
  parameters near -1 and 1;
* the weighted uniform matrix at a = b = -1/2 against the discrete sine closed form.
"""

import numpy as np
import pytest
import scipy.integrate
import scipy.special

import oracle
from oracle import jacobi as oj

TS = np.array([1e-4, 3e-3, 0.05, 0.7, 1.5, 1.6, 2.9, np.pi - 3e-3, np.pi - 1e-4])


def _wmag(t, a, b):
    e1, e2 = 2 * np.sin(t / 2) ** 2, 2 * np.cos(t / 2) ** 2
    return np.maximum(1.0, e1 ** a * e2 ** b)


@pytest.mark.parametrize(
    "a,b,ref",
    [
        (0.0, 0.0, lambda t: np.log(np.cos(t / 2) ** 2 / np.sin(t / 2) ** 2)),
        (-0.5, -0.5, lambda t: np.zeros_like(t)),
        (0.5, 0.5, lambda t: np.pi * np.cos(t)),
    ],
)
def test_stieltjes_closed_forms(a, b, ref):
    S = oracle.stieltjes_t(TS, a, b)
    assert np.all(np.abs(S - ref(TS)) <= 1e-11 * _wmag(TS, a, b))


def test_stieltjes_reflection_and_x_form():
    # S_{a,b}(x) = -S_{b,a}(-x), and the x-argument form agrees with the t form
    a, b = 0.3, -0.7
    t = np.array([0.2, 1.0, 2.2])
    assert np.allclose(oracle.stieltjes_t(t, a, b), -oracle.stieltjes_t(np.pi - t, b, a), rtol=1e-12, atol=1e-12)
    assert np.allclose(oracle.stieltjes(np.cos(t), a, b), oracle.stieltjes_t(t, a, b), rtol=1e-10)


@pytest.mark.parametrize("a,b", [(0.37, -0.61), (-0.8, 0.9), (0.0, 0.5), (-0.5, -0.5)])
def test_second_kind_h_matches_divided_difference_quadrature(a, b):
    """h_nu(x) = int w(s) (p_nu(s) - p_nu(x)) / (x - s) ds + p_nu(x) S(x); the first integral has
    a polynomial integrand under the Jacobi weight (QUADPACK QAWS with both end exponents)."""
    n = 6
    t = np.array([0.4, 1.3, 2.6])
    H = oracle.second_kind_h(t, a, b, n).astype(np.float64)
    S = oracle.stieltjes_t(t, a, b)
    for i, ti in enumerate(t):
        xi = np.cos(ti)
        px = oj.orthonormal_jacobi([xi], a, b, n).astype(np.float64)[0]
        for nu in range(n):
            dd = lambda s: (oj.orthonormal_jacobi([s], a, b, nu + 1).astype(np.float64)[0, nu] - px[nu]) / (xi - s)
            val, _ = scipy.integrate.quad(dd, -1.0, 1.0, weight="alg", wvar=(b, a), epsabs=1e-14, epsrel=1e-13)
            ref = val + px[nu] * S[i]
            assert abs(H[i, nu] - ref) <= 1e-11 * max(1.0, abs(ref))


def test_q_tilde_chebyshev_closed_forms():
    t = np.linspace(5e-4, np.pi - 5e-4, 11)
    nu = np.arange(8)
    Qm = oracle.modified_second_kind(t, -0.5, -0.5, 8).astype(np.float64)
    assert np.abs(Qm - np.sqrt(2 / np.pi) * np.sin(np.outer(t, nu))).max() < 1e-12
    Qp = oracle.modified_second_kind(t, 0.5, 0.5, 8).astype(np.float64)
    assert np.abs(Qp + np.sqrt(2 / np.pi) * np.cos(np.outer(t, nu + 1))).max() < 1e-12


def test_q_tilde_legendre_matches_ferrers():
    """a = b = 0: Q~_nu(t) = -(2/pi) sqrt(nu + 1/2) sqrt(sin t) Q_nu(cos t) with Q_nu the Ferrers
    function of the second kind (Neumann's integral)."""
    t = np.array([0.05, 0.6, 1.4, 2.0, 3.0])
    n = 12
    Q = oracle.modified_second_kind(t, 0.0, 0.0, n).astype(np.float64)
    for i, ti in enumerate(t):
        fer, _ = scipy.special.lqn(n - 1, np.cos(ti))
        ref = -(2 / np.pi) * np.sqrt(np.arange(n) + 0.5) * np.sqrt(np.sin(ti)) * fer
        assert np.abs(Q[i] - ref).max() < 1e-11


@pytest.mark.parametrize("a,b", [(0.37, -0.61), (-0.25, 0.5), (0.9, 0.8), (-0.9, -0.85), (0.3, -0.3)])
def test_wronskian_of_first_and_second_kind(a, b):
    t = np.array([0.2, 1.3, 2.8])
    h = 1e-4
    for nu in (0, 1, 2, 7, 20):
        n = nu + 1

        def P(tv):
            return oj.modified_jacobi(tv, a, b, n)[:, nu]

        def Q(tv):
            return oracle.modified_second_kind(tv, a, b, n)[:, nu]

        def d(F):
            return (-F(t + 2 * h) + 8 * F(t + h) - 8 * F(t - h) + F(t - 2 * h)) / (12 * h)

        W = (P(t) * d(Q) - d(P) * Q(t)).astype(np.float64)
        assert np.allclose(W * np.pi / (2 * nu + a + b + 1), 1.0, rtol=0, atol=2e-8)


def test_uniform_second_kind_matrix_chebyshev():
    """a = b = -1/2: nodes t_k = (2k-1) pi / (2n), weights pi/n, so sqrt(w_k) Q~_j(t_k) =
    sqrt(2/n) sin(j t_k)."""
    n = 9
    Mq = oracle.uniform_matrix_q(-0.5, -0.5, n)
    tk = (2 * np.arange(1, n + 1) - 1) * np.pi / (2 * n)
    assert np.abs(Mq - np.sqrt(2 / n) * np.sin(np.outer(tk, np.arange(n)))).max() < 1e-13
    t = np.array([0.3, 2.0])
    assert np.allclose(oracle.axis_matrix_q(4, 0.2, 0.1, t), oracle.nonuniform_matrix_q(t, 0.2, 0.1, 4))
