"""Modified Jacobi functions of the second kind -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline and
reference legs may import this module.  It shares no code with the CUDA library.

The paper pairs ``P~_nu = M cos(psi)`` with ``Q~_nu = M sin(psi)`` (Sec. 1, Eqs.
``eq:jacnonosci`` and ``eq:jacnonosci2``) and says the transform for ``Q~`` is
similar to the one for ``P~`` (Sec. 3.1, 3.2, 3.3).  It defines ``Q~`` through the
Jacobi function of the second kind (Eq. ``eq:modifiedjac2``).  On the cut
(-1, 1) we take that function as the principal-value integral

    Q_nu(x) = 1/2 (1-x)^{-a} (1+x)^{-b} PV int_{-1}^{1} (1-s)^a (1+s)^b P_nu(s) / (x-s) ds

(Szego, Orthogonal Polynomials, Sec. 4.62; for a = b = 0 it is the Ferrers function
of Neumann's integral).  With the normalisation ``C_nu`` of Eq. ``eq:C`` the printed
Eq. ``eq:modifiedjac2`` then has modulus ``pi/2`` times that of ``P~``; the reading
taken here is the one of Eq. ``eq:jacnonosci2`` (``P~`` and ``Q~`` share the amplitude
``M``), i.e.

    Q~_nu(t) = -(2/pi) C_nu Q_nu(cos t) sin(t/2)^{a+1/2} cos(t/2)^{b+1/2}
             = -(1/pi) 2^{(a+b+1)/2} sin(t/2)^{a+1/2} cos(t/2)^{b+1/2} h_nu(cos t) / w(cos t),

with ``w(x) = (1-x)^a (1+x)^b``, ``p_nu`` the orthonormal polynomials and
``h_nu(x) = PV int w(s) p_nu(s) / (x-s) ds``.  At a = b = -1/2 this is
``sqrt(2/pi) sin(nu t)`` against ``P~ = sqrt(2/pi) cos(nu t)``.

``h_0 = p_0 S(x)`` with the Stieltjes transform ``S(x) = PV int w(s)/(x-s) ds``
computed by adaptive quadrature (QUADPACK through scipy: a Cauchy-weight rule on a
window around x, algebraic endpoint weights on the rest), and ``h_nu`` for nu >= 1
from the three-term recurrence of ``p_nu`` applied under the integral:
``(s - beta) / (x - s) = (x - beta) / (x - s) - 1`` gives
``sg_{nu+1} h_{nu+1} = (x - beta_nu) h_nu - sg_nu h_{nu-1} - int w p_nu``, where the
last integral is ``mu0^{1/2}`` for nu = 0 and zero after (orthogonality to p_0).

Pinned by ``tests/test_oracle_pins.py``: closed forms of ``S`` (a = b = 0, +-1/2),
``h_nu`` against direct principal-value quadrature, ``Q~`` against the Chebyshev
closed forms (a = b = +-1/2) and the Ferrers functions (a = b = 0), and the Wronskian
``P~ Q~' - P~' Q~ = (2 nu + a + b + 1) / pi`` at general (a, b).
"""

from __future__ import annotations

import warnings

import numpy as np
import scipy.integrate

from .jacobi import LD, gauss_jacobi, mu0, recurrence_coefficients


def _graded_pieces(c: float, d: float, end: float):
    """Break points from ``c +- d`` toward ``end`` at distances ``d, 2d, 4d, ..`` from c, stopping
    half way to ``end``, so that on every piece ``1/(u - c)`` varies by at most a factor 2."""
    sgn = 1.0 if end > c else -1.0
    pts = [c + sgn * d]
    half = 0.5 * abs(end - c)
    k = d
    while 2 * k < half:
        k *= 2
        pts.append(c + sgn * k)
    return pts


def _stieltjes_near_one(eps: float, a: float, b: float) -> float:
    """``S`` at ``x = 1 - eps`` (0 < eps <= 1) in the variable ``u = 1 - s``:
    ``S = PV int_0^2 u^a (2-u)^b / (u - eps) du``, so that ``1 - s`` and ``1 - x`` are exact
    near the end point.  A Cauchy-weight rule on ``[eps/2, 3 eps/2]``, pieces graded away
    from eps on either side (Gauss--Kronrod), and the pieces touching 0 and 2 with the
    algebraic end-point weights (QUADPACK QAWC / QAGS / QAWS)."""
    opts = dict(epsabs=0.0, epsrel=1e-13, limit=400)
    d = 0.5 * eps
    f = lambda u: u ** a * (2.0 - u) ** b
    tot = scipy.integrate.quad(f, eps - d, eps + d, weight="cauchy", wvar=eps, **opts)[0]
    g = lambda u: f(u) / (u - eps)
    lp = _graded_pieces(eps, d, 0.0)
    for hi_, lo_ in zip(lp[:-1], lp[1:]):
        tot += scipy.integrate.quad(g, lo_, hi_, **opts)[0]
    tot += scipy.integrate.quad(lambda u: (2.0 - u) ** b / (u - eps), 0.0, lp[-1], weight="alg", wvar=(a, 0.0),
                                **opts)[0]
    rp = _graded_pieces(eps, d, 2.0)
    for lo_, hi_ in zip(rp[:-1], rp[1:]):
        tot += scipy.integrate.quad(g, lo_, hi_, **opts)[0]
    tot += scipy.integrate.quad(lambda u: u ** a / (u - eps), rp[-1], 2.0, weight="alg", wvar=(0.0, b), **opts)[0]
    return tot


def stieltjes_t(t, a: float, b: float) -> np.ndarray:
    """``S(cos t) = PV int_{-1}^{1} (1-s)^a (1+s)^b / (cos t - s) ds`` for angles t in (0, pi).

    For ``t <= pi/2`` the integral is taken about the end point 1 with ``1 - x = 2 sin^2(t/2)``;
    for ``t > pi/2`` through the reflection ``S_{a,b}(x) = -S_{b,a}(-x)`` (substitute s -> -s)
    about the end point -1 with ``1 + x = 2 cos^2(t/2)``."""
    t = np.asarray(t, dtype=np.float64).reshape(-1)
    out = np.empty_like(t)
    with warnings.catch_warnings():
        # QUADPACK reports round-off when asked for 1e-13; the attained accuracy is what
        # the closed-form pins in tests/test_oracle_pins.py check
        warnings.simplefilter("ignore", scipy.integrate.IntegrationWarning)
        for i, ti in enumerate(t):
            if ti <= 0.5 * np.pi:
                out[i] = _stieltjes_near_one(2.0 * np.sin(0.5 * ti) ** 2, a, b)
            else:
                out[i] = -_stieltjes_near_one(2.0 * np.cos(0.5 * ti) ** 2, b, a)
    return out


def stieltjes(x, a: float, b: float) -> np.ndarray:
    """``S(x)`` for x in (-1, 1) (through ``t = arccos x``)."""
    return stieltjes_t(np.arccos(np.asarray(x, dtype=np.float64)), a, b)


def second_kind_h(t, a: float, b: float, n: int) -> np.ndarray:
    """``h_nu(cos t_i) = PV int w(s) p_nu(s) / (cos t_i - s) ds`` for ``nu = 0..n-1``, longdouble
    ``(len(t), n)``."""
    t = np.asarray(t, dtype=np.float64).reshape(-1)
    beta, sg = recurrence_coefficients(a, b, max(n, 1))
    H = np.zeros((t.size, n), dtype=LD)
    if n == 0:
        return H
    xl = np.cos(t.astype(LD))
    p0 = 1 / np.sqrt(mu0(a, b))
    H[:, 0] = p0 * stieltjes_t(t, a, b).astype(LD)
    if n > 1:
        H[:, 1] = ((xl - beta[0]) * H[:, 0] - np.sqrt(mu0(a, b))) / sg[1]
    for j in range(1, n - 1):
        H[:, j + 1] = ((xl - beta[j]) * H[:, j] - sg[j] * H[:, j - 1]) / sg[j + 1]
    return H


def modified_second_kind(t, a: float, b: float, n: int) -> np.ndarray:
    """``Q~_j(t_i)`` (Eq. ``eq:jacnonosci2``, read as above) for ``j = 0..n-1``, longdouble."""
    t = np.asarray(t, dtype=LD).reshape(-1)
    s2 = np.sin(t / 2)
    c2 = np.cos(t / 2)
    H = second_kind_h(t.astype(np.float64), a, b, n)
    w = (2 * s2 * s2) ** LD(a) * (2 * c2 * c2) ** LD(b)
    pref = -(LD(1) / LD(np.pi)) * LD(2.0) ** LD((a + b + 1) / 2) * s2 ** LD(a + 0.5) * c2 ** LD(b + 0.5) / w
    return H * pref[:, None]


def uniform_matrix_q(a: float, b: float, n: int) -> np.ndarray:
    """``sqrt(w_k) Q~_j(t_k)`` at the Gauss--Jacobi nodes (the weighted second-kind matrix), float64."""
    t, x, omega, w = gauss_jacobi(a, b, n)
    return (np.sqrt(w)[:, None] * modified_second_kind(t, a, b, n)).astype(np.float64)


def nonuniform_matrix_q(t, a: float, b: float, n: int) -> np.ndarray:
    """``Q~_j(t_i)`` at arbitrary angles in (0, pi), float64 ``(len(t), n)``."""
    return modified_second_kind(t, a, b, n).astype(np.float64)


def axis_matrix_q(n: int, a: float, b: float, points=None) -> np.ndarray:
    """Second-kind counterpart of :func:`oracle.axis_matrix`."""
    if points is None:
        return uniform_matrix_q(a, b, n)
    return nonuniform_matrix_q(points, a, b, n)
