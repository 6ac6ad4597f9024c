"""Dense reference for the discrete Jacobi polynomial transform -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline and
reference legs may import this module.  It shares no code with the CUDA library.

Notation follows arXiv:1901.07275:

* ``P_j^{(a,b)}`` Jacobi polynomials for the weight ``(1-x)^a (1+x)^b`` on
  (-1, 1) (Sec. 1, Eq. ``eq:jactrs``; the weight is read as ``(1-x)^a``,
  not the printed ``(1+x)^a`` of Eq. ``eq:GJquadrule``);
* ``p_j`` the orthonormal polynomials ``P_j / sqrt(h_j)``; the modified function
  ``P~_j(t) = C_j P_j(cos t) sin(t/2)^{a+1/2} cos(t/2)^{b+1/2}`` (Eqs.
  ``eq:modifiedjac`` and ``eq:C``) equals ``2^{(a+b+1)/2} p_j(cos t)
  sin(t/2)^{a+1/2} cos(t/2)^{b+1/2}`` because ``C_j^2 = 2^{a+b+1} / h_j``;
* ``(t_k, w_k)`` the trigonometric Gauss--Jacobi rule (Eq.
  ``introduction:modrule``, read with ``sin^{2a+1}(t/2) cos^{2b+1}(t/2)`` so that
  it matches ``P~``); ``omega_k`` the Christoffel numbers of the x-rule (Eq.
  ``eq:GJquadrule``); ``sqrt(w_k) P~_j(t_k) = sqrt(omega_k) p_j(x_k)``;
* degrees are 0-based: ``alpha[j]`` multiplies ``P~_j``, ``j = 0..n-1``
  (Sec. 3.1, Eq. ``tf:transexp``).
"""

from __future__ import annotations

import math

import numpy as np
import scipy.linalg

LD = np.longdouble


def _ld(v):
    return np.asarray(v, dtype=LD)


def mu0(a: float, b: float) -> LD:
    """Total mass ``int_{-1}^{1} (1-x)^a (1+x)^b dx = 2^{a+b+1} B(a+1, b+1)``."""
    lg = math.lgamma(a + 1.0) + math.lgamma(b + 1.0) - math.lgamma(a + b + 2.0)
    return LD(2.0) ** LD(a + b + 1.0) * np.exp(LD(lg))


def recurrence_coefficients(a: float, b: float, n: int):
    """Jacobi-matrix coefficients of the orthonormal recurrence.

    ``x p_j = sg[j+1] p_{j+1} + beta[j] p_j + sg[j] p_{j-1}`` with
    ``beta[0] = (b-a)/(a+b+2)``, ``beta[j] = (b^2-a^2)/((2j+a+b)(2j+a+b+2))`` and
    ``sg[j]^2 = 4 j (j+a)(j+b)(j+a+b) / ((2j+a+b)^2 (2j+a+b-1)(2j+a+b+1))``.
    At ``j = 1`` the factor ``(1+a+b)`` cancels analytically, which keeps the
    formula finite at ``a+b = -1``.  These are the textbook coefficients behind
    the three-term recurrence the paper uses for low degrees (Sec. 3.1, text
    after Eq. ``tf:jn``).  Returns ``beta[0..n]`` and ``sg[0..n+1]`` (``sg[0]=0``).
    """
    a = LD(a)
    b = LD(b)
    beta = np.zeros(n + 1, dtype=LD)
    sg = np.zeros(n + 2, dtype=LD)
    beta[0] = (b - a) / (a + b + 2)
    for j in range(1, n + 1):
        s = 2 * j + a + b
        beta[j] = (b * b - a * a) / (s * (s + 2))
    for j in range(1, n + 2):
        s = 2 * j + a + b
        if j == 1:
            sg[j] = np.sqrt(4 * (1 + a) * (1 + b) / ((2 + a + b) ** 2 * (3 + a + b)))
        else:
            sg[j] = (2 / s) * np.sqrt(j * (j + a) * (j + b) * (j + a + b) / ((s - 1) * (s + 1)))
    return beta, sg


def orthonormal_jacobi(x, a: float, b: float, n: int):
    """``p_j(x_i)`` for ``j = 0..n-1`` as an ``(len(x), n)`` longdouble array."""
    x = _ld(x).reshape(-1)
    beta, sg = recurrence_coefficients(a, b, max(n, 1))
    P = np.zeros((x.size, n), dtype=LD)
    if n == 0:
        return P
    P[:, 0] = 1 / np.sqrt(mu0(a, b))
    if n > 1:
        P[:, 1] = (x - beta[0]) * P[:, 0] / sg[1]
    for j in range(1, n - 1):
        P[:, j + 1] = ((x - beta[j]) * P[:, j] - sg[j] * P[:, j - 1]) / sg[j + 1]
    return P


def _pn_and_derivative(x, a: float, b: float, n: int):
    """``p_n(x)``, ``p_n'(x)`` and ``sum_{j<n} p_j(x)^2`` by the recurrence and its derivative."""
    beta, sg = recurrence_coefficients(a, b, n)
    p_prev = np.zeros_like(x)
    d_prev = np.zeros_like(x)
    p = np.full_like(x, 1 / np.sqrt(mu0(a, b)))
    d = np.zeros_like(x)
    ssq = np.zeros_like(x)
    for j in range(n):
        ssq += p * p
        p_next = ((x - beta[j]) * p - sg[j] * p_prev) / sg[j + 1]
        d_next = ((x - beta[j]) * d + p - sg[j] * d_prev) / sg[j + 1]
        p_prev, p = p, p_next
        d_prev, d = d, d_next
    return p, d, ssq


def _newton_nodes(t0, a: float, b: float, n: int, iters: int = 12):
    """Polish zeros of ``p_n(cos t)`` by Newton's method in the angle ``t``.

    The iteration stops once every correction is at the working precision's rounding level,
    or once the largest relative correction no longer shrinks (it has reached the rounding
    level of the recurrence that evaluates ``p_n``; further steps only move the nodes within
    that level)."""
    t = _ld(t0).copy()
    prev = None
    for _ in range(iters):
        x = np.cos(t)
        p, d, _ = _pn_and_derivative(x, a, b, n)
        # d/dt p_n(cos t) = -sin(t) p_n'(x)
        dt = p / (np.sin(t) * d)
        t = t + dt
        if np.all(np.abs(dt) <= 4 * np.finfo(LD).eps * np.abs(t)):
            break
        step = float(np.max(np.abs(dt) / np.abs(t))) if t.size else 0.0
        if prev is not None and step > 0.5 * prev:
            break
        prev = step
    x = np.cos(t)
    _, _, ssq = _pn_and_derivative(x, a, b, n)
    return t, x, 1 / ssq


def _golub_welsch_angles(a: float, b: float, n: int):
    """Initial angles from the eigenvalues of the Jacobi matrix (LAPACK), ascending in t."""
    beta, sg = recurrence_coefficients(a, b, n)
    if n == 1:
        xs = np.array([float(beta[0])])
    else:
        xs = scipy.linalg.eigh_tridiagonal(
            beta[:n].astype(np.float64), sg[1:n].astype(np.float64), eigvals_only=True
        )
    return np.sort(np.arccos(np.clip(xs, -1.0, 1.0)))


def _trig_weights(t, omega, a: float, b: float):
    """``w_k = 2^{-(a+b+1)} omega_k / (sin(t_k/2)^{2a+1} cos(t_k/2)^{2b+1})``."""
    s = np.sin(t / 2)
    c = np.cos(t / 2)
    return omega * LD(2.0) ** LD(-(a + b + 1)) / (s ** LD(2 * a + 1) * c ** LD(2 * b + 1))


def gauss_jacobi(a: float, b: float, n: int):
    """n-point Gauss--Jacobi rule in the angle variable (Sec. 1, Eqs. ``eq:GJquadrule``,
    ``introduction:modrule``).

    Nodes are the zeros of ``p_n(cos t)``, ascending in ``t`` (so ``x = cos t`` is
    descending); ``omega_k = 1 / sum_{j<n} p_j(x_k)^2`` are the Christoffel numbers;
    ``w_k`` the trigonometric weights.  Returns longdouble arrays ``(t, x, omega, w)``.
    """
    t0 = _golub_welsch_angles(a, b, n)
    t, x, omega = _newton_nodes(t0, a, b, n)
    order = np.argsort(t)
    t, x, omega = t[order], x[order], omega[order]
    return t, x, omega, _trig_weights(t, omega, a, b)


def gauss_jacobi_nodes_at(a: float, b: float, n: int, idx):
    """Nodes ``(t, x, omega)`` of the n-point rule at the given ascending-t indices only.

    For a few indices the initial angles are the selected eigenvalues of the Jacobi matrix
    alone (LAPACK bisection, one eigenvalue at a time: eigenvalue ``n-1-k`` in ascending x is
    node ``k`` in ascending t); otherwise all of them.  Newton then polishes each node."""
    idx = np.asarray(idx, dtype=np.int64)
    if n > 1 and np.unique(idx).size * 8 < n:
        beta, sg = recurrence_coefficients(a, b, n)
        dd, ee = beta[:n].astype(np.float64), sg[1:n].astype(np.float64)
        t0 = np.empty(idx.size)
        for i, k in enumerate(idx):
            e = n - 1 - int(k)
            xk = scipy.linalg.eigh_tridiagonal(dd, ee, eigvals_only=True, select="i", select_range=(e, e))[0]
            t0[i] = np.arccos(np.clip(xk, -1.0, 1.0))
    else:
        t0 = _golub_welsch_angles(a, b, n)[idx]
    return _newton_nodes(t0, a, b, n)


def modified_jacobi(t, a: float, b: float, n: int):
    """``P~_j(t_i)`` (Eq. ``eq:modifiedjac``) for ``j = 0..n-1``, longdouble ``(len(t), n)``."""
    t = _ld(t).reshape(-1)
    P = orthonormal_jacobi(np.cos(t), a, b, n)
    pref = (
        LD(2.0) ** LD((a + b + 1) / 2)
        * np.sin(t / 2) ** LD(a + 0.5)
        * np.cos(t / 2) ** LD(b + 0.5)
    )
    return P * pref[:, None]


def uniform_matrix(a: float, b: float, n: int) -> np.ndarray:
    """The orthogonal matrix ``W J`` of the uniform transform (Sec. 3.1, Eq. ``tf:transout``):
    entry ``(k, j) = sqrt(w_k) P~_j(t_k) = sqrt(omega_k) p_j(x_k)``; float64 ``(n, n)``."""
    t, x, omega, _ = gauss_jacobi(a, b, n)
    return (np.sqrt(omega)[:, None] * orthonormal_jacobi(x, a, b, n)).astype(np.float64)


def uniform_rows(a: float, b: float, n: int, rows) -> np.ndarray:
    """Selected rows of ``W J`` without forming the whole matrix."""
    t, x, omega = gauss_jacobi_nodes_at(a, b, n, rows)
    return (np.sqrt(omega)[:, None] * orthonormal_jacobi(x, a, b, n)).astype(np.float64)


def nonuniform_matrix(t, a: float, b: float, n: int) -> np.ndarray:
    """The unweighted matrix ``J`` at arbitrary angles ``t`` in (0, pi) (Sec. 3.1, last
    paragraph): entry ``(i, j) = P~_j(t_i)``; float64 ``(len(t), n)``."""
    return modified_jacobi(t, a, b, n).astype(np.float64)


def axis_matrix(n: int, a: float, b: float, points=None) -> np.ndarray:
    """``W J`` for Gauss--Jacobi nodes (``points is None``) or ``J`` at the given angles."""
    if points is None:
        return uniform_matrix(a, b, n)
    return nonuniform_matrix(points, a, b, n)


def _mode_apply(arr: np.ndarray, mats, transpose: bool) -> np.ndarray:
    d = len(mats)
    out = np.asarray(arr, dtype=np.float64)
    for ax, M in enumerate(mats):
        M = np.asarray(M, dtype=np.float64)
        if transpose:
            M = M.T
        axis = out.ndim - d + ax
        out = np.moveaxis(np.tensordot(out, M, axes=([axis], [1])), -1, axis)
    return out


def forward(alpha: np.ndarray, mats) -> np.ndarray:
    """d-dimensional forward transform by dense mode products (Eqs. ``eq:2Djac``,
    ``eq:3Djac``): ``f[..., i_0, .., i_{d-1}] = sum_k prod_a M_a[i_a, k_a] alpha[..., k]``.

    The last ``len(mats)`` axes of ``alpha`` are the transform axes (row-major, last
    axis fastest); leading axes are independent right-hand sides.
    """
    return _mode_apply(alpha, mats, transpose=False)


def adjoint(g: np.ndarray, mats) -> np.ndarray:
    """Transpose of :func:`forward` (the uniform inverse, Eqs. ``eq:oneJinv``,
    ``eq:invTJ``, ``eq:invTJ3``, when the matrices are the orthogonal ``W J``)."""
    return _mode_apply(g, mats, transpose=True)


def forward_sampled(alpha: np.ndarray, row_blocks, idx) -> np.ndarray:
    """Selected entries of a single-RHS d-dim forward transform.

    ``row_blocks[a]`` holds the rows ``M_a[idx[:, a], :]`` (one per sample);
    ``idx`` is ``(S, d)``.  Entries sharing the first index share the mode-0
    contraction, as a dense evaluation would.
    """
    idx = np.asarray(idx)
    d = idx.shape[1]
    alpha = np.asarray(alpha, dtype=np.float64)
    if d == 1:
        return row_blocks[0] @ alpha
    uniq, sel = np.unique(idx[:, 0], return_inverse=True)
    # one row of M_0 per distinct first index (any sample that uses it)
    rep = np.zeros(len(uniq), dtype=np.int64)
    for s, u in enumerate(sel):
        rep[u] = s
    R0u = row_blocks[0][rep]
    T = R0u @ alpha.reshape(alpha.shape[0], -1)
    out = np.empty(idx.shape[0])
    for s in range(idx.shape[0]):
        Ts = T[sel[s]].reshape(alpha.shape[1:])
        if d == 2:
            out[s] = Ts @ row_blocks[1][s]
        else:
            out[s] = row_blocks[1][s] @ Ts @ row_blocks[2][s]
    return out
