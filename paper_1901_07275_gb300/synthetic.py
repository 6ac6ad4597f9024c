"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This module holds no arithmetic of the Jacobi transform itself: only a
counter-based random generator and the shapes of the workloads.  Both the CUDA
path and the CPU oracle receive the arrays it produces, so that they see
bit-identical inputs.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014) used in counter mode -- value ``i`` of stream
``s`` under ``seed`` is ``mix(key(seed, s) + (i + 1) * GAMMA)`` -- and the
Box--Muller transform for normal variates.
"""

from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        s = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) ^ (np.uint64(stream & 0xFFFFFFFF) * _M2)
    return _mix(np.array([s], dtype=np.uint64))[0]


def bits(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """``count`` raw 64-bit values of stream ``stream``, starting at counter ``offset``."""
    i = np.arange(offset, offset + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(_key(seed, stream) + (i + np.uint64(1)) * GAMMA)


def uniform(seed: int, stream: int, shape, offset: int = 0) -> np.ndarray:
    """Uniform float64 in the open interval (0, 1)."""
    n = int(np.prod(shape)) if shape else 1
    u = (bits(seed, stream, n, offset) >> np.uint64(11)).astype(np.float64)
    return ((u + 0.5) * 2.0**-53).reshape(shape)


def normal(seed: int, stream: int, shape) -> np.ndarray:
    """Standard normal float64 by Box--Muller on consecutive uniform pairs."""
    n = int(np.prod(shape)) if shape else 1
    u = uniform(seed, stream, (2 * ((n + 1) // 2),))
    u1, u2 = u[0::2], u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * u1.size)
    z[0::2] = r * np.cos(2 * np.pi * u2)
    z[1::2] = r * np.sin(2 * np.pi * u2)
    return z[:n].reshape(shape)


def integers(seed: int, stream: int, count: int, low: int, high: int) -> np.ndarray:
    """``count`` integers uniform in ``[low, high)`` (with replacement)."""
    u = uniform(seed, stream, (count,))
    return (low + np.floor(u * (high - low))).astype(np.int64).clip(low, high - 1)


# ------------------------------------------------------------------ workloads
# Seed of workload c is 1000 + c; streams: 0 coefficients, 1 right-hand data y,
# 2 points, 3 sample indices, 4 parameters (a, b), 5 sizes, 6 directions.

def workload(name: str, nrhs: int = 1) -> dict:
    """Shapes, parameters and seeded arrays of the named workload.

    * ``1d-1024``: 1-D uniform, n = 1024, (a, b) = (-0.25, 0.5), alpha ~ N(0, 1).
    * ``2d-512``: 2-D uniform 512 x 512, (a, b) = (0.3, -0.4) on axis 0 and
      (-0.5, 0.2) on axis 1, alpha ~ N(0, 1).
    * ``3d-256``: 3-D uniform 256^3, a_i, b_i ~ U(-0.5, 0.5) per axis, alpha ~
      N(0, 1) / (1 + |nu|) with |nu| the Euclidean norm of the 0-based degree index.
    * ``2d-nonuniform-1024``: t_x, t_y each 1024 i.i.d. U(0, pi), sorted;
      a = b = 0.25; alpha and y ~ N(0, 1).
    """
    if name == "1d-1024":
        seed, ns, ab = 1001, (1024,), [(-0.25, 0.5)]
    elif name == "2d-512":
        seed, ns, ab = 1002, (512, 512), [(0.3, -0.4), (-0.5, 0.2)]
    elif name == "3d-256":
        seed, ns = 1003, (256, 256, 256)
        u = uniform(seed, 4, (6,)) - 0.5
        ab = [(float(u[2 * i]), float(u[2 * i + 1])) for i in range(3)]
    elif name == "2d-nonuniform-1024":
        seed, ns, ab = 1005, (1024, 1024), [(0.25, 0.25), (0.25, 0.25)]
    else:
        raise KeyError(name)
    shape = (nrhs,) + ns
    alpha = normal(seed, 0, shape)
    if name == "3d-256":
        grids = np.meshgrid(*[np.arange(n, dtype=np.float64) for n in ns], indexing="ij")
        alpha = alpha / (1.0 + np.sqrt(sum(g * g for g in grids)))[None]
    points = [None] * len(ns)
    if name == "2d-nonuniform-1024":
        points = [np.sort(np.pi * uniform(seed, 2, (n,), offset=k * 100000)) for k, n in enumerate(ns)]
    return {
        "name": name,
        "seed": seed,
        "n": list(ns),
        "ab": ab,
        "points": points,
        "alpha": alpha,
        "y": normal(seed, 1, shape) if name == "2d-nonuniform-1024" else None,
    }


def batch_mix(count: int = 512, seed: int = 1004, n1=(256, 16384), n2=(64, 1024), max_rhs: int = 16):
    """The serving-style mix: ``count`` members, a fair coin between 1-D and 2-D; 1-D n
    log-uniform in ``n1``, 2-D n_x, n_y drawn independently log-uniform in ``n2``; (a, b)
    uniform in (-0.5, 0.5) per axis; nrhs uniform in 1..max_rhs.  Returns a list of dicts
    with ``n``, ``ab`` and ``nrhs`` (coefficients are drawn by the caller per member)."""
    u = uniform(seed, 5, (count, 8))
    members = []
    for i in range(count):
        two = u[i, 0] < 0.5
        lo, hi = (n2 if two else n1)
        ns = [int(round(np.exp(np.log(lo) + u[i, 1 + k] * (np.log(hi) - np.log(lo))))) for k in range(2 if two else 1)]
        ab = [(float(u[i, 3 + 2 * k] - 0.5), float(u[i, 4 + 2 * k] - 0.5)) for k in range(len(ns))]
        members.append({"n": ns, "ab": ab, "nrhs": 1 + int(u[i, 7] * max_rhs)})
    return members
