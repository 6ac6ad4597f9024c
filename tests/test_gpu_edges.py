"""Edge cases of the fused path against the oracle: the split degree nu0 at its limits, the
shortest FFT lengths on strided axes (16 and 32, where the staging is single-buffered or
the tile holds up to 256 fibres), 3-D transforms with a rank split on every axis, the
double-word kernel at L = 8192 with a rank split, ragged tiles, and a long FP32 axis at crowded
nonuniform points."""

import numpy as np
import pytest

import oracle
from paper_1901_07275_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "split": 1e-10}
EPS = {"fp32": 1e-7, "split": 1e-12}


@pytest.fixture(scope="module")
def torch_dev():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    return torch, torch.device("cuda:0")


def rel(x, ref):
    return np.linalg.norm(np.asarray(x, dtype=np.float64) - ref) / max(np.linalg.norm(ref), 1e-300)


def make(n, ab, prec, **kw):
    from paper_1901_07275_gb300 import Transform

    return Transform(n, [p[0] for p in ab], [p[1] for p in ab], eps=EPS[prec], precision=prec, **kw)


def dt(torch, prec):
    return torch.float32 if prec == "fp32" else torch.float64


@pytest.mark.parametrize("prec", ["fp32", "split"])
@pytest.mark.parametrize("nu0", [0, 1, 32])
def test_split_degree_limits(torch_dev, prec, nu0):
    """nu0 = 0 puts every degree in the low-rank part, 32 is the largest dense block; the
    transform does not depend on it (reading 3)."""
    torch, dev = torch_dev
    n = 300
    ab = [(0.2, -0.35)]
    T = make((n,), ab, prec, nu0=nu0)
    alpha = syn.normal(1100 + nu0, 0, (2, n))
    x = torch.tensor(alpha, dtype=dt(torch, prec), device=dev)
    M = [oracle.axis_matrix(n, *ab[0])]
    assert rel(T.forward(x).double().cpu().numpy(), oracle.forward(alpha, M)) < TOL[prec]
    assert rel(T.adjoint(x).double().cpu().numpy(), oracle.adjoint(alpha, M)) < TOL[prec]


@pytest.mark.parametrize("n", [(13, 700), (9, 257), (30, 150), (16, 40), (5, 3, 600)])
def test_short_strided_axes(torch_dev, n):
    torch, dev = torch_dev
    ab = [(0.1, 0.3), (-0.4, 0.2), (0.25, -0.15)][: len(n)]
    T = make(n, ab, "fp32")
    alpha = syn.normal(1200 + sum(n), 0, (3,) + n)
    x = torch.tensor(alpha, dtype=torch.float32, device=dev)
    M = [oracle.axis_matrix(m, a, b) for m, (a, b) in zip(n, ab)]
    assert rel(T.forward(x).double().cpu().numpy(), oracle.forward(alpha, M)) < TOL["fp32"]
    assert rel(T.adjoint(x).double().cpu().numpy(), oracle.adjoint(alpha, M)) < TOL["fp32"]


@pytest.mark.parametrize("kind", ["first", "second"])
def test_3d_with_rank_split(torch_dev, kind):
    torch, dev = torch_dev
    n = (40, 64, 70)
    ab = [(0.27, -0.45), (-0.16, 0.49), (-0.09, 0.13)]
    T = make(n, ab, "fp32", kind=kind)
    T.set_ksplit(4)
    alpha = syn.normal(1300, 0, n)
    x = torch.tensor(alpha, dtype=torch.float32, device=dev)
    mat = oracle.axis_matrix if kind == "first" else oracle.axis_matrix_q
    M = [mat(m, a, b) for m, (a, b) in zip(n, ab)]
    assert rel(T.forward(x).double().cpu().numpy(), oracle.forward(alpha, M)) < TOL["fp32"]
    assert rel(T.adjoint(x).double().cpu().numpy(), oracle.adjoint(alpha, M)) < TOL["fp32"]
    z = x.clone()
    T.forward(z, out=z)
    assert torch.equal(z, T.forward(x))


@pytest.mark.parametrize("ks", [1, 8])
def test_double_word_longest_axis_with_split(torch_dev, ks):
    """Split precision at n = 8000 (L = 8192, the 1024-thread double-word kernel), 40 sampled rows."""
    torch, dev = torch_dev
    n = 8000
    a, b = -0.3, 0.2
    T = make((n,), [(a, b)], "split")
    T.set_ksplit(ks)
    alpha = syn.normal(1400, 0, (1, n))
    f = T.forward(torch.tensor(alpha, dtype=torch.float64, device=dev)).cpu().numpy()
    rows = np.union1d(np.unique(syn.integers(1401, 3, 40, 0, n)), [0, n - 1])
    Q = oracle.uniform_rows(a, b, n, rows)
    assert rel(f[:, rows], alpha @ Q.T) < TOL["split"]


def test_many_right_hand_sides_ragged_tiles(torch_dev):
    """Fibre counts that leave a ragged last tile on every kernel shape of a 2-D transform."""
    torch, dev = torch_dev
    n = (100, 33)
    ab = [(0.05, 0.4), (-0.2, -0.1)]
    T = make(n, ab, "fp32")
    alpha = syn.normal(1500, 0, (7,) + n)
    x = torch.tensor(alpha, dtype=torch.float32, device=dev)
    M = [oracle.axis_matrix(m, a, b) for m, (a, b) in zip(n, ab)]
    assert rel(T.forward(x).double().cpu().numpy(), oracle.forward(alpha, M)) < TOL["fp32"]


@pytest.mark.parametrize("cluster", [6, 30])
def test_nonuniform_crowded_bins(torch_dev, cluster):
    """Nonuniform points that crowd FFT bins: up to 15 extra points a bin take the adjoint's
    per-lane lists, more take its bin_ptr / bin_idx walk; forward and adjoint against the
    oracle's dense J."""
    torch, dev = torch_dev
    n = 200
    rng_t = np.sort(np.pi * syn.uniform(1700 + cluster, 2, (n - cluster,)))
    # `cluster` points inside one bin of width 2 pi / 256
    tight = 1.0 + 0.01 * syn.uniform(1701 + cluster, 2, (cluster,))
    t = np.sort(np.concatenate([rng_t, tight]))
    ab = [(0.25, -0.1)]
    T = make((n,), ab, "fp32", points=[t])
    alpha = syn.normal(1702, 0, (3, n))
    x = torch.tensor(alpha, dtype=torch.float32, device=dev)
    M = [oracle.axis_matrix(n, *ab[0], t)]
    assert rel(T.forward(x).double().cpu().numpy(), oracle.forward(alpha, M)) < TOL["fp32"]
    assert rel(T.adjoint(x).double().cpu().numpy(), oracle.adjoint(alpha, M)) < TOL["fp32"]


@pytest.mark.parametrize("order,ks", [("sorted", 1), ("shuffled", 8)])
def test_long_fp32_axis_nonuniform_crowded(torch_dev, order, ks):
    """An FP32 axis of L = 8192 (the Stockham kernel's long instances) at nonuniform angles:
    about one bin in five holds more than two points and one holds 40, the points come sorted
    or shuffled (so that the bins' lists are walked through bin_idx), without a rank split and
    with one of 8 (the dense block then shared over the cluster).  The forward on sampled rows
    (all of the crowded bin among them) and the adjoint through them, against the oracle's J."""
    torch, dev = torch_dev
    n = 6000
    t = np.concatenate([np.pi * syn.uniform(1800, 2, (n - 40,)), 1.0 + 1e-4 * syn.uniform(1801, 2, (40,))])
    t = np.sort(t) if order == "sorted" else t[np.argsort(syn.uniform(1802, 2, (n,)))]
    ab = [(0.3, -0.2)]
    T = make((n,), ab, "fp32", points=[t])
    assert T.fft_lens == [8192]
    T.set_ksplit(ks)
    alpha = syn.normal(1803, 0, (4, n))
    f = T.forward(torch.tensor(alpha, dtype=torch.float32, device=dev)).double().cpu().numpy()
    crowd = np.nonzero((t >= 1.0) & (t <= 1.0 + 1e-4))[0]
    rows = np.union1d(np.unique(syn.integers(1804, 3, 96, 0, n)), np.concatenate([crowd, [0, n - 1]]))
    Q = oracle.nonuniform_matrix(t[rows], ab[0][0], ab[0][1], n)
    assert rel(f[:, rows], alpha @ Q.T) < TOL["fp32"]
    g = np.zeros((2, n))
    g[:, rows] = syn.normal(1805, 0, (2, rows.size))
    a = T.adjoint(torch.tensor(g, dtype=torch.float32, device=dev)).double().cpu().numpy()
    assert rel(a, g[:, rows] @ Q) < TOL["fp32"]
