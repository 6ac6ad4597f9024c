"""Plan setup with the O(n^2) steps on the GPU (jt_options.setup_device = 1): nodes, weights
and transforms agree with the host setup and with the oracle."""

import numpy as np
import pytest

import oracle
from paper_1901_07275_gb300 import binding as B
from paper_1901_07275_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_dev():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    return torch, torch.device("cuda:0")


@pytest.mark.parametrize("a,b,n", [(-0.25, 0.5, 1024), (0.3, -0.4, 300), (0.9, -0.9, 2000), (-0.5, -0.5, 64),
                                   (0.1, 0.2, 5)])
def test_gpu_setup_tables_match_host_and_oracle(torch_dev, a, b, n):
    Th = B.AxisTables(n, a, b, eps=1e-12, opt=B.options("split"))
    Tg = B.AxisTables(n, a, b, eps=1e-12, opt=B.options("split", setup_device=1))
    assert np.abs(Tg.t - Th.t).max() <= 8 * np.finfo(float).eps * np.pi
    assert np.abs(Tg.w / Th.w - 1).max() < 1e-13
    t, _, _, w = oracle.gauss_jacobi(a, b, n)
    assert np.abs(Tg.t - t.astype(float)).max() < 8 * np.finfo(float).eps * np.pi
    assert abs(Tg.rank - Th.rank) <= 1
    # the rebuilt weighted matrix against the oracle
    G = Tg.U.T @ Tg.V
    F = np.exp(2j * np.pi * np.outer(Tg.m, np.arange(Tg.nu0, n)) / Tg.L)
    D = np.concatenate([Tg.vblk, np.real(G * F)], axis=1)
    Q = oracle.uniform_matrix(a, b, n)
    assert np.linalg.norm(D - Q) <= 1e-10 * np.linalg.norm(Q)


def test_gpu_setup_second_kind_nonuniform(torch_dev):
    n = 400
    t = np.sort(np.pi * syn.uniform(930, 2, (n,)))
    opt = B.options("split", kind="second", setup_device=1)
    T = B.AxisTables(n, 0.25, -0.1, points=t, eps=1e-12, opt=opt)
    G = T.U.T @ T.V
    F = np.exp(2j * np.pi * np.outer(T.m, np.arange(T.nu0, n)) / T.L)
    D = np.concatenate([T.vblk, np.imag(G * F)], axis=1)
    Mq = oracle.nonuniform_matrix_q(t, 0.25, -0.1, n)
    assert np.linalg.norm(D - Mq) <= 1e-10 * np.linalg.norm(Mq)


@pytest.mark.parametrize("n", [16384, 8192])
def test_gpu_setup_long_axis_transform(torch_dev, n):
    """The longest axes: a plan set up on the GPU transforms like the oracle (sampled rows)."""
    torch, dev = torch_dev
    from paper_1901_07275_gb300 import Transform

    a, b = 0.1, -0.3
    prec = "fp32" if n == 16384 else "split"
    T = Transform((n,), [a], [b], precision=prec, setup_device=True)
    alpha = syn.normal(940 + n, 0, (1, n))
    f = T.forward(torch.tensor(alpha, dtype=T.dtype, device=dev)).double().cpu().numpy()
    rows = np.union1d(np.unique(syn.integers(941 + n, 3, 48, 0, n)), [0, n - 1])
    Q = oracle.uniform_rows(a, b, n, rows)
    tol = 1e-5 if prec == "fp32" else 1e-10
    assert np.linalg.norm(f[:, rows] - alpha @ Q.T) <= tol * np.linalg.norm(alpha @ Q.T)
