"""Second-kind transforms (jt_options.kind = JT_SECOND_KIND): the same fused kernels applied
with Im(B o F) and the second-kind dense block, against the oracle's quadrature-based Q~
(oracle/second_kind.py).  Tolerances as for the first kind: relative l2 1e-5 (FP32) and
1e-10 (split)."""

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


def make(n, ab, prec, points=None):
    from paper_1901_07275_gb300 import Transform

    return Transform(n, [p[0] for p in ab], [p[1] for p in ab], points=points, eps=EPS[prec], precision=prec,
                     kind="second")


def dt(torch, prec):
    return torch.float32 if prec == "fp32" else torch.float64


@pytest.mark.parametrize("prec", ["fp32", "split"])
@pytest.mark.parametrize("n", [5, 27, 100, 512, 1000])
def test_1d_second_kind(torch_dev, prec, n):
    torch, dev = torch_dev
    ab = [(0.3, -0.4)]
    T = make((n,), ab, prec)
    alpha = syn.normal(800 + n, 0, (3, n))
    x = torch.tensor(alpha, dtype=dt(torch, prec), device=dev)
    M = [oracle.axis_matrix_q(n, *ab[0])]
    assert rel(T.forward(x).double().cpu().numpy(), oracle.forward(alpha, M)) < TOL[prec]
    assert rel(T.adjoint(x).double().cpu().numpy(), oracle.adjoint(alpha, M)) < TOL[prec]


@pytest.mark.parametrize("prec", ["fp32", "split"])
def test_2d_second_kind_uniform(torch_dev, prec):
    torch, dev = torch_dev
    n = (96, 130)
    ab = [(-0.25, 0.5), (0.45, -0.2)]
    T = make(n, ab, prec)
    alpha = syn.normal(801, 0, (2,) + n)
    x = torch.tensor(alpha, dtype=dt(torch, prec), device=dev)
    M = [oracle.axis_matrix_q(m, a, b) for m, (a, b) in zip(n, ab)]
    assert rel(T.forward(x).double().cpu().numpy(), oracle.forward(alpha, M)) < TOL[prec]
    assert rel(T.adjoint(x).double().cpu().numpy(), oracle.adjoint(alpha, M)) < TOL[prec]


def test_2d_second_kind_nonuniform_fp32(torch_dev):
    torch, dev = torch_dev
    n = (256, 200)
    ab = [(0.25, 0.25), (0.25, 0.25)]
    pts = [np.sort(np.pi * syn.uniform(1006, 2, (m,), offset=k * 100000)) for k, m in enumerate(n)]
    T = make(n, ab, "fp32", points=pts)
    alpha = syn.normal(802, 0, n)
    x = torch.tensor(alpha, dtype=torch.float32, device=dev)
    M = [oracle.axis_matrix_q(m, a, b, p) for m, (a, b), p in zip(n, ab, pts)]
    assert rel(T.forward(x).double().cpu().numpy(), oracle.forward(alpha, M)) < TOL["fp32"]
    assert rel(T.adjoint(x).double().cpu().numpy(), oracle.adjoint(alpha, M)) < TOL["fp32"]


@pytest.mark.parametrize("ks", [1, 4])
def test_second_kind_long_axis_sampled(torch_dev, ks):
    """n = 6000 (L = 8192, general kernel), 64 sampled output rows; with and without rank split."""
    torch, dev = torch_dev
    n = 6000
    a, b = -0.2, 0.35
    T = make((n,), [(a, b)], "fp32")
    T.set_ksplit(ks)
    alpha = syn.normal(803, 0, (2, n))
    f = T.forward(torch.tensor(alpha, dtype=torch.float32, device=dev)).double().cpu().numpy()
    rows = np.union1d(np.unique(syn.integers(804, 3, 64, 0, n)), [0, n - 1])
    t, _, _, w = oracle.gauss_jacobi(a, b, n)
    Qr = (np.sqrt(w[rows])[:, None] * oracle.modified_second_kind(t[rows], a, b, n)).astype(np.float64)
    assert rel(f[:, rows], alpha @ Qr.T) < TOL["fp32"]


def test_second_kind_has_no_inverse_and_no_plain_path(torch_dev):
    torch, dev = torch_dev
    from paper_1901_07275_gb300 import Transform
    from paper_1901_07275_gb300 import binding as B

    T = make((64,), [(0.1, 0.2)], "fp32")
    x = torch.zeros(64, dtype=torch.float32, device=dev)
    with pytest.raises(B.JTError) as e:
        T.inverse(x)
    assert e.value.status == B.JT_ENOTSUP
    with pytest.raises(B.JTError) as e:
        Transform((64,), [0.1], [0.2], precision="fp64_plain", kind="second")
    assert e.value.status == B.JT_ENOTSUP


def test_second_kind_in_a_batch(torch_dev):
    """A batch may mix first- and second-kind plans; each member equals its own run."""
    torch, dev = torch_dev
    from paper_1901_07275_gb300 import Batch, Transform

    Ts = [Transform((300,), [0.1], [0.2], kind="second"), Transform((64, 90), [0.3, -0.1], [0.0, 0.2]),
          Transform((700,), [-0.3], [0.4], kind="second")]
    xs = [torch.tensor(syn.normal(805 + i, 0, (2,) + T.n), dtype=torch.float32, device=dev) for i, T in enumerate(Ts)]
    batch = Batch(Ts, [2, 2, 2])
    fb = batch.forward(xs)
    for T, x, f in zip(Ts, xs, fb):
        assert torch.equal(f, T.forward(x))
