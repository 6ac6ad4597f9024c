"""Rank split (jt_plan_set_ksplit / jt_plan_tune / jt_plan_schedule): a tile of fibres shared
by a cluster of 2, 4 or 8 CTAs, each applying a share of the rank terms, with the partial
sums added in distributed shared memory.  Every split gives the transform (against the
oracle), splits agree with one another to rounding, a split is reproducible bit for bit,
and the occupancy rule and the tuner pick valid splits."""

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


# (precision, n): the general kernel at L = 8, the four-step kernel with T = 8, 64, 256 lanes a
# fibre, the general kernel at L = 8192 (FP32 and double-word) and the 1024-thread L = 16384
@pytest.mark.parametrize(
    "prec,n",
    [("fp32", 7), ("fp32", 100), ("fp32", 1000), ("fp32", 3000), ("fp32", 5000), ("fp32", 12000),
     ("split", 100), ("split", 3000)],
)
@pytest.mark.parametrize("ks", [2, 4, 8])
def test_split_1d_matches_oracle(torch_dev, prec, n, ks):
    torch, dev = torch_dev
    ab = [(0.15, -0.35)]
    T = make((n,), ab, prec)
    T.set_ksplit(ks)
    assert T.schedule(0, 0, 3) == ks and T.schedule(0, 1, 3) == ks
    alpha = syn.normal(500 + n, 0, (3, n))
    x = torch.tensor(alpha, dtype=dt(torch, prec), device=dev)
    f = T.forward(x).double().cpu().numpy()
    g = T.adjoint(x).double().cpu().numpy()
    if n <= 1000:
        M = [oracle.axis_matrix(n, *ab[0])]
        assert rel(f, oracle.forward(alpha, M)) < TOL[prec]
        assert rel(g, oracle.adjoint(alpha, M)) < TOL[prec]
    else:
        rows = np.union1d(np.unique(syn.integers(501 + n, 3, 64, 0, n)), [0, n - 1])
        Q = oracle.uniform_rows(ab[0][0], ab[0][1], n, rows)
        assert rel(f[:, rows], alpha @ Q.T) < TOL[prec]
        # adjoint: <g, A alpha> = <A^T g, alpha> with g supported on the sampled rows
        gr = np.zeros((1, n))
        gr[0, rows] = syn.normal(502 + n, 0, (rows.size,))
        a = T.adjoint(torch.tensor(gr, dtype=dt(torch, prec), device=dev)).double().cpu().numpy()
        assert rel(a, gr[:, rows] @ Q) < TOL[prec]
    # the unsplit sweep agrees to rounding, and the split is reproducible
    T.set_ksplit(1)
    f1 = T.forward(x).double().cpu().numpy()
    assert rel(f, f1) < TOL[prec]
    T.set_ksplit(ks)
    assert torch.equal(T.forward(x), T.forward(x))


@pytest.mark.parametrize("prec", ["fp32", "split"])
@pytest.mark.parametrize("ks", [2, 8])
def test_split_2d_strided_and_in_place(torch_dev, prec, ks):
    """Both sweeps of a 2-D transform (the strided one through the cluster's fibre-major
    stores), out of place and in place."""
    torch, dev = torch_dev
    n = (37, 300)
    ab = [(0.3, -0.4), (-0.5, 0.2)]
    T = make(n, ab, prec)
    T.set_ksplit(ks)
    alpha = syn.normal(601, 0, (2,) + n)
    x = torch.tensor(alpha, dtype=dt(torch, prec), device=dev)
    M = [oracle.axis_matrix(m, a, b) for m, (a, b) in zip(n, ab)]
    f = T.forward(x)
    assert rel(f.double().cpu().numpy(), oracle.forward(alpha, M)) < TOL[prec]
    assert rel(T.adjoint(x).double().cpu().numpy(), oracle.adjoint(alpha, M)) < TOL[prec]
    z = x.clone()
    T.forward(z, out=z)
    assert torch.equal(z, f)


def test_occupancy_rule_splits_few_fibres_only(torch_dev):
    torch, dev = torch_dev
    T = make((9000,), [(0.1, 0.2)], "fp32")
    r = T.ranks[0]
    k1 = T.schedule(0, 0, 1)
    assert k1 in (2, 4, 8) and k1 <= r
    # many right-hand sides fill the GPU without a split
    assert T.schedule(0, 0, 4096) == 1
    S = make((512, 512), [(0.3, -0.4), (-0.5, 0.2)], "fp32")
    assert S.schedule(0, 0, 16) == 1 and S.schedule(1, 1, 16) == 1


def test_tune_keeps_a_measured_split(torch_dev):
    torch, dev = torch_dev
    n = 6000
    ab = [(-0.2, 0.3)]
    T = make((n,), ab, "fp32")
    T.tune(2)
    for d in (0, 1):
        assert T.schedule(0, d, 2) in (1, 2, 4, 8)
    alpha = syn.normal(700, 0, (2, n))
    f = T.forward(torch.tensor(alpha, dtype=torch.float32, device=dev)).double().cpu().numpy()
    rows = np.union1d(np.unique(syn.integers(701, 3, 64, 0, n)), [0, n - 1])
    Q = oracle.uniform_rows(ab[0][0], ab[0][1], n, rows)
    assert rel(f[:, rows], alpha @ Q.T) < TOL["fp32"]


def test_schedule_argument_errors(torch_dev):
    torch, dev = torch_dev
    from paper_1901_07275_gb300 import binding as B

    T = make((64,), [(0.0, 0.0)], "fp32")
    for args in [(3, -1, -1), (0, 2, 0), (0, 0, 5)]:
        with pytest.raises(B.JTError) as e:
            B.jt_plan_set_ksplit(T._plan, args[1], args[2], args[0])
        assert e.value.status == B.JT_EINVAL
    P = make((64,), [(0.0, 0.0)], "split")
    P.set_ksplit(0)
    from paper_1901_07275_gb300 import Transform

    Q = Transform((64,), [0.0], [0.0], precision="fp64_plain")
    with pytest.raises(B.JTError) as e:
        Q.set_ksplit(2)
    assert e.value.status == B.JT_ENOTSUP


def test_autotuned_batch_equals_members(torch_dev):
    """A batch of plans created with autotune = 1 measures the splits of its members' sweeps;
    the members then run with the same splits, so the batch equals them bit for bit."""
    torch, dev = torch_dev
    from paper_1901_07275_gb300 import Batch, Transform

    mix = syn.batch_mix(10, seed=4200, n1=(2000, 12000), n2=(64, 400), max_rhs=3)
    Ts = [Transform(m["n"], [p[0] for p in m["ab"]], [p[1] for p in m["ab"]], autotune=True) for m in mix]
    xs = [torch.tensor(syn.normal(4200 + i, 0, (m["nrhs"],) + tuple(m["n"])), dtype=torch.float32, device=dev)
          for i, m in enumerate(mix)]
    batch = Batch(Ts, [m["nrhs"] for m in mix])
    fb = batch.forward(xs)
    ab = batch.adjoint(xs)
    for T, x, f, a in zip(Ts, xs, fb, ab):
        assert torch.equal(f, T.forward(x))
        assert torch.equal(a, T.adjoint(x))
