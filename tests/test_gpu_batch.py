"""Batched execution (jt_batch_*): a serving-style mix of 1-D and 2-D transforms of uneven n,
different (a, b) and 1..16 right-hand sides, run together, equals running each member on
its own -- bit for bit, since the batched launch performs the same arithmetic -- and can be
captured in a CUDA graph and replayed."""

import numpy as np
import pytest

import oracle
from paper_1901_07275_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_dev():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    return torch, torch.device("cuda:0")


def _members(torch, dev, prec, count, seed, n1, n2):
    from paper_1901_07275_gb300 import Transform

    mix = syn.batch_mix(count, seed=seed, n1=n1, n2=n2, max_rhs=5)
    dtype = torch.float32 if prec == "fp32" else torch.float64
    Ts, xs = [], []
    for i, m in enumerate(mix):
        T = Transform(m["n"], [p[0] for p in m["ab"]], [p[1] for p in m["ab"]], precision=prec)
        Ts.append(T)
        xs.append(torch.tensor(syn.normal(seed + i, 0, (m["nrhs"],) + tuple(m["n"])), dtype=dtype, device=dev))
    return mix, Ts, xs


@pytest.mark.parametrize("prec", ["fp32", "split"])
def test_batch_equals_members_one_by_one(torch_dev, prec):
    torch, dev = torch_dev
    from paper_1901_07275_gb300 import Batch

    n1 = (16, 16384) if prec == "fp32" else (16, 4096)
    mix, Ts, xs = _members(torch, dev, prec, 28, 4000, n1, (8, 300))
    batch = Batch(Ts, [m["nrhs"] for m in mix])
    fb = batch.forward(xs)
    ab = batch.adjoint(xs)
    for T, x, f, a in zip(Ts, xs, fb, ab):
        assert torch.equal(f, T.forward(x))
        assert torch.equal(a, T.adjoint(x))
    # one member against the oracle as well
    m, x = mix[0], xs[0]
    M = [oracle.axis_matrix(n, a, b) for n, (a, b) in zip(m["n"], m["ab"])]
    ref = oracle.forward(x.double().cpu().numpy(), M)
    tol = 1e-5 if prec == "fp32" else 1e-10
    assert np.linalg.norm(fb[0].double().cpu().numpy() - ref) <= tol * np.linalg.norm(ref)


def test_batch_in_place_and_graph_replay(torch_dev):
    torch, dev = torch_dev
    from paper_1901_07275_gb300 import Batch

    mix, Ts, xs = _members(torch, dev, "fp32", 20, 4100, (32, 2048), (16, 200))
    batch = Batch(Ts, [m["nrhs"] for m in mix])
    ref = [T.forward(x) for T, x in zip(Ts, xs)]
    bufs = [x.clone() for x in xs]
    batch.forward(bufs, bufs)  # in place, warms every kernel up before capture
    for b, r in zip(bufs, ref):
        assert torch.equal(b, r)
    src = [x.clone() for x in xs]
    dst = [torch.empty_like(x) for x in xs]
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        batch.forward(src, dst, stream=stream)
    for _ in range(2):
        for d in dst:
            d.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        for d, r in zip(dst, ref):
            assert torch.equal(d, r)


def test_batch_rejects_mixed_precisions(torch_dev):
    torch, dev = torch_dev
    from paper_1901_07275_gb300 import Batch, Transform
    from paper_1901_07275_gb300 import binding as B

    T1 = Transform((64,), [0.1], [0.2], precision="fp32")
    T2 = Transform((64,), [0.1], [0.2], precision="split")
    with pytest.raises(B.JTError) as e:
        Batch([T1, T2], [1, 1])
    assert e.value.status == B.JT_EINVAL
    T3 = Transform((64,), [0.1], [0.2], precision="fp64_plain")
    with pytest.raises(B.JTError) as e:
        Batch([T3], [1])
    assert e.value.status == B.JT_ENOTSUP


def test_batch_groups_beyond_one_launch(torch_dev):
    """300 small 2-D members of one FFT length (L = 32) and one rank split: each stage's group
    holds more jobs than one launch takes (256), so it runs as two launches; the batch still
    equals the members one by one, bit for bit, and the oracle."""
    torch, dev = torch_dev
    from paper_1901_07275_gb300 import Batch, Transform

    count = 300
    Ts, xs, shapes = [], [], []
    u = syn.uniform(4200, 4, (count, 4))
    for i in range(count):
        n = (28 + i % 5, 28 + (i // 5) % 5)
        ab = [(float(u[i, 0] - 0.5), float(u[i, 1] - 0.5)), (float(u[i, 2] - 0.5), float(u[i, 3] - 0.5))]
        T = Transform(n, [p[0] for p in ab], [p[1] for p in ab], precision="fp32")
        T.set_ksplit(1)
        Ts.append(T)
        shapes.append((n, ab))
        xs.append(torch.tensor(syn.normal(4200 + i, 0, (1 + i % 3,) + n), dtype=torch.float32, device=dev))
    batch = Batch(Ts, [x.shape[0] for x in xs])
    fb = batch.forward(xs)
    ab_ = batch.adjoint(xs)
    for T, x, f, a in zip(Ts, xs, fb, ab_):
        assert torch.equal(f, T.forward(x))
        assert torch.equal(a, T.adjoint(x))
    for i in (0, 257, count - 1):
        n, ab = shapes[i]
        M = [oracle.axis_matrix(m, a, b) for m, (a, b) in zip(n, ab)]
        ref = oracle.forward(xs[i].double().cpu().numpy(), M)
        assert np.linalg.norm(fb[i].double().cpu().numpy() - ref) <= 1e-5 * np.linalg.norm(ref)
    batch.close()
    for T in Ts:
        T.close()
