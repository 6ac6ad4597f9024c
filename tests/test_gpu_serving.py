"""Serving helpers: a saved plan reloads with no setup and computes bit for bit what the
original did; corrupted bytes are rejected; plans created together equal plans created one
by one."""

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


CASES = [
    dict(n=(300,), ab=[(0.1, -0.2)], precision="fp32", kind="first"),
    dict(n=(64, 90), ab=[(0.3, -0.4), (-0.5, 0.2)], precision="split", kind="first"),
    dict(n=(40, 33), ab=[(0.2, 0.1), (-0.3, 0.25)], precision="fp64_plain", kind="first"),
    dict(n=(200,), ab=[(-0.25, 0.5)], precision="fp32", kind="second"),
    dict(n=(5000,), ab=[(0.2, 0.3)], precision="fp32", kind="first"),
]


def _make(c, points=None):
    from paper_1901_07275_gb300 import Transform

    return Transform(c["n"], [p[0] for p in c["ab"]], [p[1] for p in c["ab"]], points=points,
                     precision=c["precision"], kind=c["kind"])


@pytest.mark.parametrize("ci", range(len(CASES)))
def test_saved_plan_reloads_bit_for_bit(torch_dev, ci):
    torch, dev = torch_dev
    from paper_1901_07275_gb300 import Transform

    c = CASES[ci]
    T = _make(c)
    data = T.save()
    U = Transform.load(data)
    assert U.n == T.n and U.precision == T.precision and U.kind == T.kind and U.ranks == T.ranks
    assert U.save() == data
    x = torch.tensor(syn.normal(900 + ci, 0, (2,) + c["n"]), dtype=T.dtype, device=dev)
    assert torch.equal(T.forward(x), U.forward(x))
    assert torch.equal(T.adjoint(x), U.adjoint(x))
    if c["kind"] == "first":
        assert torch.equal(T.inverse(x), U.inverse(x))


def test_saved_nonuniform_plan(torch_dev):
    torch, dev = torch_dev
    from paper_1901_07275_gb300 import Transform

    n = (128, 96)
    pts = [np.sort(np.pi * syn.uniform(910, 2, (m,), offset=k * 1000)) for k, m in enumerate(n)]
    T = Transform(n, [0.25, 0.25], [0.25, 0.25], points=pts)
    U = Transform.load(T.save())
    assert not U.uniform
    x = torch.tensor(syn.normal(911, 0, n), dtype=torch.float32, device=dev)
    assert torch.equal(T.forward(x), U.forward(x))
    M = [oracle.axis_matrix(m, 0.25, 0.25, p) for m, p in zip(n, pts)]
    f = U.forward(x).double().cpu().numpy()
    ref = oracle.forward(x.double().cpu().numpy(), M)
    assert np.linalg.norm(f - ref) <= 1e-5 * np.linalg.norm(ref)


def test_corrupted_or_truncated_bytes_are_rejected(torch_dev):
    from paper_1901_07275_gb300 import Transform
    from paper_1901_07275_gb300 import binding as B

    data = _make(CASES[0]).save()
    for bad in (data[:-1], data[: len(data) // 2], data[:100] + bytes([data[100] ^ 1]) + data[101:]):
        with pytest.raises(B.JTError) as e:
            Transform.load(bad)
        assert e.value.status == B.JT_EINVAL


def test_create_many_equals_one_by_one(torch_dev):
    torch, dev = torch_dev
    from paper_1901_07275_gb300 import Transform

    mix = syn.batch_mix(12, seed=4300, n1=(64, 3000), n2=(16, 200), max_rhs=2)
    specs = [{"n": m["n"], "a": [p[0] for p in m["ab"]], "b": [p[1] for p in m["ab"]],
              "kind": "second" if i % 3 == 0 else "first"} for i, m in enumerate(mix)]
    many = Transform.create_many(specs)
    for i, (sp, T) in enumerate(zip(specs, many)):
        R = Transform(sp["n"], sp["a"], sp["b"], kind=sp["kind"])
        assert T.ranks == R.ranks and T.save() == R.save()
        x = torch.tensor(syn.normal(920 + i, 0, tuple(sp["n"])), dtype=torch.float32, device=dev)
        assert torch.equal(T.forward(x), R.forward(x))


@pytest.mark.parametrize("prec", ["fp32", "split"])
@pytest.mark.parametrize("direction", ["forward", "adjoint", "inverse"])
def test_transform_host_equals_device_transform(torch_dev, prec, direction):
    """Host arrays through a small work area (several chunks on the two plan streams) give the
    device transform of each right-hand side."""
    torch, dev = torch_dev
    from paper_1901_07275_gb300 import Transform

    n = (96, 130)
    T = Transform(n, [0.3, -0.5], [-0.4, 0.2], precision=prec)
    x = torch.tensor(syn.normal(1600, 0, (11,) + n), dtype=T.dtype).pin_memory()
    per = x[0].numel() * x.element_size()
    fn = {"forward": T.forward, "adjoint": T.adjoint, "inverse": T.inverse}[direction]
    # three buffers of 2 right-hand sides, and two buffers of one
    for mult in (7, 2):
        ws = torch.empty(mult * per, dtype=torch.uint8, device=dev)
        y = T.transform_host(x, direction=direction, workspace=ws)
        torch.cuda.synchronize()
        for r in range(x.shape[0]):
            ref = fn(x[r].to(dev)).cpu()
            assert torch.allclose(y[r], ref, rtol=0, atol=1e-6 * float(ref.abs().max()))


def test_transform_host_pageable_and_single_buffer(torch_dev):
    torch, dev = torch_dev
    from paper_1901_07275_gb300 import Transform
    from paper_1901_07275_gb300 import binding as B

    T = Transform((500,), [0.1], [0.2])
    x = torch.tensor(syn.normal(1601, 0, (3, 500)), dtype=torch.float32)  # pageable
    ws = torch.empty(500 * 4, dtype=torch.uint8, device=dev)  # room for one right-hand side
    y = T.transform_host(x, workspace=ws)
    torch.cuda.synchronize()
    assert torch.allclose(y, T.forward(x.to(dev)).cpu(), rtol=0, atol=1e-6)
    Q = Transform((64,), [0.1], [0.2], kind="second")
    with pytest.raises(B.JTError) as e:
        Q.transform_host(torch.zeros(64), direction="inverse")
    assert e.value.status == B.JT_ENOTSUP
    with pytest.raises(B.JTError) as e:
        T.transform_host(x, workspace=torch.empty(16, dtype=torch.uint8, device=dev))
    assert e.value.status == B.JT_EINVAL
