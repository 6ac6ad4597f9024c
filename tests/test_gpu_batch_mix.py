"""The whole serving mix as one batch, every member against the oracle.

The mix: 512 transforms, a fair coin between 1-D (n log-uniform in [256, 16384]) and 2-D (n_x,
n_y each log-uniform in [64, 1024]); (a, b) uniform in (-0.5, 0.5) per axis; 1..16 right-hand
sides.  It runs through ``Batch`` (jt_batch_forward / jt_batch_adjoint) in FP32 (eps 1e-7) and
in split precision (eps 1e-12) on the seeded inputs of the host generator.  The forward is the
uniform transform W J of Sec. 3.1 (Eq. tf:transout) along every axis, the adjoint its
transpose (Eq. eq:oneJinv); in d dimensions the axes are swept as in Eq. eq:TJ.

Oracle: the dense W J of each axis where that matrix is cheap to build (every 2-D member and
1-D members up to n = 2048), every output compared; for longer 1-D axes 68 seeded rows of W J
(the two ends included): the forward on those rows, and the adjoint of an input that is zero
off those rows, whose every output the rows determine.  The oracle runs in spawned worker
processes while the GPU works.  Bar: relative l2 error per member and direction <= 1e-5 (FP32)
and <= 1e-10 (split).
"""

import concurrent.futures as cf
import multiprocessing as mp
import os

import numpy as np
import pytest

from paper_1901_07275_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

COUNT = 512
FULL_1D_MAX = 2048
TOL = {"fp32": 1e-5, "split": 1e-10}
EPS = {"fp32": 1e-7, "split": 1e-12}


def _oracle_tables(job):
    """(member index, kind, tables): dense W J per axis ("full"), or the sampled rows of W J
    of a long 1-D axis ("rows")."""
    import oracle

    i, n, ab, rows = job
    if rows is None:
        return i, "full", [oracle.uniform_matrix(a, b, m) for m, (a, b) in zip(n, ab)]
    return i, "rows", oracle.uniform_rows(ab[0][0], ab[0][1], n[0], rows)


def _inputs(i, m):
    """Seeded coefficients of member i, and the adjoint's input (zero off the sampled rows for
    a long 1-D member)."""
    shape = (m["nrhs"],) + tuple(m["n"])
    x = syn.normal(5000 + i, 0, shape)
    rows = _rows(i, m)
    if rows is None:
        return x, x, None
    g = np.zeros(shape)
    g[:, rows] = syn.normal(5000 + i, 1, (m["nrhs"], rows.size))
    return x, g, rows


def _rows(i, m):
    n = m["n"]
    if len(n) == 2 or n[0] <= FULL_1D_MAX:
        return None
    r = np.unique(syn.integers(5000 + i, 3, 64, 0, n[0]))
    return np.union1d(r, [0, 1, n[0] - 2, n[0] - 1])


@pytest.fixture(scope="module")
def mix_and_oracle():
    """The mix, and the oracle's tables computed in spawned processes (started before any GPU
    work of this module and collected lazily)."""
    mix = syn.batch_mix(COUNT)
    jobs = [(i, m["n"], m["ab"], _rows(i, m)) for i, m in enumerate(mix)]
    # largest first, so the pool's tail is short
    jobs.sort(key=lambda j: -(np.prod(j[1]) * max(j[1]) if j[3] is None else j[1][0] * 4))
    ex = cf.ProcessPoolExecutor(max_workers=min(16, os.cpu_count() or 1), mp_context=mp.get_context("spawn"))
    futs = [ex.submit(_oracle_tables, j) for j in jobs]
    tables = {}

    def get(i):
        while i not in tables:
            for f in cf.as_completed(futs):
                k, kind, t = f.result()
                tables[k] = (kind, t)
                futs.remove(f)
                break
        return tables[i]

    inputs = [_inputs(i, m) for i, m in enumerate(mix)]
    yield mix, get, inputs
    ex.shutdown(wait=True, cancel_futures=True)


@pytest.fixture(scope="module")
def torch_dev():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    return torch, torch.device("cuda:0")


def _rel(x, ref):
    return float(np.linalg.norm(x - ref) / max(np.linalg.norm(ref), 1e-300))


@pytest.mark.parametrize("prec", ["fp32", "split"])
def test_serving_mix_batch_every_member_against_oracle(torch_dev, mix_and_oracle, prec):
    torch, dev = torch_dev
    import oracle
    from paper_1901_07275_gb300 import Batch, Transform

    mix, tables, inputs = mix_and_oracle
    dtype = torch.float32 if prec == "fp32" else torch.float64
    Ts = Transform.create_many([{"n": m["n"], "a": [p[0] for p in m["ab"]], "b": [p[1] for p in m["ab"]],
                                 "eps": EPS[prec], "precision": prec} for m in mix])
    xs, gs, rows = [], [], []
    for i, m in enumerate(mix):
        x, g, r = inputs[i]
        xs.append(torch.tensor(x, dtype=dtype, device=dev))
        gs.append(torch.tensor(g, dtype=dtype, device=dev))
        rows.append(r)
    batch = Batch(Ts, [m["nrhs"] for m in mix])
    fs = batch.forward(xs)
    adj = batch.adjoint(gs)
    torch.cuda.synchronize()
    worst = {"forward": (0.0, -1), "adjoint": (0.0, -1)}
    failures = []
    for i, m in enumerate(mix):
        kind, t = tables(i)
        # the oracle sees the inputs the kernels saw (FP32-rounded for FP32 plans)
        x = xs[i].double().cpu().numpy()
        g = gs[i].double().cpu().numpy()
        f = fs[i].double().cpu().numpy()
        a = adj[i].double().cpu().numpy()
        if kind == "full":
            ef = _rel(f, oracle.forward(x, t))
            ea = _rel(a, oracle.adjoint(g, t))
        else:
            r = rows[i]
            ef = _rel(f[:, r], x @ t.T)
            ea = _rel(a, g[:, r] @ t)
        for name, e in (("forward", ef), ("adjoint", ea)):
            if not e <= TOL[prec]:
                failures.append((i, m["n"], name, e))
            if e > worst[name][0]:
                worst[name] = (e, i)
    batch.close()
    for T in Ts:
        T.close()
    print(f"{prec}: worst forward {worst['forward']}, worst adjoint {worst['adjoint']}")
    assert not failures, failures[:10]
