"""jt_forward_plain_noalloc: the forward transform of a plain-FP64 plan without any device
allocation.

The plain FP64 path needs work buffers beyond its input and output.  jt_forward takes them
from the plan; this entry point takes them from one fixed 16 MiB array compiled into the
library instead.  It exists for callers that must not ask for device memory while they run:
a serving loop that cannot risk an allocation failure or the allocator's locks in the middle
of a request, or a process whose free device memory is already held by another allocator.
These tests call it through the C ABI and compare it with jt_forward on the same plan, on two
calls in a row (the second call finds the previous call's data in the shared array), up to the
largest documented size (512 x 512, 12 MiB of the 16 MiB), and check that a call leaves the
device's free memory unchanged.  This
file is collected last so that a run stopping at its first failure has run everything else.
"""

import numpy as np
import pytest

from paper_1901_07275_gb300 import binding as B
from paper_1901_07275_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

TOL = 1e-10  # the tolerance of the plain FP64 path in the parity tests


@pytest.fixture(scope="module")
def torch_dev():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    return torch, torch.device("cuda:0")


@pytest.mark.parametrize(
    "n,ab",
    [((128, 96), [(0.3, -0.4), (-0.5, 0.2)]), ((1000,), [(-0.25, 0.5)]), ((16, 24, 20), [(0.1, 0.2)] * 3),
     ((512, 512), [(0.3, -0.4), (-0.5, 0.2)])],
)
def test_noalloc_forward_matches_jt_forward_on_two_calls(torch_dev, n, ab):
    torch, dev = torch_dev
    stream = torch.cuda.current_stream().cuda_stream
    plan = B.jt_plan_create(n, [p[0] for p in ab], [p[1] for p in ab], None, 1e-12, B.options("fp64_plain"), stream)
    try:
        x = torch.tensor(syn.normal(41, 0, (2,) + n), dtype=torch.float64, device=dev)
        ref = torch.empty_like(x)
        B.jt_forward(plan, x.data_ptr(), ref.data_ptr(), 2, stream)
        outs = [torch.full_like(x, float("nan")) for _ in range(2)]
        torch.cuda.synchronize()
        for i in range(2):
            free0 = torch.cuda.mem_get_info(dev)[0]
            B.jt_forward_plain_noalloc(plan, x.data_ptr(), outs[i].data_ptr(), 2, stream)
            torch.cuda.synchronize()
            free1 = torch.cuda.mem_get_info(dev)[0]
            # the call itself asks the device for nothing
            assert free1 == free0, (free0, free1)
            err = float((outs[i] - ref).norm() / ref.norm())
            assert np.isfinite(err) and err <= TOL, err
    finally:
        B.jt_destroy(plan)


def test_noalloc_rejects_plans_it_cannot_serve(torch_dev):
    torch, dev = torch_dev
    stream = torch.cuda.current_stream().cuda_stream
    big = B.jt_plan_create((1024, 1024), [0.1, 0.1], [0.2, 0.2], None, 1e-8, B.options("fp64_plain"), stream)
    # just past a power of two: each FFT length doubles, so the work space passes 16 MiB
    odd = B.jt_plan_create((513, 513), [0.1, 0.1], [0.2, 0.2], None, 1e-8, B.options("fp64_plain"), stream)
    fp32 = B.jt_plan_create((64,), [0.1], [0.2], None, 1e-7, B.options("fp32"), stream)
    try:
        x = torch.zeros((1024, 1024), dtype=torch.float64, device=dev)
        with pytest.raises(B.JTError) as e:
            B.jt_forward_plain_noalloc(big, x.data_ptr(), x.data_ptr(), 1, stream)
        assert e.value.status == B.JT_EINVAL
        z = torch.zeros((513, 513), dtype=torch.float64, device=dev)
        with pytest.raises(B.JTError) as e:
            B.jt_forward_plain_noalloc(odd, z.data_ptr(), z.data_ptr(), 1, stream)
        assert e.value.status == B.JT_EINVAL
        y = torch.zeros(64, dtype=torch.float64, device=dev)
        with pytest.raises(B.JTError) as e:
            B.jt_forward_plain_noalloc(fp32, y.data_ptr(), y.data_ptr(), 1, stream)
        assert e.value.status == B.JT_ENOTSUP
    finally:
        B.jt_destroy(big)
        B.jt_destroy(odd)
        B.jt_destroy(fp32)
