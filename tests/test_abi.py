"""The C-ABI library loads, exports every symbol ``include/jt.h`` declares, and rejects
bad arguments on the host (no GPU needed for any of this)."""

import ctypes
import os
import re

import pytest

from paper_1901_07275_gb300 import binding as B
from paper_1901_07275_gb300 import build as build_mod

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build_mod.build()
    return B.lib()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "jt.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(jt_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(B.EXPORTS) == names


def test_defaults_and_status_strings(lib):
    o = B.Options()
    lib.jt_options_default(ctypes.byref(o))
    assert (o.prec, o.nu0, o.rank_cap, o.oversample_q, o.fft_len_policy, o.autotune, o.kind, o.setup_device) == (
        0, 27, 0, 3, 0, 0, 0, 0)
    for s in range(7):
        assert B.status_string(s).startswith("JT_")


@pytest.mark.parametrize(
    "kw",
    [
        dict(n=[64], a=[1.0], b=[0.0]),
        dict(n=[64], a=[0.0], b=[-1.0]),
        dict(n=[64], a=[float("nan")], b=[0.0]),
        dict(n=[0], a=[0.0], b=[0.0]),
        dict(n=[64], a=[0.0], b=[0.0], eps=0.0),
        dict(n=[64], a=[0.0], b=[0.0], eps=1.5),
        dict(n=[8, 8, 8, 8], a=[0.0] * 4, b=[0.0] * 4),
    ],
)
def test_plan_create_rejects_bad_arguments(lib, kw):
    eps = kw.pop("eps", 1e-7)
    with pytest.raises(B.JTError) as e:
        B.jt_plan_create(kw["n"], kw["a"], kw["b"], None, eps)
    assert e.value.status == B.JT_EINVAL


def test_plan_create_rejects_points_outside_interval(lib):
    with pytest.raises(B.JTError) as e:
        B.jt_plan_create([4], [0.0], [0.0], [[0.1, 0.2, 3.2, 1.0]], 1e-7)
    assert e.value.status == B.JT_EINVAL


def test_too_long_axis_is_not_supported(lib):
    with pytest.raises(B.JTError) as e:
        B.jt_plan_create([16385], [0.0], [0.0], None, 1e-7)
    assert e.value.status == B.JT_ENOTSUP
    with pytest.raises(B.JTError) as e:
        B.jt_plan_create([16385], [0.0], [0.0], None, 1e-12, B.options("split"))
    assert e.value.status == B.JT_ENOTSUP


def test_transform_calls_reject_null_plan(lib):
    for fn in (lib.jt_forward, lib.jt_adjoint, lib.jt_inverse):
        assert fn(None, None, None, 1, None) == B.JT_EINVAL
    assert lib.jt_plan_info(None, 0, None, None, None, None) == B.JT_EINVAL
    lib.jt_destroy(None)  # NULL-safe


def test_axis_tables_reject_bad_arguments(lib):
    for args in [(0, 0.0, 0.0), (10, -1.0, 0.0), (10, 0.0, 1.0)]:
        with pytest.raises(B.JTError):
            B.AxisTables(*args)


def test_plan_load_rejects_malformed_bytes_before_any_gpu_call(lib):
    """jt_plan_load checks magic, version, checksum and every size on the host; none of these
    buffers reaches the device upload (this test runs without a GPU)."""
    bad = [b"", b"JTPLAN", b"\x00" * 64, b"JTPLAN\x00\x01" + b"\x00" * 40,
           b"JTPLAN\x00\x01" + bytes(range(200))]
    for data in bad:
        with pytest.raises(B.JTError) as e:
            B.jt_plan_load(data)
        assert e.value.status == B.JT_EINVAL
    h = ctypes.c_void_p()
    assert lib.jt_plan_load(ctypes.byref(h), None, 100, None) == B.JT_EINVAL
    assert lib.jt_plan_load(None, b"x", 1, None) == B.JT_EINVAL


def test_plan_save_and_create_many_argument_checks(lib):
    size = ctypes.c_size_t(0)
    assert lib.jt_plan_save(None, None, ctypes.byref(size)) == B.JT_EINVAL
    assert lib.jt_plan_create_many(0, None, None, None) == B.JT_OK
    assert lib.jt_plan_create_many(-1, None, None, None) == B.JT_EINVAL
    # a descriptor with a parameter outside (-1, 1) is rejected before any setup or upload
    with pytest.raises(B.JTError) as e:
        B.jt_plan_create_many([{"n": [64], "a": [0.1], "b": [0.2]}, {"n": [64], "a": [1.5], "b": [0.2]}])
    assert e.value.status == B.JT_EINVAL
    assert lib.jt_plan_shape(None, None, None, None, None, None) == B.JT_EINVAL


def test_gpu_setup_needs_a_device(lib):
    """setup_device = 1 runs the O(n^2) setup steps on the GPU: without a usable device the
    host setup entry point reports JT_ECUDA instead of falling back to the host."""
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    opt = B.options("fp32", setup_device=1)
    with pytest.raises(B.JTError) as e:
        B.AxisTables(256, 0.1, 0.2, eps=1e-7, opt=opt)
    assert e.value.status == B.JT_ECUDA
    opt.setup_device = 2
    with pytest.raises(B.JTError) as e:
        B.AxisTables(256, 0.1, 0.2, eps=1e-7, opt=opt)
    assert e.value.status == B.JT_EINVAL
