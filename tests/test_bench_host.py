"""Host-side pieces of bench.py that need no GPU: the DRAM traffic recorded from an ncu capture
is reported only while the kernel sources it was taken from are unchanged, and the algorithmic
work and byte counts follow the per-fibre formula r (5 L log2 L + 8 n) + 55 n."""

import hashlib
import os
import shutil

import pytest

import bench

CSRC = os.path.join(bench.ROOT, "paper_1901_07275_gb300", "csrc")


def _copy_tree(tmp_path, edit=None):
    root = tmp_path / "repo"
    (root / "profiles").mkdir(parents=True)
    (root / "paper_1901_07275_gb300" / "csrc").mkdir(parents=True)
    shutil.copy(os.path.join(bench.ROOT, "profiles", "axis_kernels_2d512_fp32_traffic.txt"), root / "profiles")
    for f in ("jt_warp.cuh", "jt_axis.cuh"):
        text = open(os.path.join(CSRC, f)).read()
        if edit and f == "jt_axis.cuh":
            text += edit
        (root / "paper_1901_07275_gb300" / "csrc" / f).write_text(text)
    return str(root)


def test_traffic_reported_for_the_captured_sources(tmp_path, monkeypatch):
    fields = dict(l.split(":", 1) for l in open(os.path.join(bench.ROOT, "profiles", "axis_kernels_2d512_fp32_traffic.txt"))
                  if ":" in l and not l.startswith("#"))
    src = "".join(open(os.path.join(CSRC, f)).read() for f in ("jt_warp.cuh", "jt_axis.cuh"))
    current = hashlib.sha256(src.encode()).hexdigest()[:16] == fields["kernel_source_sha256_16"].strip()
    monkeypatch.setattr(bench, "ROOT", _copy_tree(tmp_path))
    got = bench.captured_traffic()
    if current:
        assert got == pytest.approx(float(fields["traffic_bytes_per_launch"]))
    else:
        assert got is None


def test_traffic_withdrawn_once_a_kernel_source_changes(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", _copy_tree(tmp_path, edit="\n// changed\n"))
    assert bench.captured_traffic() is None


def test_algorithmic_counts():
    # one fibre of n = L = 512 at rank 10: 10 (5 * 512 * 9 + 8 * 512) + 55 * 512
    assert bench.axis_flops(512, 512, 10) == 10 * (5 * 512 * 9 + 8 * 512) + 55 * 512
    # tables read once a launch: v (r x L) and u (r x n) complex, bins, dense block, twiddles
    b = bench.axis_table_bytes(512, 512, 10, 27, 4)
    assert b == 10 * 512 * 8 + 10 * 512 * 8 + 4 * 512 + 27 * 512 * 4 + 512 * 8 + 4 * (256 + 2) + 4 * 512
    assert bench.aggregate(2, 1000.0, 5, 10.0) == pytest.approx(2 * 1000.0 * 5 / 0.010)


def test_double_word_flops_per_real_operation():
    """The split roofline's count: a real sum costs SloppyDWPlusDW's 11 FP32 operations, a real
    product the FMA-based DWTimesDW's 9 operations of which 3 are FMAs (12 flops), and the FFT
    count 5 L log2 L is 6 sums to 4 products (a radix-2 butterfly)."""
    sums, products = 6, 4
    assert bench.DW_FLOPS_PER_FLOP == pytest.approx((sums * 11 + products * (9 + 3)) / (sums + products))
    assert bench.DW_FLOPS_PER_FLOP == pytest.approx(11.4)
