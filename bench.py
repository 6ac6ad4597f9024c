#!/usr/bin/env python
"""Throughput of the fast Jacobi transform on one GB300 (or N replicas).

Workload: the 2-D uniform tensor-grid transform of size 512 x 512 with (a, b) = (0.3, -0.4)
on axis 0 and (-0.5, 0.2) on axis 1, alpha i.i.d. N(0, 1) from the seeded generator,
batched over ``--nrhs`` right-hand sides (default 256, i.e. 256 MiB of FP32 input -- larger
than the 129 MB L2, so no L2 flush is needed between steps).  One step = one forward
transform followed by one inverse transform of the whole batch with the fused FP32 axis
kernels (factorisation accuracy 1e-7).  The metric is Jacobi coefficients per second:
2 * nrhs * 512^2 per step.

Also reported on the same line: the double-word (split) kernels, the plain FP64 r^2-FFT
path (cuFFT Z2Z), accuracy against the CPU oracle, the end-to-end number through host
buffers, the roofline of the axis kernel, and the oracle timed on the host cores.

``--impl reference`` times the CPU oracle (dense mode products in FP64) on a bounded
sample of the same workload and prints the same line with "impl": "reference".
"""

from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N = (512, 512)
AB = [(0.3, -0.4), (-0.5, 0.2)]
METRIC = "Jacobi coeffs/sec (2-D 512x512 forward+inverse, FP32 fused axis kernels, rel l2 <= 1e-5 vs FP64 oracle)"
UNIT = "coeffs/s"
FP32_LANES_PER_SM = 128  # used only for the nominal figure beside the measured peak
SPLIT_MAX_N = 16384  # longest axis of a split (double-word) plan


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def captured_traffic():
    """DRAM bytes per launch of the axis kernels from the committed ncu capture, or None when
    the kernel sources have changed since the counters were taken."""
    import hashlib

    path = os.path.join(ROOT, "profiles", "axis_kernels_2d512_fp32_traffic.txt")
    csrc = os.path.join(ROOT, "paper_1901_07275_gb300", "csrc")
    try:
        fields = {}
        for line in open(path):
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                fields[k.strip()] = v.strip()
        src = "".join(open(os.path.join(csrc, f)).read() for f in ("jt_warp.cuh", "jt_axis.cuh"))
        if hashlib.sha256(src.encode()).hexdigest()[:16] != fields.get("kernel_source_sha256_16"):
            return None
        return float(fields["traffic_bytes_per_launch"])
    except Exception:
        return None


# FP32 flops of the double-word arithmetic per real flop of the algorithmic count: a sum is
# SloppyDWPlusDW (11 FP32 operations), a product the FMA-based DWTimesDW (9 operations, 3 of them
# FMAs: 12 flops); the FFT count 5 L log2 L is 60 % sums and 40 % products (a radix-2 butterfly:
# 6 sums, 4 products), so one real flop costs 0.6 x 11 + 0.4 x 12 = 11.4 FP32 flops.
DW_FLOPS_PER_FLOP = 0.6 * 11 + 0.4 * 12


def axis_flops(n, L, r):
    """Algorithmic FP32 flops of one fibre of one axis: r (5 L log2 L + 8 n) + 55 n."""
    return r * (5 * L * math.log2(L) + 8 * n) + 55 * n


def axis_table_bytes(n, L, r, nu0, real_bytes):
    """Plan tables one launch reads once: v (r x L), u (r x n) complex, bins, dense block, twiddles."""
    cplx = 2 * real_bytes
    return r * L * cplx + r * n * cplx + 4 * n + nu0 * n * real_bytes + L * cplx + 4 * (L // 2 + 2) + 4 * n


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 20 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        self.gpu_index = gpu_index

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        smax = max(float(r[2]) for r in rows if r[2].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        pw = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": smax, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(pw) if pw else None}


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(world, v):
    """Largest value over all ranks (the timed region of the slowest replica)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist

    device = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(world, coeffs_per_step_per_rank, steps, total_ms):
    """Whole-job throughput of `world` replicas: all ranks' work over the slowest rank's time."""
    return world * coeffs_per_step_per_rank * steps / (total_ms * 1e-3)


# --------------------------------------------------------------- CPU oracle
def oracle_throughput(nrhs_max, target_s=12.0, threads=None):
    """Dense FP64 mode products of the oracle on a bounded sample of right-hand sides.
    Matrices are built once (their cost is reported separately); returns coeffs/s."""
    import numpy as np

    import oracle
    from paper_1901_07275_gb300 import synthetic as syn

    t0 = time.perf_counter()
    mats = [oracle.uniform_matrix(a, b, m) for (a, b), m in zip(AB, N)]
    setup_s = time.perf_counter() - t0
    probe = syn.normal(1002, 0, (1,) + N)
    t0 = time.perf_counter()
    f = oracle.forward(probe, mats)
    oracle.adjoint(f, mats)
    per_rhs = max(time.perf_counter() - t0, 1e-4)
    s = int(max(1, min(nrhs_max, target_s / per_rhs)))
    alpha = syn.normal(1002, 0, (s,) + N)
    reps = 0
    t0 = time.perf_counter()
    while True:  # repeat the batch until about target_s of CPU work has been timed
        f = oracle.forward(alpha, mats)
        oracle.adjoint(f, mats)
        reps += 1
        dt = time.perf_counter() - t0
        if dt >= target_s or reps >= 64:
            break
    coeffs = 2 * s * N[0] * N[1] * reps
    return {"value": coeffs / dt, "unit": UNIT, "cores": threads or os.cpu_count(), "kind": "oracle",
            "sample": f"{reps} x {s} right-hand sides of the 512x512 workload, forward + inverse by dense "
                      f"FP64 mode products ({dt:.1f} s); axis matrices built once in {setup_s:.1f} s, not counted",
            "seconds": dt}


def run_reference(args):
    world, rank, _ = int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), 0
    if rank != 0:
        return 0
    steps, warm = args.steps, args.warmup
    import numpy as np

    import oracle
    from paper_1901_07275_gb300 import synthetic as syn

    mats = [oracle.uniform_matrix(a, b, m) for (a, b), m in zip(AB, N)]
    probe = syn.normal(1002, 0, (1,) + N)
    t0 = time.perf_counter()
    oracle.adjoint(oracle.forward(probe, mats), mats)
    per_rhs = max(time.perf_counter() - t0, 1e-4)
    # each step: a bounded sample so that warm-up + steps end within about two minutes
    s = int(max(1, min(args.nrhs, 120.0 / ((steps + warm) * per_rhs))))
    alpha = syn.normal(1002, 0, (s,) + N)
    for _ in range(warm):
        oracle.adjoint(oracle.forward(alpha, mats), mats)
    t0 = time.perf_counter()
    for _ in range(steps):
        oracle.adjoint(oracle.forward(alpha, mats), mats)
    dt = time.perf_counter() - t0
    coeffs = 2 * s * N[0] * N[1] * steps
    v = coeffs / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": steps,
        "warmup": warm, "ms_per_step": 1e3 * dt / steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "2d-512x512 uniform, (a,b)=(0.3,-0.4)x(-0.5,0.2)", "nrhs": s,
                   "step": "forward + inverse", "l2": "host CPU run"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                         "sample": f"{s} right-hand sides per step, dense FP64 mode products"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# --------------------------------------------------------------- GPU arm
def fp32_peak(dev, stream, gpu_index):
    """The FP32 rate that bounds the axis kernels, measured: jt_probe_fp32_fma (independent FMA
    chains over 4 CTAs of 256 threads per SM) as one FMA an instruction and as two
    (fma.rn.f32x2), each launch about 50 ms, timed with CUDA events on the launching stream
    with the clocks sampled during it; the best of 3 launches per form."""
    import torch

    from paper_1901_07275_gb300 import binding as B

    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sink = torch.empty(1024 * sms, dtype=torch.float32, device=dev)
    out = {"sm_count": sms}
    iters = 100000
    for label, paired in (("fma_f32", False), ("fma_f32x2", True)):
        B.jt_probe_fp32_fma(paired, 1000, sink.data_ptr(), sink.numel(), stream.cuda_stream)  # warm-up
        torch.cuda.synchronize()
        best = None
        with ClockSampler(gpu_index) as clk:
            for _ in range(3):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                flops = B.jt_probe_fp32_fma(paired, iters, sink.data_ptr(), sink.numel(), stream.cuda_stream)
                e1.record(stream)
                torch.cuda.synchronize()
                tf = flops / (e0.elapsed_time(e1) * 1e-3) / 1e12
                best = tf if best is None else max(best, tf)
        c = clk.summary()
        out[label] = {"tflops": best, "sm_mhz": c["sm_mhz"], "clock_samples": c["samples"], "reasons": c["reasons"]}
    out["peak_tflops"] = max(out["fma_f32"]["tflops"], out["fma_f32x2"]["tflops"])
    return out


def other_configs(dev, stream):
    """Throughput of the FP32 kernels on the other workloads (forward + inverse/adjoint per
    step, CUDA events, 2 warm-up and 3 timed steps each)."""
    import torch

    from paper_1901_07275_gb300 import Transform
    from paper_1901_07275_gb300 import synthetic as syn

    out = {}
    cases = [
        ("1d-1024 x 1 rhs", "1d-1024", 1),
        ("1d-1024 x 256 rhs", "1d-1024", 256),
        ("1d-1024 x 8192 rhs", "1d-1024", 8192),
        ("3d-256", "3d-256", 1),
        ("2d-nonuniform-1024 x 16 rhs (forward + adjoint)", "2d-nonuniform-1024", 16),
    ]
    for label, name, nr in cases:
        w = syn.workload(name, nrhs=1)
        T = Transform(w["n"], [p[0] for p in w["ab"]], [p[1] for p in w["ab"]], points=w["points"], eps=1e-7)
        x = torch.tensor(w["alpha"], dtype=torch.float32, device=dev).expand((nr,) + tuple(w["n"])).contiguous()
        f = torch.empty_like(x)
        y = torch.empty_like(x)
        back = T.inverse if T.uniform else T.adjoint

        def step():
            T.forward(x, out=f)
            back(f, out=y)

        for _ in range(2):
            step()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        # small cases: enough steps for about 20 ms of timed work
        torch.cuda.synchronize()
        e0.record(stream)
        step()
        e1.record(stream)
        torch.cuda.synchronize()
        reps = int(min(2000, max(3, 20.0 / max(e0.elapsed_time(e1), 1e-3))))
        e0.record(stream)
        for _ in range(reps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        coeffs = 2 * x.numel()
        total = x.numel()
        flops = 0.0
        for ax, m in enumerate(w["n"]):
            flops += 2 * (total // m) * axis_flops(m, T.fft_lens[ax], T.ranks[ax])
        out[label] = {"coeffs_per_s": coeffs / (ms * 1e-3), "ms_per_step": ms, "steps_timed": reps,
                      "ranks": T.ranks, "fft_len": T.fft_lens,
                      "rank_split": [T.schedule(a, 0, nr) for a in range(len(w["n"]))],
                      "algorithmic_tflops": flops / (ms * 1e-3) / 1e12}
        T.close()
        del x, f, y
    return out


def paper_configs(dev, stream):
    """Two comparisons the method is judged on, beside the FP32 kernels.

    1-D, n = 1024, (a, b) = (-0.25, 0.5), eps 1e-12 (1e-7 for FP32): the plain FP64 r-term FFT
    path (cuFFT Z2Z), the double-word kernels and the FP32 kernels, forward + inverse of 1 and of
    256 right-hand sides, each forward's relative error against the oracle's dense matrix.

    3-D 256^3 with the FP32 plan's accuracy (eps 1e-7, ranks 9 a axis): one forward of one
    right-hand side by the plain FP64 r^3 path (2^(d-1) r^3 = 2916 three-dimensional FFTs for the
    all-high-degree block) against the FP32 fused kernels, with the relative difference of the
    two results."""
    import numpy as np
    import torch

    import oracle
    from paper_1901_07275_gb300 import Transform
    from paper_1901_07275_gb300 import synthetic as syn

    out = {}
    w = syn.workload("1d-1024", nrhs=256)
    (a, b), n = w["ab"][0], w["n"][0]
    ref = oracle.forward(w["alpha"][:1], [oracle.uniform_matrix(a, b, n)])
    for prec, eps in (("fp64_plain", 1e-12), ("split", 1e-12), ("fp32", 1e-7)):
        T = Transform((n,), [a], [b], eps=eps, precision=prec)
        dt = torch.float32 if prec == "fp32" else torch.float64
        row = {"rank": T.ranks[0], "eps": eps}
        for nr in (1, 256):
            x = torch.tensor(w["alpha"][:nr], dtype=dt, device=dev)
            f = torch.empty_like(x)
            y = torch.empty_like(x)
            for _ in range(2):
                T.forward(x, out=f)
                T.inverse(f, out=y)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 20
            e0.record(stream)
            for _ in range(reps):
                T.forward(x, out=f)
                T.inverse(f, out=y)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            row[f"{nr}_rhs"] = {"ms_per_step": ms, "coeffs_per_s": 2 * x.numel() / (ms * 1e-3)}
            if nr == 1:
                row["rel_err_forward"] = float(np.linalg.norm(f.double().cpu().numpy() - ref) / np.linalg.norm(ref))
        out[f"1d-1024 {prec}"] = row
        T.close()
    plain = out["1d-1024 fp64_plain"]
    for prec in ("split", "fp32"):
        for nr in (1, 256):
            out[f"1d-1024 {prec}"][f"speedup_over_plain_{nr}_rhs"] = (
                plain[f"{nr}_rhs"]["ms_per_step"] / out[f"1d-1024 {prec}"][f"{nr}_rhs"]["ms_per_step"])

    w = syn.workload("3d-256", nrhs=1)
    res = {}
    fwd = {}
    for prec in ("fp64_plain", "fp32"):
        T = Transform(w["n"], [p[0] for p in w["ab"]], [p[1] for p in w["ab"]], eps=1e-7, precision=prec)
        dt = torch.float32 if prec == "fp32" else torch.float64
        x = torch.tensor(w["alpha"], dtype=dt, device=dev)
        f = torch.empty_like(x)
        T.forward(x, out=f)  # warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 1 if prec == "fp64_plain" else 10
        e0.record(stream)
        for _ in range(reps):
            T.forward(x, out=f)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        res[prec] = {"forward_ms": ms, "coeffs_per_s": x.numel() / (ms * 1e-3), "ranks": T.ranks,
                     "forwards_timed": reps}
        fwd[prec] = f.double().cpu().numpy()
        T.close()
        del x, f
    res["speedup_fp32_over_plain"] = res["fp64_plain"]["forward_ms"] / res["fp32"]["forward_ms"]
    res["rel_diff_fp32_vs_plain"] = float(np.linalg.norm(fwd["fp32"] - fwd["fp64_plain"]) / np.linalg.norm(fwd["fp64_plain"]))
    out["3d-256 forward, eps 1e-7"] = res
    return out


def setup_timings():
    """Plan creation time (host FP64/double-word setup, then the upload) for the longest axes,
    with the O(n^2) steps on the host cores or in FP64 kernels on the GPU (setup_device)."""
    from paper_1901_07275_gb300 import Transform

    out = {}
    for label, n, prec, eps in (("1d-16384 fp32 eps 1e-7", 16384, "fp32", 1e-7),
                                ("1d-8192 split eps 1e-12", 8192, "split", 1e-12),
                                ("1d-4096 fp32 eps 1e-7", 4096, "fp32", 1e-7)):
        row = {}
        for dev_setup in (False, True):
            t0 = time.perf_counter()
            T = Transform((n,), [0.1], [-0.3], eps=eps, precision=prec, setup_device=dev_setup)
            row["gpu_setup_s" if dev_setup else "host_setup_s"] = time.perf_counter() - t0
            row["rank_gpu_setup" if dev_setup else "rank_host_setup"] = T.ranks[0]
            T.close()
        out[label] = row
    return out


def sweep_times(dev, stream):
    """Per-sweep times of the bench workload: the 2-D forward and adjoint, and the same 1-D
    plan as the 2-D plan's contiguous axis over all 512 x nrhs fibres; the strided sweep is the
    difference.  FP32 with 256 right-hand sides, split with 64."""
    import torch

    from paper_1901_07275_gb300 import Transform

    def timed(fn, reps=20):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    out = {}
    for prec, nr, eps in (("fp32", 256, 1e-7), ("split", 64, 1e-12)):
        dt = torch.float32 if prec == "fp32" else torch.float64
        T2 = Transform(N, [p[0] for p in AB], [p[1] for p in AB], eps=eps, precision=prec)
        T1 = Transform((N[1],), [AB[1][0]], [AB[1][1]], eps=eps, precision=prec)
        x = torch.randn((nr,) + N, device=dev, dtype=dt)
        y = torch.empty_like(x)
        x1, y1 = x.reshape(-1, N[1]), y.reshape(-1, N[1])
        r = {"nrhs": nr, "ranks": T2.ranks}
        r["forward_2d_ms"] = timed(lambda: T2.forward(x, out=y))
        r["adjoint_2d_ms"] = timed(lambda: T2.adjoint(x, out=y))
        r["forward_contiguous_ms"] = timed(lambda: T1.forward(x1, out=y1))
        r["adjoint_contiguous_ms"] = timed(lambda: T1.adjoint(x1, out=y1))
        r["forward_strided_ms"] = r["forward_2d_ms"] - r["forward_contiguous_ms"]
        r["adjoint_strided_ms"] = r["adjoint_2d_ms"] - r["adjoint_contiguous_ms"]
        out[prec] = r
        T1.close()
        T2.close()
        del x, y
    return out


def fac_and_app(dev, stream):
    """Factorisation (plan creation: host setup, or its O(n^2) steps on the GPU, then the
    upload) beside application (one forward of one right-hand side, CUDA events) for the
    workloads, as the paper reports fac and app times side by side (Sec. 4)."""
    import torch

    from paper_1901_07275_gb300 import Transform
    from paper_1901_07275_gb300 import synthetic as syn

    out = {}
    cases = [("1d-1024", "fp32", 1e-7), ("1d-1024", "split", 1e-12), ("2d-512", "fp32", 1e-7),
             ("2d-512", "split", 1e-12), ("3d-256", "fp32", 1e-7), ("2d-nonuniform-1024", "fp32", 1e-7)]
    for name, prec, eps in cases:
        w = syn.workload(name, nrhs=1)
        row = {"eps": eps}
        for dev_setup in (False, True):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            T = Transform(w["n"], [p[0] for p in w["ab"]], [p[1] for p in w["ab"]], points=w["points"], eps=eps,
                          precision=prec, setup_device=dev_setup)
            torch.cuda.synchronize()
            row["fac_gpu_setup_s" if dev_setup else "fac_host_s"] = time.perf_counter() - t0
            if not dev_setup:
                dt = torch.float32 if prec == "fp32" else torch.float64
                x = torch.tensor(w["alpha"], dtype=dt, device=dev)
                f = torch.empty_like(x)
                for _ in range(3):
                    T.forward(x, out=f)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(10):
                    T.forward(x, out=f)
                e1.record(stream)
                torch.cuda.synchronize()
                row["app_forward_ms"] = e0.elapsed_time(e1) / 10
                row["ranks"] = T.ranks
                del x, f
            T.close()
        out[f"{name} {prec}"] = row
    return out


def batch_mix_throughput(dev, stream, count=64):
    """The serving-style mix (1-D n log-uniform in [256, 16384] or 2-D n_x, n_y in [64, 1024],
    (a, b) ~ U(-0.5, 0.5), 1..16 right-hand sides), FP32: one batched forward + adjoint per
    step, eager and replayed from a CUDA graph, against the members launched one by one."""
    import torch

    from paper_1901_07275_gb300 import Batch, Transform
    from paper_1901_07275_gb300 import synthetic as syn

    t0 = time.perf_counter()
    mix = syn.batch_mix(count)
    Ts = [Transform(m["n"], [p[0] for p in m["ab"]], [p[1] for p in m["ab"]], eps=1e-7) for m in mix]
    setup_s = time.perf_counter() - t0
    # the same plans with their host setups side by side, and reloaded from saved bytes
    t0 = time.perf_counter()
    many = Transform.create_many([{"n": m["n"], "a": [p[0] for p in m["ab"]], "b": [p[1] for p in m["ab"]],
                                   "eps": 1e-7} for m in mix])
    many_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    many_gpu = Transform.create_many([{"n": m["n"], "a": [p[0] for p in m["ab"]], "b": [p[1] for p in m["ab"]],
                                       "eps": 1e-7, "setup_device": True} for m in mix])
    many_gpu_s = time.perf_counter() - t0
    for T in many_gpu:
        T.close()
    saved = [T.save() for T in Ts]
    t0 = time.perf_counter()
    loaded = [Transform.load(b) for b in saved]
    load_s = time.perf_counter() - t0
    same = all(a.save() == b for a, b in zip(many, saved))
    for T in many + loaded:
        T.close()
    xs = [torch.tensor(syn.normal(2000 + i, 0, (m["nrhs"],) + tuple(m["n"])), dtype=torch.float32, device=dev)
          for i, m in enumerate(mix)]
    fs = [torch.empty_like(x) for x in xs]
    gs = [torch.empty_like(x) for x in xs]
    batch = Batch(Ts, [m["nrhs"] for m in mix])
    coeffs = 2 * sum(x.numel() for x in xs)

    def timed(fn, reps=5):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    def batched():
        batch.forward(xs, fs)
        batch.adjoint(fs, gs)

    def one_by_one():
        for T, x, f, g in zip(Ts, xs, fs, gs):
            T.forward(x, out=f)
            T.adjoint(f, out=g)

    ms_batch = timed(batched)
    ms_single = timed(one_by_one)
    side = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(graph, stream=side):
        batch.forward(xs, fs, stream=side)
        batch.adjoint(fs, gs, stream=side)
    ms_graph = timed(graph.replay)
    out = {"members": count, "coeffs_per_step": coeffs, "plan_setup_s": setup_s,
           "plan_setup_many_s": many_s, "plan_setup_many_gpu_s": many_gpu_s, "plan_load_s": load_s, "saved_bytes": sum(len(b) for b in saved),
           "many_equals_one_by_one": same,
           "batched": {"coeffs_per_s": coeffs / (ms_batch * 1e-3), "ms_per_step": ms_batch},
           "graph_replay": {"coeffs_per_s": coeffs / (ms_graph * 1e-3), "ms_per_step": ms_graph},
           "one_by_one": {"coeffs_per_s": coeffs / (ms_single * 1e-3), "ms_per_step": ms_single}}
    batch.close()
    for T in Ts:
        T.close()
    return out


def batch_full_mix(dev, stream, count=512):
    """The whole serving mix: 512 members (a fair coin between 1-D n log-uniform in
    [256, 16384] and 2-D n_x, n_y log-uniform in [64, 1024]; (a, b) ~ U(-0.5, 0.5) per axis;
    1..16 right-hand sides).  FP32 at eps 1e-7 and double-word (split) at eps 1e-12: plans by
    create_many (host setups side by side), the rank split of every member's sweeps measured
    for its nrhs (jt_plan_tune), then one batched forward + adjoint per step, eager and replayed
    from a CUDA graph.  The coefficients of member i are the seeded host normals
    synthetic.normal(5000 + i, 0, .) -- the inputs on which tests/test_gpu_batch_mix.py checks
    every member against the oracle."""
    import torch

    from paper_1901_07275_gb300 import Batch, Transform
    from paper_1901_07275_gb300 import synthetic as syn

    mix = syn.batch_mix(count)
    out = {"members": count, "one_d_members": sum(len(m["n"]) == 1 for m in mix),
           "inputs": "seeded host generator, synthetic.normal(5000 + member, 0, (nrhs,) + n)"}
    t0 = time.perf_counter()
    host = [syn.normal(5000 + i, 0, (m["nrhs"],) + tuple(m["n"])) for i, m in enumerate(mix)]
    out["input_generation_s"] = time.perf_counter() - t0
    split_idx = [i for i, m in enumerate(mix) if max(m["n"]) <= SPLIT_MAX_N]
    for prec, eps, idx in (("fp32", 1e-7, list(range(count))), ("split", 1e-12, split_idx)):
        members = [mix[i] for i in idx]
        t0 = time.perf_counter()
        Ts = Transform.create_many([{"n": m["n"], "a": [p[0] for p in m["ab"]], "b": [p[1] for p in m["ab"]],
                                     "eps": eps, "precision": prec} for m in members])
        setup_s = time.perf_counter() - t0
        t0 = time.perf_counter()
        for T, m in zip(Ts, members):
            T.tune(m["nrhs"], stream=stream)
        torch.cuda.synchronize()
        tune_s = time.perf_counter() - t0
        # the tuner's choices: how many sweeps (member x axis x direction) took each rank split
        chosen = {}
        for T, m in zip(Ts, members):
            for ax in range(len(m["n"])):
                for d in (0, 1):
                    ks = T.schedule(ax, d, m["nrhs"])
                    chosen[str(ks)] = chosen.get(str(ks), 0) + 1
        dt = torch.float32 if prec == "fp32" else torch.float64
        xs = [torch.tensor(host[i], dtype=dt, device=dev) for i in idx]
        fs = [torch.empty_like(x) for x in xs]
        gs = [torch.empty_like(x) for x in xs]
        t0 = time.perf_counter()
        batch = Batch(Ts, [m["nrhs"] for m in members])
        batch_s = time.perf_counter() - t0
        coeffs = 2 * sum(x.numel() for x in xs)

        def batched():
            batch.forward(xs, fs)
            batch.adjoint(fs, gs)

        for _ in range(2):
            batched()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 5
        e0.record(stream)
        for _ in range(reps):
            batched()
        e1.record(stream)
        torch.cuda.synchronize()
        ms_batch = e0.elapsed_time(e1) / reps
        side = torch.cuda.Stream()
        graph = torch.cuda.CUDAGraph()
        torch.cuda.synchronize()
        with torch.cuda.graph(graph, stream=side):
            batch.forward(xs, fs, stream=side)
            batch.adjoint(fs, gs, stream=side)
        graph.replay()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            graph.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        ms_graph = e0.elapsed_time(e1) / reps
        out[prec] = {"members": len(members), "coeffs_per_step": coeffs, "eps": eps,
                     "plan_setup_many_s": setup_s, "tune_s": tune_s, "batch_create_s": batch_s,
                     "tuned_rank_split_sweeps": chosen,
                     "batched": {"coeffs_per_s": coeffs / (ms_batch * 1e-3), "ms_per_step": ms_batch,
                                 "transforms_per_s": 2 * sum(m["nrhs"] for m in members) / (ms_batch * 1e-3)},
                     "graph_replay": {"coeffs_per_s": coeffs / (ms_graph * 1e-3), "ms_per_step": ms_graph,
                                      "transforms_per_s": 2 * sum(m["nrhs"] for m in members) / (ms_graph * 1e-3)}}
        del graph
        batch.close()
        for T in Ts:
            T.close()
        del xs, fs, gs
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--nrhs", type=int, default=256)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="time the FP32 step only (profiling runs)")
    args = ap.parse_args()
    if args.warmup < 3 and not args.no_extras:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch

    import __graft_entry__

    world, rank, local = dist_init()
    torch.cuda.set_device(local)
    __graft_entry__.build()
    from paper_1901_07275_gb300 import Transform
    from paper_1901_07275_gb300 import synthetic as syn

    dev = torch.device("cuda", local)
    peaks, peak_src = load_peaks()
    nrhs = args.nrhs
    T = Transform(N, [p[0] for p in AB], [p[1] for p in AB], eps=1e-7, precision="fp32")
    ranks, Ls = T.ranks, T.fft_lens
    alpha = syn.normal(1002 + rank, 0, (nrhs,) + N)
    x = torch.tensor(alpha, dtype=torch.float32, device=dev)
    f = torch.empty_like(x)
    y = torch.empty_like(x)
    stream = torch.cuda.current_stream()

    def step():
        T.forward(x, out=f)
        T.inverse(f, out=y)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    gpu_index = vis.split(",")[local] if vis else str(local)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(gpu_index) as clk:
        barrier(world)
        torch.cuda.synchronize()
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for i in range(args.steps):
            ev[i][0].record(stream)
            T.forward(x, out=f)
            ev[i][1].record(stream)
            T.inverse(f, out=y)
            ev[i][2].record(stream)
        t_end.record(stream)
        torch.cuda.synchronize()
        barrier(world)
    total_ms = max_over_ranks(world, t_start.elapsed_time(t_end))
    kern_ms = sum(a.elapsed_time(b) + b.elapsed_time(c) for a, b, c in ev)
    clocks = clk.summary()

    coeffs_per_step = 2 * nrhs * N[0] * N[1]
    value = aggregate(world, coeffs_per_step, args.steps, total_ms)

    # roofline of the fused axis kernel: 4 launches per step (2 axes x forward/inverse)
    flops_step = 2 * sum(nrhs * (N[0] * N[1] // N[a]) * axis_flops(N[a], Ls[a], ranks[a]) for a in range(2))
    bytes_step = 2 * sum(2 * 4 * nrhs * N[0] * N[1] + axis_table_bytes(N[a], Ls[a], ranks[a], 27, 4) for a in range(2))
    achieved_tflops = flops_step * args.steps / (kern_ms * 1e-3) / 1e12
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    nominal_peak = sm_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    probe = fp32_peak(dev, stream, gpu_index)
    alu_peak = probe["peak_tflops"]
    hbm_gbs = bytes_step * args.steps / (kern_ms * 1e-3) / 1e9
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    launches = 4 * args.steps

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "2d-512x512 uniform, (a,b)=(0.3,-0.4)x(-0.5,0.2), alpha~N(0,1)",
                   "nrhs": nrhs, "step": "forward + inverse, fused FP32 axis kernels, eps=1e-7",
                   "ranks": ranks, "fft_len": Ls,
                   "l2": f"inputs {4 * nrhs * N[0] * N[1] / 2**20:.0f} MiB > L2 129 MB, no flush",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "roofline": {"bound": "alu", "achieved": achieved_tflops, "peak": alu_peak, "unit": "TFLOP/s",
                     "frac": achieved_tflops / alu_peak, "traffic": captured_traffic(),
                     "traffic_unit": "bytes per launch (ncu dram read + write)",
                     "algorithmic_bytes_per_launch": bytes_step / 4,
                     "peak_note": "measured: best FP32 FMA-chain rate of jt_probe_fp32_fma (scalar and "
                                  "f32x2 forms) in this run",
                     "peak_probe": probe,
                     "nominal_peak": {"tflops": nominal_peak,
                                      "rule": f"{sm_count} SMs x {FP32_LANES_PER_SM} lanes x 2 x {sm_max:.0f} MHz "
                                              f"(sm_max from MEASURED_PEAKS: {peak_src})"},
                     "hbm": {"achieved_gbs": hbm_gbs, "peak_gbs": hbm_peak, "frac": hbm_gbs / hbm_peak,
                             "peak_source": peak_src}},
        "clocks": clocks, "gpu_launches": launches,
        "transforms_per_s": 2 * nrhs * world * args.steps / (total_ms * 1e-3),
    }

    if rank == 0 and not args.no_extras:
        import oracle

        # accuracy on right-hand side 0 against the oracle (forward, and the inverse of it)
        mats = [oracle.uniform_matrix(a, b, m) for (a, b), m in zip(AB, N)]
        ref = oracle.forward(alpha[:1], mats)
        err_f = float(np.linalg.norm(f[:1].double().cpu().numpy() - ref) / np.linalg.norm(ref))
        err_i = float(np.linalg.norm(y[:1].double().cpu().numpy() - alpha[:1]) / np.linalg.norm(alpha[:1]))
        line["rel_err"] = {"fp32_forward": err_f, "fp32_inverse_of_forward": err_i}

        # end to end through the public API with host buffers (pinned), copies inside the region:
        # Transform.transform_host (jt_transform_host) streams the right-hand sides through a
        # 64 MiB device work area, copies overlapped with the transforms; a step is the forward
        # (host alpha -> host f) and the inverse (host f -> host alpha)
        xh = torch.tensor(alpha, dtype=torch.float32).pin_memory()
        fh = torch.empty_like(xh).pin_memory()
        yh = torch.empty_like(xh).pin_memory()
        ws = torch.empty(64 << 20, dtype=torch.uint8, device=dev)
        ke = min(args.steps, 5)

        def e2e_step():
            T.transform_host(xh, out=fh, direction="forward", workspace=ws, stream=stream)
            T.transform_host(fh, out=yh, direction="inverse", workspace=ws, stream=stream)

        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(ke):
            e2e_step()
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = e0.elapsed_time(e1) / ke
        e2e_err = float(np.linalg.norm(yh[:1].double().numpy() - alpha[:1]) / np.linalg.norm(alpha[:1]))
        # the same step with whole-array copies around device transforms, not overlapped
        e0.record(stream)
        for _ in range(ke):
            x.copy_(xh, non_blocking=True)
            step()
            yh.copy_(y, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        serial_ms = e0.elapsed_time(e1) / ke
        line["e2e"] = {"value": coeffs_per_step / (e2e_ms * 1e-3), "unit": UNIT,
                       "h2d_bytes_per_step": 2 * xh.numel() * 4, "d2h_bytes_per_step": 2 * xh.numel() * 4,
                       "ms_per_step": e2e_ms, "api": "Transform.transform_host (jt_transform_host), 64 MiB work area",
                       "rel_err_inverse_of_forward": e2e_err,
                       "unoverlapped_copies": {"value": coeffs_per_step / (serial_ms * 1e-3), "ms_per_step": serial_ms,
                                               "h2d_bytes_per_step": xh.numel() * 4,
                                               "d2h_bytes_per_step": yh.numel() * 4}}
        del xh, fh, yh, ws

        # double-word (split) kernels on a batch of 64 (134 MB of FP64 input)
        n2 = min(nrhs, 64)
        T2 = Transform(N, [p[0] for p in AB], [p[1] for p in AB], eps=1e-12, precision="split")
        x2 = torch.tensor(alpha[:n2], dtype=torch.float64, device=dev)
        f2 = torch.empty_like(x2)
        y2 = torch.empty_like(x2)
        for _ in range(3):
            T2.forward(x2, out=f2)
            T2.inverse(f2, out=y2)
        torch.cuda.synchronize()
        e0.record(stream)
        ks = 5
        for _ in range(ks):
            T2.forward(x2, out=f2)
            T2.inverse(f2, out=y2)
        e1.record(stream)
        torch.cuda.synchronize()
        split_ms = e0.elapsed_time(e1) / ks
        ref2 = ref
        err2 = float(np.linalg.norm(f2[:1].cpu().numpy() - ref2) / np.linalg.norm(ref2))
        err2i = float(np.linalg.norm(y2[:1].cpu().numpy() - alpha[:1]) / np.linalg.norm(alpha[:1]))
        split_v = 2 * n2 * N[0] * N[1] / (split_ms * 1e-3)
        # roofline of the double-word sweeps: the algorithmic count in FP32 instructions of the
        # double-word algorithms (DW_FLOPS_PER_FLOP a real operation), over the measured FP32 peak
        flops_split = 2 * sum(n2 * (N[0] * N[1] // N[a]) * axis_flops(N[a], T2.fft_lens[a], T2.ranks[a]) for a in range(2))
        dw_tflops = flops_split * DW_FLOPS_PER_FLOP / (split_ms * 1e-3) / 1e12
        line["split"] = {"roofline": {"bound": "alu", "achieved": dw_tflops, "peak": alu_peak, "unit": "TFLOP/s",
                                      "frac": dw_tflops / alu_peak,
                                      "algorithmic_flops_per_step": flops_split,
                                      "dw_flops_per_flop": DW_FLOPS_PER_FLOP,
                                      "note": "algorithmic flops x the FP32 operations of the double-word "
                                              "algorithms (sum 11, product 12 counting an FMA as 2), timed over "
                                              "the whole step (4 sweeps)"},
                         "value": split_v, "unit": UNIT, "nrhs": n2, "ms_per_step": split_ms, "ranks": T2.ranks,
                         "rel_err_forward": err2, "rel_err_inverse_of_forward": err2i, "dtype": "f32x2 (f64 io)"}
        del x2, f2, y2
        T2.close()

        # plain FP64 r^2-FFT path (cuFFT Z2Z): the same 64 right-hand sides as the split kernels,
        # in chunks with one batched 2-D cuFFT call per (pattern, rank-term pair)
        Tp = Transform(N, [p[0] for p in AB], [p[1] for p in AB], eps=1e-12, precision="fp64_plain")
        xp = torch.tensor(alpha[:n2], dtype=torch.float64, device=dev)
        fp_ = torch.empty_like(xp)
        yp = torch.empty_like(xp)
        Tp.forward(xp, out=fp_)
        Tp.inverse(fp_, out=yp)
        torch.cuda.synchronize()
        e0.record(stream)
        kp = 2
        for _ in range(kp):
            Tp.forward(xp, out=fp_)
            Tp.inverse(fp_, out=yp)
        e1.record(stream)
        torch.cuda.synchronize()
        plain_ms = e0.elapsed_time(e1) / kp
        errp = float(np.linalg.norm(fp_[:1].cpu().numpy() - ref) / np.linalg.norm(ref))
        plain_v = 2 * n2 * N[0] * N[1] / (plain_ms * 1e-3)
        line["plain_fp64"] = {"value": plain_v, "unit": UNIT, "nrhs": n2, "ms_per_step": plain_ms,
                              "ranks": Tp.ranks, "rel_err_forward": errp,
                              "speedup_fp32_over_plain": value / world / plain_v,
                              "speedup_split_over_plain": split_v / plain_v}
        Tp.close()

        # second-kind transform (Q~) on the same workload: forward + adjoint, FP32
        Tq = Transform(N, [p[0] for p in AB], [p[1] for p in AB], eps=1e-7, kind="second")
        for _ in range(2):
            Tq.forward(x, out=f)
            Tq.adjoint(f, out=y)
        torch.cuda.synchronize()
        e0.record(stream)
        kq = 5
        for _ in range(kq):
            Tq.forward(x, out=f)
            Tq.adjoint(f, out=y)
        e1.record(stream)
        torch.cuda.synchronize()
        q_ms = e0.elapsed_time(e1) / kq
        mq = [oracle.uniform_matrix_q(a, b, m) for (a, b), m in zip(AB, N)]
        refq = oracle.forward(alpha[:1], mq)
        Tq.forward(x, out=f)
        errq = float(np.linalg.norm(f[:1].double().cpu().numpy() - refq) / np.linalg.norm(refq))
        line["second_kind"] = {"value": coeffs_per_step / (q_ms * 1e-3), "unit": UNIT, "nrhs": nrhs,
                               "ms_per_step": q_ms, "step": "forward + adjoint", "ranks": Tq.ranks,
                               "rel_err_forward": errq}
        Tq.close()

        line["other_configs"] = other_configs(dev, stream)
        line["paper_configs"] = paper_configs(dev, stream)
        line["batch"] = batch_mix_throughput(dev, stream)
        line["batch_512"] = batch_full_mix(dev, stream)
        line["setup"] = setup_timings()
        line["fac_app"] = fac_and_app(dev, stream)
        line["sweeps"] = sweep_times(dev, stream)

        if world == 1:
            line["cpu_baseline"] = oracle_throughput(nrhs)

    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
