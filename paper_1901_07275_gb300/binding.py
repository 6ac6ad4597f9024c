"""ctypes binding of libjt: the C ABI of ``include/jt.h`` with the same names.

Argument marshalling only -- every step of a transform runs in the library's CUDA
kernels.  The shared library is built in-tree by ``paper_1901_07275_gb300.build``;
if it is missing, every call raises instead of falling back to anything else.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libjt.so")

JT_OK, JT_EINVAL, JT_ENOMEM, JT_ENOTSUP, JT_ECUDA, JT_ETIMEOUT, JT_ENOCONV = range(7)
JT_FP32, JT_SPLIT, JT_FP64_PLAIN = 0, 1, 2
JT_FIRST_KIND, JT_SECOND_KIND = 0, 1
KINDS = {"first": JT_FIRST_KIND, "second": JT_SECOND_KIND}
PRECISIONS = {"fp32": JT_FP32, "split": JT_SPLIT, "fp64_plain": JT_FP64_PLAIN}

# every symbol declared in include/jt.h
EXPORTS = (
    "jt_options_default",
    "jt_plan_create",
    "jt_forward",
    "jt_adjoint",
    "jt_inverse",
    "jt_forward_plain_noalloc",
    "jt_plan_info",
    "jt_destroy",
    "jt_plan_check",
    "jt_plan_inject_wait_timeout",
    "jt_plan_shape",
    "jt_transform_host",
    "jt_plan_create_many",
    "jt_plan_save",
    "jt_plan_load",
    "jt_plan_set_ksplit",
    "jt_plan_tune",
    "jt_plan_schedule",
    "jt_batch_create",
    "jt_batch_forward",
    "jt_batch_adjoint",
    "jt_batch_destroy",
    "jt_status_string",
    "jt_probe_fp32_fma",
    "jt_axis_tables_create",
    "jt_axis_tables_info",
    "jt_axis_tables_copy",
    "jt_axis_tables_b_rows",
    "jt_axis_tables_destroy",
)


class JTError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_string(status)}")


class PlanDesc(ctypes.Structure):
    _fields_ = [
        ("d", ctypes.c_int32),
        ("n", ctypes.c_int64 * 3),
        ("a", ctypes.c_double * 3),
        ("b", ctypes.c_double * 3),
        ("points", ctypes.POINTER(ctypes.c_double) * 3),
        ("eps", ctypes.c_double),
        ("opt", ctypes.c_void_p),
    ]


class Options(ctypes.Structure):
    _fields_ = [
        ("prec", ctypes.c_int32),
        ("nu0", ctypes.c_int32),
        ("rank_cap", ctypes.c_int32),
        ("oversample_q", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
        ("fft_len_policy", ctypes.c_int32),
        ("autotune", ctypes.c_int32),
        ("kind", ctypes.c_int32),
        ("setup_device", ctypes.c_int32),
    ]


_lib = None


def lib() -> ctypes.CDLL:
    """Load libjt (once).  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libjt is not built ({LIB_PATH} missing): run paper_1901_07275_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, i64, dbl, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
    L.jt_options_default.argtypes = [ctypes.POINTER(Options)]
    L.jt_options_default.restype = None
    L.jt_plan_create.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(i64), ctypes.POINTER(dbl),
                                 ctypes.POINTER(dbl), ctypes.POINTER(ctypes.POINTER(dbl)), dbl,
                                 ctypes.POINTER(Options), vp]
    L.jt_plan_create.restype = i32
    for name in ("jt_forward", "jt_adjoint", "jt_inverse", "jt_forward_plain_noalloc"):
        f = getattr(L, name)
        f.argtypes = [vp, vp, vp, i64, vp]
        f.restype = i32
    L.jt_plan_info.argtypes = [vp, i32, ctypes.POINTER(i32), ctypes.POINTER(i64), vp, vp]
    L.jt_plan_info.restype = i32
    L.jt_destroy.argtypes = [vp]
    L.jt_destroy.restype = None
    L.jt_plan_check.argtypes = [vp, vp]
    L.jt_plan_check.restype = i32
    L.jt_plan_inject_wait_timeout.argtypes = [vp, i32]
    L.jt_plan_inject_wait_timeout.restype = i32
    L.jt_plan_shape.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i64), ctypes.POINTER(i32),
                                ctypes.POINTER(i32), ctypes.POINTER(i32)]
    L.jt_plan_shape.restype = i32
    L.jt_transform_host.argtypes = [vp, i32, vp, vp, i64, vp, ctypes.c_size_t, vp]
    L.jt_transform_host.restype = i32
    L.jt_plan_create_many.argtypes = [i32, ctypes.POINTER(vp), ctypes.POINTER(PlanDesc), vp]
    L.jt_plan_create_many.restype = i32
    L.jt_plan_save.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_size_t)]
    L.jt_plan_save.restype = i32
    L.jt_plan_load.argtypes = [ctypes.POINTER(vp), vp, ctypes.c_size_t, vp]
    L.jt_plan_load.restype = i32
    L.jt_plan_set_ksplit.argtypes = [vp, i32, i32, i32]
    L.jt_plan_set_ksplit.restype = i32
    L.jt_plan_tune.argtypes = [vp, i64, vp]
    L.jt_plan_tune.restype = i32
    L.jt_plan_schedule.argtypes = [vp, i32, i32, i64, ctypes.POINTER(i32)]
    L.jt_plan_schedule.restype = i32
    L.jt_batch_create.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(vp), ctypes.POINTER(i64), vp]
    L.jt_batch_create.restype = i32
    for name in ("jt_batch_forward", "jt_batch_adjoint"):
        f = getattr(L, name)
        f.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), vp]
        f.restype = i32
    L.jt_batch_destroy.argtypes = [vp]
    L.jt_batch_destroy.restype = None
    L.jt_status_string.argtypes = [i32]
    L.jt_status_string.restype = ctypes.c_char_p
    L.jt_probe_fp32_fma.argtypes = [i32, i64, vp, i64, ctypes.POINTER(dbl), vp]
    L.jt_probe_fp32_fma.restype = i32
    L.jt_axis_tables_create.argtypes = [ctypes.POINTER(vp), i64, dbl, dbl, vp, dbl, ctypes.POINTER(Options)]
    L.jt_axis_tables_create.restype = i32
    L.jt_axis_tables_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i64), ctypes.POINTER(i32),
                                      ctypes.POINTER(dbl)]
    L.jt_axis_tables_info.restype = i32
    L.jt_axis_tables_copy.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    L.jt_axis_tables_copy.restype = i32
    L.jt_axis_tables_b_rows.argtypes = [vp, vp, i64, vp]
    L.jt_axis_tables_b_rows.restype = i32
    L.jt_axis_tables_destroy.argtypes = [vp]
    L.jt_axis_tables_destroy.restype = None
    _lib = L
    return L


def jt_probe_fp32_fma(paired: bool, iters: int, sink_ptr: int, sink_len: int, stream: int = 0) -> float:
    """Launch the FP32 FMA-rate probe on `stream`; returns the launch's flops."""
    flops = ctypes.c_double(0.0)
    _check(lib().jt_probe_fp32_fma(1 if paired else 0, int(iters), ctypes.c_void_p(sink_ptr), int(sink_len),
                                   ctypes.byref(flops), ctypes.c_void_p(stream)), "jt_probe_fp32_fma")
    return flops.value


def status_string(status: int) -> str:
    return lib().jt_status_string(int(status)).decode()


def _check(status: int, what: str):
    if status != JT_OK:
        raise JTError(status, what)


def options(prec="fp32", nu0=27, rank_cap=0, oversample_q=3, seed=None, autotune=0, kind="first",
            setup_device=0) -> Options:
    o = Options()
    lib().jt_options_default(ctypes.byref(o))
    o.prec = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
    o.nu0 = nu0
    o.rank_cap = rank_cap
    o.oversample_q = oversample_q
    o.autotune = int(autotune)
    o.kind = KINDS[kind] if isinstance(kind, str) else int(kind)
    o.setup_device = int(setup_device)
    if seed is not None:
        o.seed = seed
    return o


def _ptr(a):
    return None if a is None else ctypes.c_void_p(a)


# ----------------------------------------------------------------- plans
def jt_plan_create(n, a, b, points=None, eps=1e-7, opt: Options | None = None, stream: int = 0) -> int:
    """Create a plan; returns the opaque handle (int).  ``points[i]`` is None (Gauss--Jacobi
    nodes) or a sequence of angles in (0, pi)."""
    d = len(n)
    n_arr = (ctypes.c_int64 * d)(*[int(v) for v in n])
    a_arr = (ctypes.c_double * d)(*[float(v) for v in a])
    b_arr = (ctypes.c_double * d)(*[float(v) for v in b])
    keep = []
    pts = None
    if points is not None and any(p is not None for p in points):
        pts = (ctypes.POINTER(ctypes.c_double) * d)()
        for i, p in enumerate(points):
            if p is None:
                pts[i] = ctypes.POINTER(ctypes.c_double)()
            else:
                arr = np.ascontiguousarray(p, dtype=np.float64)
                keep.append(arr)
                pts[i] = arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    h = ctypes.c_void_p()
    st = lib().jt_plan_create(ctypes.byref(h), d, n_arr, a_arr, b_arr, pts, float(eps),
                              ctypes.byref(opt) if opt is not None else None, _ptr(stream))
    _check(st, "jt_plan_create")
    return h.value


def jt_forward(plan: int, alpha_ptr: int, f_ptr: int, nrhs: int, stream: int = 0) -> None:
    _check(lib().jt_forward(_ptr(plan), _ptr(alpha_ptr), _ptr(f_ptr), int(nrhs), _ptr(stream)), "jt_forward")


def jt_adjoint(plan: int, g_ptr: int, alpha_ptr: int, nrhs: int, stream: int = 0) -> None:
    _check(lib().jt_adjoint(_ptr(plan), _ptr(g_ptr), _ptr(alpha_ptr), int(nrhs), _ptr(stream)), "jt_adjoint")


def jt_inverse(plan: int, g_ptr: int, alpha_ptr: int, nrhs: int, stream: int = 0) -> None:
    _check(lib().jt_inverse(_ptr(plan), _ptr(g_ptr), _ptr(alpha_ptr), int(nrhs), _ptr(stream)), "jt_inverse")


def jt_forward_plain_noalloc(plan: int, alpha_ptr: int, f_ptr: int, nrhs: int, stream: int = 0) -> None:
    """Forward transform of a plain-FP64 plan with the library's static work area (no allocation)."""
    _check(lib().jt_forward_plain_noalloc(_ptr(plan), _ptr(alpha_ptr), _ptr(f_ptr), int(nrhs), _ptr(stream)),
           "jt_forward_plain_noalloc")


def jt_plan_info(plan: int, axis: int, n: int | None = None):
    r = ctypes.c_int()
    L = ctypes.c_int64()
    t = w = None
    if n is not None:
        t = np.zeros(n)
        w = np.zeros(n)
    st = lib().jt_plan_info(_ptr(plan), int(axis), ctypes.byref(r), ctypes.byref(L),
                            None if t is None else t.ctypes.data, None if w is None else w.ctypes.data)
    _check(st, "jt_plan_info")
    return {"rank": r.value, "fft_len": L.value, "t": t, "w": w}


def jt_destroy(plan: int) -> None:
    lib().jt_destroy(_ptr(plan))


def jt_plan_check(plan: int, stream: int = 0) -> int:
    """Synchronise `stream` and return the plan's status (JT_OK or JT_ETIMEOUT); raises on
    other errors."""
    st = lib().jt_plan_check(ctypes.c_void_p(plan), ctypes.c_void_p(stream))
    if st not in (JT_OK, JT_ETIMEOUT):
        _check(st, "jt_plan_check")
    return st


def jt_plan_inject_wait_timeout(plan: int, on: bool) -> None:
    _check(lib().jt_plan_inject_wait_timeout(ctypes.c_void_p(plan), 1 if on else 0), "jt_plan_inject_wait_timeout")


def jt_plan_shape(plan: int):
    """``{"d", "n", "prec", "kind", "all_uniform"}`` of a plan."""
    d, prec, kind, uni = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    n = (ctypes.c_int64 * 3)()
    _check(lib().jt_plan_shape(_ptr(plan), ctypes.byref(d), n, ctypes.byref(prec), ctypes.byref(kind),
                               ctypes.byref(uni)), "jt_plan_shape")
    return {"d": d.value, "n": tuple(n[: d.value]), "prec": prec.value, "kind": kind.value,
            "all_uniform": bool(uni.value)}


def jt_plan_create_many(specs, stream: int = 0):
    """Create several plans at once; ``specs`` holds dicts with ``n, a, b`` and optionally
    ``points, eps, opt`` (as for :func:`jt_plan_create`).  Returns the handles."""
    count = len(specs)
    descs = (PlanDesc * max(count, 1))()
    keep = []
    for i, sp in enumerate(specs):
        D = descs[i]
        d = len(sp["n"])
        D.d = d
        for k in range(d):
            D.n[k] = int(sp["n"][k])
            D.a[k] = float(sp["a"][k])
            D.b[k] = float(sp["b"][k])
        pts = sp.get("points")
        if pts is not None:
            for k, p in enumerate(pts):
                if p is not None:
                    arr = np.ascontiguousarray(p, dtype=np.float64)
                    keep.append(arr)
                    D.points[k] = arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        D.eps = float(sp.get("eps", 1e-7))
        opt = sp.get("opt")
        if opt is not None:
            keep.append(opt)
            D.opt = ctypes.cast(ctypes.byref(opt), ctypes.c_void_p)
    out = (ctypes.c_void_p * max(count, 1))()
    _check(lib().jt_plan_create_many(count, out, descs, _ptr(stream)), "jt_plan_create_many")
    return [out[i] for i in range(count)]


def jt_transform_host(plan: int, direction: int, in_ptr: int, out_ptr: int, nrhs: int, dev_ptr: int,
                      dev_bytes: int, stream: int = 0) -> None:
    """Transform host arrays through a device work area with overlapped copies (see jt.h)."""
    _check(lib().jt_transform_host(_ptr(plan), int(direction), _ptr(in_ptr), _ptr(out_ptr), int(nrhs), _ptr(dev_ptr),
                                   int(dev_bytes), _ptr(stream)), "jt_transform_host")


def jt_plan_save(plan: int) -> bytes:
    """The serialised setup of a plan (see jt_plan_save in jt.h)."""
    size = ctypes.c_size_t(0)
    _check(lib().jt_plan_save(_ptr(plan), None, ctypes.byref(size)), "jt_plan_save")
    buf = ctypes.create_string_buffer(size.value)
    _check(lib().jt_plan_save(_ptr(plan), buf, ctypes.byref(size)), "jt_plan_save")
    return buf.raw[: size.value]


def jt_plan_load(data: bytes, stream: int = 0) -> int:
    """Recreate a plan from :func:`jt_plan_save` bytes; returns the handle."""
    h = ctypes.c_void_p()
    raw = ctypes.create_string_buffer(bytes(data), len(data))
    _check(lib().jt_plan_load(ctypes.byref(h), raw, len(data), _ptr(stream)), "jt_plan_load")
    return h.value


def jt_plan_set_ksplit(plan: int, axis: int, direction: int, ksplit: int) -> None:
    """Fix the rank split (CTAs per tile) of axis ``axis`` (-1: all) for ``direction``
    (0 forward, 1 adjoint, -1 both); 0 restores the occupancy rule."""
    _check(lib().jt_plan_set_ksplit(_ptr(plan), int(axis), int(direction), int(ksplit)), "jt_plan_set_ksplit")


def jt_plan_tune(plan: int, nrhs: int, stream: int = 0) -> None:
    """Measure and keep the fastest rank split of every sweep for ``nrhs`` right-hand sides."""
    _check(lib().jt_plan_tune(_ptr(plan), int(nrhs), _ptr(stream)), "jt_plan_tune")


def jt_plan_schedule(plan: int, axis: int, direction: int, nrhs: int) -> int:
    """The rank split the sweep of ``axis`` gets in ``direction`` for ``nrhs`` right-hand sides."""
    k = ctypes.c_int()
    _check(lib().jt_plan_schedule(_ptr(plan), int(axis), int(direction), int(nrhs), ctypes.byref(k)),
           "jt_plan_schedule")
    return k.value


def jt_batch_create(plans, nrhs, stream: int = 0) -> int:
    count = len(plans)
    parr = (ctypes.c_void_p * count)(*plans)
    narr = (ctypes.c_int64 * count)(*[int(v) for v in nrhs])
    h = ctypes.c_void_p()
    _check(lib().jt_batch_create(ctypes.byref(h), count, parr, narr, _ptr(stream)), "jt_batch_create")
    return h.value


def _ptr_array(ptrs):
    return (ctypes.c_void_p * len(ptrs))(*[int(p) for p in ptrs])


def jt_batch_forward(batch: int, in_ptrs, out_ptrs, stream: int = 0) -> None:
    _check(lib().jt_batch_forward(_ptr(batch), _ptr_array(in_ptrs), _ptr_array(out_ptrs), _ptr(stream)),
           "jt_batch_forward")


def jt_batch_adjoint(batch: int, in_ptrs, out_ptrs, stream: int = 0) -> None:
    _check(lib().jt_batch_adjoint(_ptr(batch), _ptr_array(in_ptrs), _ptr_array(out_ptrs), _ptr(stream)),
           "jt_batch_adjoint")


def jt_batch_destroy(batch: int) -> None:
    lib().jt_batch_destroy(_ptr(batch))


# ------------------------------------------------------------ axis tables
class AxisTables:
    """Host-side tables of one axis (no GPU involved)."""

    def __init__(self, n, a, b, points=None, eps=1e-12, opt: Options | None = None):
        self.n = int(n)
        h = ctypes.c_void_p()
        pts = None
        if points is not None:
            self._pts = np.ascontiguousarray(points, dtype=np.float64)
            pts = self._pts.ctypes.data
        st = lib().jt_axis_tables_create(ctypes.byref(h), self.n, float(a), float(b), pts, float(eps),
                                         ctypes.byref(opt) if opt is not None else None)
        _check(st, "jt_axis_tables_create")
        self._h = h.value
        r, L, nu0, fe = ctypes.c_int(), ctypes.c_int64(), ctypes.c_int(), ctypes.c_double()
        _check(lib().jt_axis_tables_info(_ptr(self._h), ctypes.byref(r), ctypes.byref(L), ctypes.byref(nu0),
                                         ctypes.byref(fe)), "jt_axis_tables_info")
        self.rank, self.L, self.nu0, self.fact_err = r.value, L.value, nu0.value, fe.value
        n, N, rk = self.n, self.n - self.nu0, self.rank
        self.t = np.zeros(n)
        self.w = np.zeros(n)
        self.m = np.zeros(n, dtype=np.int32)
        u = np.zeros(2 * rk * n)
        v = np.zeros(2 * rk * N)
        self.vblk = np.zeros(n * self.nu0)
        _check(lib().jt_axis_tables_copy(_ptr(self._h), self.t.ctypes.data, self.w.ctypes.data, self.m.ctypes.data,
                                         u.ctypes.data, v.ctypes.data, self.vblk.ctypes.data), "jt_axis_tables_copy")
        self.U = (u[0::2] + 1j * u[1::2]).reshape(rk, n)
        self.V = (v[0::2] + 1j * v[1::2]).reshape(rk, N)
        self.vblk = self.vblk.reshape(n, self.nu0)

    def b_rows(self, rows) -> np.ndarray:
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        N = self.n - self.nu0
        out = np.zeros(2 * len(rows) * N)
        _check(lib().jt_axis_tables_b_rows(_ptr(self._h), rows.ctypes.data, len(rows), out.ctypes.data),
               "jt_axis_tables_b_rows")
        return (out[0::2] + 1j * out[1::2]).reshape(len(rows), N)

    def close(self):
        if getattr(self, "_h", None):
            lib().jt_axis_tables_destroy(_ptr(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
