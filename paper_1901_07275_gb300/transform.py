"""PyTorch front end: device memory and streams come from torch, every step of the
transform runs in libjt's kernels through the C ABI."""

from __future__ import annotations

import math

from . import binding as B

_DEFAULT_EPS = {"fp32": 1e-7, "split": 1e-12, "fp64_plain": 1e-12}
_DTYPES = {"fp32": "float32", "split": "float64", "fp64_plain": "float64"}


class Transform:
    """A d-dimensional Jacobi transform plan (d = len(n)).

    ``points[i]`` None selects the Gauss--Jacobi nodes of axis i (uniform, orthogonal
    ``W J``); otherwise it holds the angles in (0, pi) of a nonuniform axis (``J``).
    Inputs are torch tensors on the plan's CUDA device, contiguous, of shape
    ``(..., n_0, .., n_{d-1})`` -- leading dimensions are independent right-hand sides --
    and dtype float32 (``precision="fp32"``) or float64 (``"split"``, ``"fp64_plain"``).
    ``kind="second"`` expands in the second-kind functions Q~ (forward and adjoint only).
    """

    def __init__(self, n, a, b, points=None, eps=None, precision="fp32", nu0=27, rank_cap=0,
                 oversample_q=3, seed=None, autotune=False, kind="first", setup_device=False, stream=None):
        import torch

        self.n = tuple(int(v) for v in n)
        self.d = len(self.n)
        self.a = tuple(float(v) for v in a)
        self.b = tuple(float(v) for v in b)
        self.precision = precision
        self.eps = _DEFAULT_EPS[precision] if eps is None else float(eps)
        self.dtype = getattr(torch, _DTYPES[precision])
        self.uniform = points is None or all(p is None for p in points)
        self.kind = kind
        opt = B.options(precision, nu0=nu0, rank_cap=rank_cap, oversample_q=oversample_q, seed=seed,
                        autotune=1 if autotune else 0, kind=kind, setup_device=1 if setup_device else 0)
        s = self._stream(stream)
        self._plan = B.jt_plan_create(self.n, self.a, self.b, points, self.eps, opt, s)
        self.info = [B.jt_plan_info(self._plan, i, self.n[i]) for i in range(self.d)]

    @classmethod
    def _from_handle(cls, plan):
        """Wrap an existing plan handle (from jt_plan_load or jt_plan_create_many)."""
        import torch

        self = cls.__new__(cls)
        sh = B.jt_plan_shape(plan)
        self._plan = plan
        self.n = sh["n"]
        self.d = sh["d"]
        self.precision = {B.JT_FP32: "fp32", B.JT_SPLIT: "split", B.JT_FP64_PLAIN: "fp64_plain"}[sh["prec"]]
        self.kind = "second" if sh["kind"] == B.JT_SECOND_KIND else "first"
        self.dtype = getattr(torch, _DTYPES[self.precision])
        self.uniform = sh["all_uniform"]
        self.a = self.b = None
        self.eps = None
        self.info = [B.jt_plan_info(plan, i, self.n[i]) for i in range(self.d)]
        return self

    def save(self) -> bytes:
        """The plan's setup as bytes (:meth:`load` recreates it without setup work)."""
        return B.jt_plan_save(self._plan)

    @classmethod
    def load(cls, data: bytes, stream=None):
        """A plan from :meth:`save` bytes: only the device upload runs."""
        return cls._from_handle(B.jt_plan_load(data, cls._stream(stream)))

    @classmethod
    def create_many(cls, specs, stream=None):
        """Several plans whose host setups run side by side.  ``specs``: dicts with ``n, a, b``
        and optionally ``points, eps, precision, kind, nu0, rank_cap, oversample_q, seed``."""
        raw = []
        for sp in specs:
            prec = sp.get("precision", "fp32")
            opt = B.options(prec, nu0=sp.get("nu0", 27), rank_cap=sp.get("rank_cap", 0),
                            oversample_q=sp.get("oversample_q", 3), seed=sp.get("seed"),
                            kind=sp.get("kind", "first"), setup_device=1 if sp.get("setup_device") else 0)
            raw.append({"n": sp["n"], "a": sp["a"], "b": sp["b"], "points": sp.get("points"),
                        "eps": sp.get("eps", _DEFAULT_EPS[prec]), "opt": opt})
        return [cls._from_handle(h) for h in B.jt_plan_create_many(raw, cls._stream(stream))]

    @staticmethod
    def _stream(stream):
        import torch

        if stream is None:
            stream = torch.cuda.current_stream()
        return int(stream.cuda_stream)

    @property
    def ranks(self):
        return [i["rank"] for i in self.info]

    @property
    def fft_lens(self):
        return [i["fft_len"] for i in self.info]

    def set_ksplit(self, ksplit, axis=-1, direction=-1):
        """Fix the rank split (CTAs sharing a tile: 1, 2, 4, 8; 0 = occupancy rule)."""
        B.jt_plan_set_ksplit(self._plan, axis, direction, ksplit)

    def tune(self, nrhs, stream=None):
        """Measure and keep the fastest rank split of every sweep for ``nrhs`` right-hand sides."""
        B.jt_plan_tune(self._plan, nrhs, self._stream(stream))

    def schedule(self, axis, direction, nrhs):
        """Rank split of the sweep of ``axis`` in ``direction`` (0 forward, 1 adjoint)."""
        return B.jt_plan_schedule(self._plan, axis, direction, nrhs)

    def nodes(self, axis):
        return self.info[axis]["t"]

    def weights(self, axis):
        return self.info[axis]["w"]

    def _check(self, x):
        import torch

        if not isinstance(x, torch.Tensor) or not x.is_cuda:
            raise TypeError("expected a CUDA tensor")
        if x.dtype != self.dtype:
            raise TypeError(f"expected dtype {self.dtype}, got {x.dtype}")
        if tuple(x.shape[x.dim() - self.d:]) != self.n:
            raise ValueError(f"trailing shape {tuple(x.shape)} does not match {self.n}")
        if not x.is_contiguous():
            raise ValueError("expected a contiguous tensor")
        nrhs = math.prod(x.shape[: x.dim() - self.d]) if x.dim() > self.d else 1
        return nrhs

    def _run(self, fn, x, out, stream):
        import torch

        nrhs = self._check(x)
        if out is None:
            out = torch.empty_like(x)
        else:
            self._check(out)
        if nrhs > 0:
            fn(self._plan, x.data_ptr(), out.data_ptr(), nrhs, self._stream(stream))
        return out

    def forward(self, alpha, out=None, stream=None):
        """f = (A_0 (x) .. (x) A_{d-1}) alpha."""
        return self._run(B.jt_forward, alpha, out, stream)

    def adjoint(self, g, out=None, stream=None):
        """alpha = (A_0 (x) .. (x) A_{d-1})^T g."""
        return self._run(B.jt_adjoint, g, out, stream)

    def inverse(self, g, out=None, stream=None):
        """Inverse of :meth:`forward` (uniform axes only)."""
        return self._run(B.jt_inverse, g, out, stream)

    def transform_host(self, x, out=None, direction="forward", workspace=None, stream=None):
        """Transform a HOST tensor (pinned for overlap) through a device work area in chunks of
        right-hand sides, copies and transforms overlapped (jt_transform_host).  ``workspace``
        is a CUDA uint8 tensor; by default one of up to 256 MiB is allocated."""
        import torch

        if x.is_cuda or x.dtype != self.dtype or not x.is_contiguous():
            raise TypeError("expected a contiguous host tensor of the plan's dtype")
        if tuple(x.shape[x.dim() - self.d:]) != self.n:
            raise ValueError(f"trailing shape {tuple(x.shape)} does not match {self.n}")
        nrhs = math.prod(x.shape[: x.dim() - self.d]) if x.dim() > self.d else 1
        if out is None:
            out = torch.empty_like(x, pin_memory=x.is_pinned())
        per = x.element_size() * math.prod(self.n)
        if workspace is None:
            workspace = torch.empty(max(per, min(nrhs * per, 256 << 20)), dtype=torch.uint8, device="cuda")
        code = {"forward": 0, "adjoint": 1, "inverse": 2}[direction]
        B.jt_transform_host(self._plan, code, x.data_ptr(), out.data_ptr(), nrhs, workspace.data_ptr(),
                            workspace.numel(), self._stream(stream))
        return out

    __call__ = forward

    def close(self):
        if getattr(self, "_plan", None):
            B.jt_destroy(self._plan)
            self._plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Several transforms of one precision executed together (``jt_batch_*``): each member
    has its own :class:`Transform` and number of right-hand sides; ``forward`` and
    ``adjoint`` take lists of tensors, one per member, shaped ``(nrhs_i, *n_i)``."""

    def __init__(self, transforms, nrhs, stream=None):
        self.transforms = list(transforms)
        self.nrhs = [int(v) for v in nrhs]
        if len(self.transforms) != len(self.nrhs) or not self.transforms:
            raise ValueError("one nrhs per transform")
        self._batch = B.jt_batch_create([t._plan for t in self.transforms], self.nrhs,
                                        Transform._stream(stream))

    def _run(self, fn, xs, outs, stream):
        import torch

        if len(xs) != len(self.transforms):
            raise ValueError("one input per member")
        if outs is None:
            outs = [torch.empty_like(x) for x in xs]
        for T, r, x, o in zip(self.transforms, self.nrhs, xs, outs):
            if T._check(x) != r or T._check(o) != r:
                raise ValueError("input or output does not match the member's nrhs")
        fn(self._batch, [x.data_ptr() for x in xs], [o.data_ptr() for o in outs], Transform._stream(stream))
        return outs

    def forward(self, xs, outs=None, stream=None):
        return self._run(B.jt_batch_forward, xs, outs, stream)

    def adjoint(self, gs, outs=None, stream=None):
        return self._run(B.jt_batch_adjoint, gs, outs, stream)

    def close(self):
        if getattr(self, "_batch", None):
            B.jt_batch_destroy(self._batch)
            self._batch = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _make_fn():
    import torch

    class JacobiFn(torch.autograd.Function):
        """f = T(alpha) with the hand-written adjoint kernel as its backward pass."""

        @staticmethod
        def forward(ctx, alpha, transform):
            ctx.transform = transform
            return transform.forward(alpha.contiguous())

        @staticmethod
        def backward(ctx, grad_f):
            return ctx.transform.adjoint(grad_f.contiguous()), None

    return JacobiFn


_FN = None


def jacobi_fn(alpha, transform):
    """Differentiable forward transform (backward = adjoint kernel)."""
    global _FN
    if _FN is None:
        _FN = _make_fn()
    return _FN.apply(alpha, transform)
