"""GB300-native Fast Finite Shearlet Transform (arXiv:1202.1773).

The transform runs in libffst.so, a C-ABI CUDA library for sm_103a
(``include/ffst.h``).  This package is its binding:

* ``ffst_plan``, ``ffst_spectra``, ``ffst_forward``, ``ffst_inverse``,
  ``ffst_adjoint``, ... : the C entry points, argument marshalling only
  (device pointers as ints or tensors, stream handles);
* ``Plan``: the same calls on torch CUDA tensors (PyTorch provides device
  memory and the current stream, nothing else);
* ``FFSTFunction`` / ``shearlet_transform``: the forward transform as a
  differentiable layer whose backward pass is the hand-written adjoint.

There is no CPU fallback: without the built library every call raises.
"""

from __future__ import annotations

from . import _lib
from ._lib import (  # noqa: F401
    FFST_ERR_CUDA,
    FFST_ERR_INVALID_ARG,
    FFST_ERR_OUT_OF_MEMORY,
    FFST_ERR_TIMEOUT,
    FFST_ERR_UNSUPPORTED_SIZE,
    FFST_OK,
    FFST_STORE_BF16,
    FFST_STORE_F16,
    FFST_STORE_F32,
    FFSTError,
    ffst_adjoint,
    ffst_batch_destroy,
    ffst_batch_info,
    ffst_destroy,
    ffst_forward_batched,
    ffst_graph_capture_batched,
    ffst_graph_destroy,
    ffst_graph_launch,
    ffst_inverse_batched,
    ffst_plan_autotune,
    ffst_plan_batched,
    ffst_plan_check,
    ffst_plan_get_inverse_split,
    ffst_plan_get_schedule,
    ffst_plan_group_mb,
    ffst_plan_schedule_info,
    ffst_plan_set_inverse_split,
    ffst_plan_set_schedule,
    ffst_forward,
    ffst_forward_noalloc,
    ffst_forward_stats,
    ffst_forward_complex,
    ffst_inverse_complex,
    ffst_inverse,
    ffst_plan,
    ffst_plan_info,
    ffst_plane_index,
    ffst_spectra,
    ffst_timing_enable,
    ffst_timing_kinds,
    ffst_timing_read,
    ffst_timing_reset,
)

__all__ = ["Plan", "BatchPlan", "Graph", "FFSTFunction", "shearlet_transform", "FFSTError"] + [n for n, _, _ in _lib.SIGNATURES]


def _torch():
    import torch

    return torch


def _storage_of(dtype) -> int:
    torch = _torch()
    if dtype == torch.float32:
        return FFST_STORE_F32
    if dtype == torch.float16:
        return FFST_STORE_F16
    if dtype == torch.bfloat16:
        return FFST_STORE_BF16
    raise ValueError(f"unsupported coefficient dtype {dtype}")


class Plan:
    """A libffst plan for rows x cols float32 images on one CUDA device.

    Sizes 8..4096 per side.  Heights that are powers of two or 240, 320,
    384, 480, 640, 768 (widths: twice one of those) run native FFT lines;
    any other length up to 2048 (odd and prime included) runs Bluestein
    lines.  Square powers of two from 256 use the fused plane passes.

    Construction options (ffst_plan_ex): smooth=True builds the smooth
    shearlets of Sec. 3.4; vfun picks the auxiliary function v ("meyer",
    "quadratic", ("poly", k) or "cinf"); max_scale="min" uses the smaller
    grid extent X = 2^{2 j0 - 2}; spacing="per_axis" stretches both axes of
    a non-square image to [-X, X] instead of one grid step for both (Sec.
    3.5.1).  ``inverse_split`` sets the plane chunks of the inverse's sum
    (ffst_plan_set_inverse_split).
    """

    _VFUNS = {"meyer": _lib.FFST_V_MEYER, "quadratic": _lib.FFST_V_QUADRATIC, "cinf": _lib.FFST_V_CINF}

    def __init__(self, rows: int, cols: int, scales: int = 0, device=None, smooth: bool = False, vfun="meyer",
                 max_scale: str = "max", spacing: str = "common"):
        torch = _torch()
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.smooth = bool(smooth)
        if isinstance(vfun, tuple) and len(vfun) == 2 and vfun[0] == "poly":
            vcode, vorder = _lib.FFST_V_POLY, int(vfun[1])
        elif vfun in self._VFUNS:
            vcode, vorder = self._VFUNS[vfun], 0
        else:
            raise ValueError(f"unknown vfun {vfun!r}")
        if max_scale not in ("max", "min"):
            raise ValueError(f"max_scale must be 'max' or 'min', not {max_scale!r}")
        if spacing not in ("common", "per_axis"):
            raise ValueError(f"spacing must be 'common' or 'per_axis', not {spacing!r}")
        with torch.cuda.device(self.device):
            self.handle = ffst_plan(rows, cols, scales,
                                    _lib.FFST_VARIANT_SMOOTH if smooth else _lib.FFST_VARIANT_CLASSIC, vcode, vorder,
                                    _lib.FFST_MAXSCALE_MIN if max_scale == "min" else _lib.FFST_MAXSCALE_MAX,
                                    _lib.FFST_SPACING_PER_AXIS if spacing == "per_axis" else _lib.FFST_SPACING_COMMON)
        self.rows, self.cols, self.scales, self.num_planes = ffst_plan_info(self.handle)
        self.p0, self.p1 = 0, self.num_planes

    # -- bookkeeping ----------------------------------------------------------
    def close(self):
        if getattr(self, "handle", None):
            ffst_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def plane_index(self, i: int):
        """(kind, j, k) of plane i in the order of Sec. 3.5.2."""
        cone, j, k = ffst_plane_index(self.handle, i)
        return _lib.CONE_NAMES[cone], j, k

    def plane_table(self):
        return [self.plane_index(i) for i in range(self.num_planes)]

    @property
    def shape(self):
        """Shape of a coefficient stack: the active planes [p0, p1) (all by default)."""
        return (self.p1 - self.p0, self.rows, self.cols)

    @property
    def full_shape(self):
        return (self.num_planes, self.rows, self.cols)

    @property
    def kernels(self):
        """(fuse_fwd, fuse_inv, row_fwd, row_inv): the kernel configuration (ffst_plan_get_kernels)."""
        return _lib.ffst_plan_get_kernels(self.handle)

    def set_kernels(self, fuse_fwd: int = 1, fuse_inv: int = 1, row_fwd: int = 0, row_inv: int = 0):
        """Fused launches per direction and the row-FFT variant of separate row
        launches (ffst_plan_set_kernels)."""
        _lib.ffst_plan_set_kernels(self.handle, fuse_fwd, fuse_inv, row_fwd, row_inv)

    def set_planes(self, p0: int, p1: int):
        """Restrict the transforms to the planes [p0, p1) (ffst_plan_set_planes):
        stacks then hold those planes only, plane p0 first."""
        torch = _torch()
        with torch.cuda.device(self.device):
            _lib.ffst_plan_set_planes(self.handle, p0, p1)
        self.p0, self.p1 = int(p0), int(p1)

    def _stream(self):
        return _torch().cuda.current_stream(self.device).cuda_stream

    def _check_img(self, img):
        torch = _torch()
        if img.device != self.device or img.dtype != torch.float32 or tuple(img.shape) != (self.rows, self.cols):
            raise ValueError(f"expected a {self.rows}x{self.cols} float32 tensor on {self.device}, "
                             f"got {tuple(img.shape)} {img.dtype} on {img.device}")
        if not img.is_contiguous():
            raise ValueError("image must be contiguous")

    def _check_coeffs(self, c):
        if c.device != self.device or tuple(c.shape) != self.shape or not c.is_contiguous():
            raise ValueError(f"expected a contiguous {self.shape} tensor on {self.device}, "
                             f"got {tuple(c.shape)} on {c.device}")

    # -- transforms -----------------------------------------------------------
    def spectra(self, out=None):
        """Every plane's spectrum psi_hat_i, [eta, rows, cols] in FFT order."""
        torch = _torch()
        if out is None:
            out = torch.empty(self.full_shape, dtype=torch.float32, device=self.device)
        if out.device != self.device or tuple(out.shape) != self.full_shape or not out.is_contiguous():
            raise ValueError(f"expected a contiguous {self.full_shape} tensor on {self.device}")
        ffst_spectra(self.handle, out, self._stream())
        return out

    def forward(self, img, dtype=None, out=None, plane_scale=None):
        """Coefficient stack [eta, rows, cols].  For float16/bfloat16 storage
        also returns the per-plane scales (stored values are c_i * s_i)."""
        torch = _torch()
        self._check_img(img)
        if out is None:
            out = torch.empty(self.shape, dtype=dtype or torch.float32, device=self.device)
        self._check_coeffs(out)
        storage = _storage_of(out.dtype)
        if storage != FFST_STORE_F32 and plane_scale is None:
            plane_scale = torch.empty(self.num_planes, dtype=torch.float32, device=self.device)
        ffst_forward(self.handle, img, out, storage, plane_scale if storage != FFST_STORE_F32 else None,
                     self._stream())
        return (out, plane_scale) if storage != FFST_STORE_F32 else out

    def forward_stats(self, img, shrink=None, thresh=None, dtype=None, out=None, plane_scale=None):
        """Forward with fused per-plane statistics and optional shrinkage.

        shrink: None, "soft" or "hard"; thresh: per-plane thresholds (tensor
        [eta] on the device, or a float for every plane).  Returns
        (coeffs, mean_abs) with mean_abs[i] = d(i) of the unthresholded
        coefficients, plus the plane scales for float16/bfloat16 storage.
        """
        torch = _torch()
        self._check_img(img)
        if out is None:
            out = torch.empty(self.shape, dtype=dtype or torch.float32, device=self.device)
        self._check_coeffs(out)
        storage = _storage_of(out.dtype)
        if storage != FFST_STORE_F32 and plane_scale is None:
            plane_scale = torch.empty(self.num_planes, dtype=torch.float32, device=self.device)
        code = {None: 0, "soft": 1, "hard": 2}.get(shrink)
        if code is None:
            raise ValueError(f"shrink must be None, 'soft' or 'hard', not {shrink!r}")
        if code and thresh is None:
            raise ValueError("thresh is required for shrinkage")
        if code and not torch.is_tensor(thresh):
            thresh = torch.full((self.num_planes,), float(thresh), dtype=torch.float32, device=self.device)
        mean_abs = torch.empty(self.num_planes, dtype=torch.float32, device=self.device)
        ffst_forward_stats(self.handle, img, out, storage, plane_scale if storage != FFST_STORE_F32 else None, code,
                           thresh if code else None, mean_abs, self._stream())
        if storage != FFST_STORE_F32:
            return out, mean_abs, plane_scale
        return out, mean_abs

    def forward_complex(self, img, out=None):
        """One-sided (complex) shearlet coefficients of Sec. 3.8.2 as a planar
        float32 tensor [eta, 2, rows, cols] (real parts, imaginary parts);
        ``torch.complex(z[:, 0], z[:, 1])`` gives a complex64 copy."""
        torch = _torch()
        self._check_img(img)
        shape = (self.num_planes, 2, self.rows, self.cols)
        if out is None:
            out = torch.empty(shape, dtype=torch.float32, device=self.device)
        if out.device != self.device or out.dtype != torch.float32 or tuple(out.shape) != shape \
                or not out.is_contiguous():
            raise ValueError(f"expected a contiguous float32 tensor of shape {shape} on {self.device}")
        ffst_forward_complex(self.handle, img, out, self._stream())
        return out

    def inverse_complex(self, z, out=None):
        """Image from a planar complex stack of forward_complex."""
        torch = _torch()
        shape = (self.num_planes, 2, self.rows, self.cols)
        if z.device != self.device or z.dtype != torch.float32 or tuple(z.shape) != shape or not z.is_contiguous():
            raise ValueError(f"expected a contiguous float32 tensor of shape {shape} on {self.device}")
        if out is None:
            out = torch.empty((self.rows, self.cols), dtype=torch.float32, device=self.device)
        self._check_img(out)
        ffst_inverse_complex(self.handle, z, out, self._stream())
        return out

    def _synth(self, fn, coeffs, plane_scale, out):
        torch = _torch()
        self._check_coeffs(coeffs)
        storage = _storage_of(coeffs.dtype)
        if storage != FFST_STORE_F32 and plane_scale is None:
            raise ValueError("plane_scale is required for float16/bfloat16 coefficients")
        if out is None:
            out = torch.empty((self.rows, self.cols), dtype=torch.float32, device=self.device)
        self._check_img(out)
        fn(self.handle, coeffs, storage, plane_scale if storage != FFST_STORE_F32 else None, out, self._stream())
        return out

    def inverse(self, coeffs, plane_scale=None, out=None):
        return self._synth(ffst_inverse, coeffs, plane_scale, out)

    def adjoint(self, coeffs, plane_scale=None, out=None):
        return self._synth(ffst_adjoint, coeffs, plane_scale, out)

    def inverse_partial(self, coeffs, plane_scale=None, out=None):
        """sum over the active planes of psi_hat_i * fft2(c_i): the half spectrum
        [rows, cols//2 + 1] as complex64 (ffst_inverse_partial)."""
        torch = _torch()
        self._check_coeffs(coeffs)
        storage = _storage_of(coeffs.dtype)
        if storage != FFST_STORE_F32 and plane_scale is None:
            raise ValueError("plane_scale is required for float16/bfloat16 coefficients")
        shape = (self.rows, self.cols // 2 + 1)
        if out is None:
            out = torch.empty(shape, dtype=torch.complex64, device=self.device)
        if out.dtype != torch.complex64 or tuple(out.shape) != shape or not out.is_contiguous():
            raise ValueError(f"expected a contiguous complex64 tensor of shape {shape}")
        _lib.ffst_inverse_partial(self.handle, coeffs, storage, plane_scale if storage != FFST_STORE_F32 else None,
                                  torch.view_as_real(out), self._stream())
        return out

    def inverse_finish(self, spectrum, normalise: bool = True, out=None):
        """Image from a (reduced) half spectrum of inverse_partial; `spectrum` is
        overwritten (ffst_inverse_finish)."""
        torch = _torch()
        shape = (self.rows, self.cols // 2 + 1)
        if spectrum.dtype != torch.complex64 or tuple(spectrum.shape) != shape or not spectrum.is_contiguous():
            raise ValueError(f"expected a contiguous complex64 tensor of shape {shape}")
        if out is None:
            out = torch.empty((self.rows, self.cols), dtype=torch.float32, device=self.device)
        self._check_img(out)
        _lib.ffst_inverse_finish(self.handle, torch.view_as_real(spectrum), normalise, out, self._stream())
        return out

    # -- tuning ---------------------------------------------------------------
    def autotune(self, dtype=None, reps: int = 3):
        """Measure the plane-group budgets, keep the fastest per direction; returns (forward MB, inverse MB)."""
        torch = _torch()
        with torch.cuda.device(self.device):
            return ffst_plan_autotune(self.handle, _storage_of(dtype or torch.float32), reps)

    @property
    def group_mb(self):
        """(forward MB, inverse MB) plane-group budgets."""
        return ffst_plan_group_mb(self.handle)

    @property
    def schedule(self) -> int:
        """Schedule of the plane passes in effect (ffst_plan_set_schedule): 1 persistent, 0 grouped."""
        return ffst_plan_get_schedule(self.handle)

    @schedule.setter
    def schedule(self, mode: int):
        ffst_plan_set_schedule(self.handle, mode)

    @property
    def inverse_split(self) -> int:
        """Plane chunks of the inverse column pass (ffst_plan_set_inverse_split)."""
        return ffst_plan_get_inverse_split(self.handle)

    @inverse_split.setter
    def inverse_split(self, nsplit: int):
        ffst_plan_set_inverse_split(self.handle, nsplit)

    def schedule_info(self) -> dict:
        """Resident blocks, forward/inverse task counts and ring size of the persistent schedule."""
        return ffst_plan_schedule_info(self.handle)

    def check(self) -> int:
        """Synchronise the plan's stream; FFST_ERR_BOUNDS if a checked build caught an index outside its
        buffer, FFST_ERR_TIMEOUT if a bounded device wait ran out, else 0."""
        return ffst_plan_check(self.handle, self._stream())

    # -- timing ---------------------------------------------------------------
    def timing(self, enable: bool):
        ffst_timing_enable(self.handle, enable)

    def timing_reset(self):
        ffst_timing_reset(self.handle)

    def timing_read(self):
        """{kernel kind: (total_ms, launches, algorithmic_bytes)}"""
        out = {}
        for k in range(ffst_timing_kinds()):
            name, ms, n, by = ffst_timing_read(self.handle, k)
            out[name] = (ms, n, by)
        return out


class Graph:
    """An instantiated CUDA graph of batched transforms (ffst_graph_capture_batched)."""

    def __init__(self, handle: int, device, keep):
        self.handle = handle
        self.device = device
        self._keep = keep  # the tensors whose addresses are baked into the graph

    def launch(self, stream=None):
        torch = _torch()
        s = stream if stream is not None else torch.cuda.current_stream(self.device).cuda_stream
        ffst_graph_launch(self.handle, s)

    def close(self):
        if getattr(self, "handle", None):
            ffst_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchPlan:
    """Transforms of a batch of images of uneven sizes (ffst_plan_batched)."""

    def __init__(self, shapes, scales=None, lanes: int = 4, device=None):
        torch = _torch()
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        rows = [r for r, _ in shapes]
        cols = [c for _, c in shapes]
        with torch.cuda.device(self.device):
            self.handle = ffst_plan_batched(rows, cols, scales, lanes)
        self.info = [ffst_batch_info(self.handle, i) for i in range(len(shapes))]

    def __len__(self):
        return len(self.info)

    def shape(self, i):
        r, c, _, eta, _ = self.info[i]
        return (eta, r, c)

    def lanes(self):
        return [x[4] for x in self.info]

    def autotune(self, dtype=None, reps: int = 3):
        """Tune every distinct image shape once and use its configuration on all
        plans of that shape (ffst_batch_autotune)."""
        torch = _torch()
        with torch.cuda.device(self.device):
            _lib.ffst_batch_autotune(self.handle, _storage_of(dtype or torch.float32), reps)

    def close(self):
        if getattr(self, "handle", None):
            ffst_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _stream(self):
        return _torch().cuda.current_stream(self.device).cuda_stream

    def empty_stacks(self, dtype=None):
        torch = _torch()
        return [torch.empty(self.shape(i), dtype=dtype or torch.float32, device=self.device) for i in range(len(self))]

    def forward(self, imgs, outs=None, dtype=None, plane_scales=None):
        torch = _torch()
        outs = outs if outs is not None else self.empty_stacks(dtype)
        storage = _storage_of(outs[0].dtype)
        if storage != FFST_STORE_F32 and plane_scales is None:
            plane_scales = [torch.empty(self.shape(i)[0], device=self.device) for i in range(len(self))]
        ffst_forward_batched(self.handle, imgs, outs, storage, plane_scales if storage != FFST_STORE_F32 else None,
                             self._stream())
        return (outs, plane_scales) if storage != FFST_STORE_F32 else outs

    def inverse(self, stacks, plane_scales=None, outs=None):
        torch = _torch()
        outs = outs if outs is not None else [
            torch.empty(self.shape(i)[1:], device=self.device) for i in range(len(self))]
        ffst_inverse_batched(self.handle, stacks, _storage_of(stacks[0].dtype), plane_scales, outs, self._stream())
        return outs

    def capture(self, imgs, stacks, outs, what: int = 3, plane_scales=None) -> Graph:
        """One CUDA graph of the batched forward (what & 1) and/or inverse (what & 2)."""
        torch = _torch()
        with torch.cuda.device(self.device):
            h = ffst_graph_capture_batched(self.handle, what, imgs, stacks, _storage_of(stacks[0].dtype),
                                           plane_scales, outs)
        return Graph(h, self.device, (imgs, stacks, outs, plane_scales))


def _make_autograd():
    torch = _torch()

    class _Adjoint(torch.autograd.Function):
        @staticmethod
        def forward(ctx, coeffs, plan):
            ctx.plan = plan
            return plan.adjoint(coeffs.contiguous())

        @staticmethod
        def backward(ctx, grad_img):
            return _Forward.apply(grad_img.contiguous(), ctx.plan), None

    class _Forward(torch.autograd.Function):
        """x -> T x (Sec. 3.1); backward g -> T* g (the hand-written adjoint)."""

        @staticmethod
        def forward(ctx, img, plan):
            ctx.plan = plan
            return plan.forward(img.contiguous())

        @staticmethod
        def backward(ctx, grad_coeffs):
            return _Adjoint.apply(grad_coeffs.contiguous(), ctx.plan), None

    return _Forward, _Adjoint


_AUTOGRAD = None


def _autograd():
    global _AUTOGRAD
    if _AUTOGRAD is None:
        _AUTOGRAD = _make_autograd()
    return _AUTOGRAD


class _FFSTFunctionProxy:
    """``FFSTFunction.apply(img, plan)``: the differentiable forward transform."""

    @staticmethod
    def apply(img, plan):
        return _autograd()[0].apply(img, plan)


FFSTFunction = _FFSTFunctionProxy


def shearlet_transform(img, plan: Plan):
    """Differentiable T img; gradients flow through ``ffst_adjoint``."""
    return _autograd()[0].apply(img, plan)


def shearlet_adjoint(coeffs, plan: Plan):
    """Differentiable T* coeffs; its gradient is the forward transform."""
    return _autograd()[1].apply(coeffs, plan)
