"""ctypes binding of libffst.so: the C ABI declared in include/ffst.h.

Each ``ffst_*`` function here has the name and argument order of the C
entry point and does argument marshalling only (integers, device pointers
as Python ints, stream handles).  A missing or unloadable library raises:
there is no CPU fallback.
"""

from __future__ import annotations

import ctypes
import os

from . import build as _build

FFST_OK = 0
FFST_ERR_INVALID_ARG = 1
FFST_ERR_UNSUPPORTED_SIZE = 2
FFST_ERR_OUT_OF_MEMORY = 3
FFST_ERR_CUDA = 4
FFST_ERR_TIMEOUT = 5
FFST_ERR_BOUNDS = 6

FFST_STORE_F32 = 0
FFST_STORE_F16 = 1
FFST_STORE_BF16 = 2

CONE_NAMES = {0: "lowpass", 1: "h", 2: "v", 3: "seam"}

# (name, restype, argtypes) of every entry point in include/ffst.h
_VP = ctypes.c_void_p
_I = ctypes.c_int
SIGNATURES = [
    ("ffst_plan", _I, [_I, _I, _I, ctypes.POINTER(_VP)]),
    ("ffst_plan_ex", _I, [_I, _I, _I, _I, _I, _I, _I, _I, ctypes.POINTER(_VP)]),
    ("ffst_plan_info", _I, [_VP, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    ("ffst_plane_index", _I, [_VP, _I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    ("ffst_spectra", _I, [_VP, _VP, _VP]),
    ("ffst_forward", _I, [_VP, _VP, _VP, _I, _VP, _VP]),
    ("ffst_inverse", _I, [_VP, _VP, _I, _VP, _VP, _VP]),
    ("ffst_adjoint", _I, [_VP, _VP, _I, _VP, _VP, _VP]),
    ("ffst_forward_noalloc", _I, [_I, _I, _I, _VP, _VP, _VP]),
    ("ffst_forward_stats", _I, [_VP, _VP, _VP, _I, _VP, _I, _VP, _VP, _VP]),
    ("ffst_forward_complex", _I, [_VP, _VP, _VP, _VP]),
    ("ffst_inverse_complex", _I, [_VP, _VP, _VP, _VP]),
    ("ffst_plan_autotune", _I, [_VP, _I, _I, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    ("ffst_plan_group_mb", _I, [_VP, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    ("ffst_plan_set_schedule", _I, [_VP, _I]),
    ("ffst_plan_get_schedule", _I, [_VP, ctypes.POINTER(_I)]),
    ("ffst_plan_set_inverse_split", _I, [_VP, _I]),
    ("ffst_plan_set_planes", _I, [_VP, _I, _I]),
    ("ffst_plan_set_kernels", _I, [_VP, _I, _I, _I, _I]),
    ("ffst_plan_get_kernels", _I, [_VP, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I),
                                   ctypes.POINTER(_I)]),
    ("ffst_plan_get_planes", _I, [_VP, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    ("ffst_inverse_partial", _I, [_VP, _VP, _I, _VP, _VP, _VP]),
    ("ffst_inverse_finish", _I, [_VP, _VP, _I, _VP, _VP]),
    ("ffst_plan_get_inverse_split", _I, [_VP, ctypes.POINTER(_I)]),
    ("ffst_plan_check", _I, [_VP, _VP]),
    ("ffst_plan_schedule_info", _I, [_VP, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I),
                                     ctypes.POINTER(ctypes.c_double)]),
    ("ffst_plan_batched", _I, [_I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I), _I,
                               ctypes.POINTER(_VP)]),
    ("ffst_batch_info", _I, [_VP, _I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I),
                             ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    ("ffst_forward_batched", _I, [_VP, ctypes.POINTER(_VP), ctypes.POINTER(_VP), _I, ctypes.POINTER(_VP), _VP]),
    ("ffst_inverse_batched", _I, [_VP, ctypes.POINTER(_VP), _I, ctypes.POINTER(_VP), ctypes.POINTER(_VP), _VP]),
    ("ffst_batch_destroy", None, [_VP]),
    ("ffst_batch_autotune", _I, [_VP, _I, _I]),
    ("ffst_graph_capture_batched", _I, [_VP, _I, ctypes.POINTER(_VP), ctypes.POINTER(_VP), _I,
                                        ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.POINTER(_VP)]),
    ("ffst_graph_launch", _I, [_VP, _VP]),
    ("ffst_graph_destroy", None, [_VP]),
    ("ffst_destroy", None, [_VP]),
    ("ffst_last_error", ctypes.c_char_p, []),
    ("ffst_status_string", ctypes.c_char_p, [_I]),
    ("ffst_timing_enable", _I, [_VP, _I]),
    ("ffst_timing_reset", _I, [_VP]),
    ("ffst_timing_kinds", _I, []),
    ("ffst_timing_read", _I, [_VP, _I, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_double),
                              ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_double)]),
]

_LIB = None


class FFSTError(RuntimeError):
    """A libffst call returned a status other than FFST_OK."""

    def __init__(self, fn: str, status: int, message: str):
        super().__init__(f"{fn}: {status_name(status)}: {message}")
        self.status = status


def library_path() -> str:
    """The library to load: ``FFST_LIB_PATH`` if set (a tagged variant
    build), else the default in-tree build."""
    return os.environ.get("FFST_LIB_PATH") or _build.LIB


def lib() -> ctypes.CDLL:
    """Load libffst.so (built in-tree by ``build()``) and declare its prototypes."""
    global _LIB
    if _LIB is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"libffst.so is not built ({path}); run paper_1202_1773_gb300.build.build()")
        handle = ctypes.CDLL(path)
        for name, res, args in SIGNATURES:
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = handle
    return _LIB


def status_name(status: int) -> str:
    return lib().ffst_status_string(int(status)).decode()


def last_error() -> str:
    return lib().ffst_last_error().decode()


def _check(fn: str, status: int):
    if status != FFST_OK:
        raise FFSTError(fn, status, last_error())


def _ptr(x) -> int | None:
    """Device pointer of a tensor-like object, or an int/None passed through."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


# --- C-ABI wrappers (same names as the C entry points) -----------------------

FFST_VARIANT_CLASSIC = 0
FFST_VARIANT_SMOOTH = 1
FFST_V_MEYER, FFST_V_QUADRATIC, FFST_V_POLY, FFST_V_CINF = 0, 1, 2, 3
FFST_MAXSCALE_MAX, FFST_MAXSCALE_MIN = 0, 1
FFST_SPACING_COMMON, FFST_SPACING_PER_AXIS = 0, 1


def ffst_plan(rows: int, cols: int, scales: int = 0, variant: int = FFST_VARIANT_CLASSIC, vfun: int = FFST_V_MEYER,
              vorder: int = 0, max_scale: int = FFST_MAXSCALE_MAX, spacing: int = FFST_SPACING_COMMON) -> int:
    out = _VP()
    if (variant, vfun, max_scale, spacing) == (FFST_VARIANT_CLASSIC, FFST_V_MEYER, FFST_MAXSCALE_MAX,
                                               FFST_SPACING_COMMON):
        _check("ffst_plan", lib().ffst_plan(int(rows), int(cols), int(scales), ctypes.byref(out)))
    else:
        _check("ffst_plan_ex", lib().ffst_plan_ex(int(rows), int(cols), int(scales), int(variant), int(vfun),
                                                  int(vorder), int(max_scale), int(spacing), ctypes.byref(out)))
    return out.value


def ffst_plan_info(plan: int):
    r, c, s, n = _I(), _I(), _I(), _I()
    _check("ffst_plan_info", lib().ffst_plan_info(plan, ctypes.byref(r), ctypes.byref(c), ctypes.byref(s),
                                                  ctypes.byref(n)))
    return r.value, c.value, s.value, n.value


def ffst_plane_index(plan: int, i: int):
    cone, j, k = _I(), _I(), _I()
    _check("ffst_plane_index", lib().ffst_plane_index(plan, int(i), ctypes.byref(cone), ctypes.byref(j),
                                                      ctypes.byref(k)))
    return cone.value, j.value, k.value


def ffst_spectra(plan: int, psi, stream=None):
    _check("ffst_spectra", lib().ffst_spectra(plan, _ptr(psi), stream))


def ffst_forward(plan: int, img, coeffs, storage: int = FFST_STORE_F32, plane_scale=None, stream=None):
    _check("ffst_forward", lib().ffst_forward(plan, _ptr(img), _ptr(coeffs), int(storage), _ptr(plane_scale), stream))


def ffst_forward_stats(plan: int, img, coeffs, storage: int, plane_scale, shrink: int, thresh, mean_abs, stream: int):
    _check("ffst_forward_stats", lib().ffst_forward_stats(plan, _ptr(img), _ptr(coeffs), int(storage), _ptr(plane_scale),
                                                          int(shrink), _ptr(thresh), _ptr(mean_abs), stream))


def ffst_forward_complex(plan: int, img, coeffs, stream: int):
    _check("ffst_forward_complex", lib().ffst_forward_complex(plan, _ptr(img), _ptr(coeffs), stream))


def ffst_inverse_complex(plan: int, coeffs, img, stream: int):
    _check("ffst_inverse_complex", lib().ffst_inverse_complex(plan, _ptr(coeffs), _ptr(img), stream))


def ffst_inverse(plan: int, coeffs, storage: int, plane_scale, img, stream=None):
    _check("ffst_inverse", lib().ffst_inverse(plan, _ptr(coeffs), int(storage), _ptr(plane_scale), _ptr(img), stream))


def ffst_adjoint(plan: int, coeffs, storage: int, plane_scale, img, stream=None):
    _check("ffst_adjoint", lib().ffst_adjoint(plan, _ptr(coeffs), int(storage), _ptr(plane_scale), _ptr(img), stream))


def ffst_forward_noalloc(rows: int, cols: int, scales: int, img, coeffs, stream=None):
    """Allocation-free forward transform of a small image (see include/ffst.h)."""
    _check("ffst_forward_noalloc", lib().ffst_forward_noalloc(int(rows), int(cols), int(scales), _ptr(img),
                                                              _ptr(coeffs), stream))


def ffst_plan_autotune(plan: int, storage: int = FFST_STORE_F32, reps: int = 3):
    """(forward MB, inverse MB) chosen."""
    f, i = ctypes.c_double(), ctypes.c_double()
    _check("ffst_plan_autotune", lib().ffst_plan_autotune(plan, int(storage), int(reps), ctypes.byref(f), ctypes.byref(i)))
    return f.value, i.value


def ffst_plan_group_mb(plan: int):
    """(forward MB, inverse MB)."""
    f, i = ctypes.c_double(), ctypes.c_double()
    _check("ffst_plan_group_mb", lib().ffst_plan_group_mb(plan, ctypes.byref(f), ctypes.byref(i)))
    return f.value, i.value


def ffst_plan_set_schedule(plan: int, mode: int):
    _check("ffst_plan_set_schedule", lib().ffst_plan_set_schedule(plan, int(mode)))


def ffst_plan_get_schedule(plan: int) -> int:
    mode = _I()
    _check("ffst_plan_get_schedule", lib().ffst_plan_get_schedule(plan, ctypes.byref(mode)))
    return mode.value


def ffst_plan_check(plan: int, stream: int = 0) -> int:
    """Status of the device-side checks since the last call: FFST_ERR_BOUNDS, FFST_ERR_TIMEOUT or 0; raises nothing."""
    return int(lib().ffst_plan_check(plan, stream))


def ffst_plan_set_inverse_split(plan: int, nsplit: int):
    _check("ffst_plan_set_inverse_split", lib().ffst_plan_set_inverse_split(plan, int(nsplit)))


def ffst_plan_set_kernels(plan: int, fuse_fwd: int, fuse_inv: int, row_fwd: int, row_inv: int):
    _check("ffst_plan_set_kernels", lib().ffst_plan_set_kernels(plan, int(fuse_fwd), int(fuse_inv), int(row_fwd),
                                                                int(row_inv)))


def ffst_plan_get_kernels(plan: int):
    v = [_I() for _ in range(4)]
    _check("ffst_plan_get_kernels", lib().ffst_plan_get_kernels(plan, *[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)


def ffst_plan_set_planes(plan: int, p0: int, p1: int):
    _check("ffst_plan_set_planes", lib().ffst_plan_set_planes(plan, int(p0), int(p1)))


def ffst_plan_get_planes(plan: int):
    a, b = _I(), _I()
    _check("ffst_plan_get_planes", lib().ffst_plan_get_planes(plan, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def ffst_inverse_partial(plan: int, coeffs, storage: int, plane_scale, spectrum, stream=None):
    _check("ffst_inverse_partial", lib().ffst_inverse_partial(plan, _ptr(coeffs), int(storage), _ptr(plane_scale),
                                                              _ptr(spectrum), stream))


def ffst_inverse_finish(plan: int, spectrum, normalise: bool, img, stream=None):
    _check("ffst_inverse_finish", lib().ffst_inverse_finish(plan, _ptr(spectrum), int(bool(normalise)), _ptr(img),
                                                            stream))


def ffst_plan_get_inverse_split(plan: int) -> int:
    n = _I()
    _check("ffst_plan_get_inverse_split", lib().ffst_plan_get_inverse_split(plan, ctypes.byref(n)))
    return n.value


def ffst_plan_schedule_info(plan: int) -> dict:
    b, f, i, mb = _I(), _I(), _I(), ctypes.c_double()
    _check("ffst_plan_schedule_info", lib().ffst_plan_schedule_info(plan, ctypes.byref(b), ctypes.byref(f),
                                                                   ctypes.byref(i), ctypes.byref(mb)))
    return {"blocks": b.value, "fwd_tasks": f.value, "inv_tasks": i.value, "ring_mb": mb.value}


def _ints(vals):
    return (_I * len(vals))(*[int(v) for v in vals])


def _ptrs(vals):
    if vals is None:
        return None
    return (_VP * len(vals))(*[_ptr(v) for v in vals])


def ffst_plan_batched(rows, cols, scales=None, lanes: int = 4) -> int:
    out = _VP()
    n = len(rows)
    _check("ffst_plan_batched", lib().ffst_plan_batched(n, _ints(rows), _ints(cols),
                                                        _ints(scales) if scales is not None else None, int(lanes),
                                                        ctypes.byref(out)))
    return out.value


def ffst_batch_info(batch: int, i: int):
    r, c, s, n, lane = _I(), _I(), _I(), _I(), _I()
    _check("ffst_batch_info", lib().ffst_batch_info(batch, int(i), ctypes.byref(r), ctypes.byref(c), ctypes.byref(s),
                                                    ctypes.byref(n), ctypes.byref(lane)))
    return r.value, c.value, s.value, n.value, lane.value


def ffst_forward_batched(batch: int, imgs, coeffs, storage: int = FFST_STORE_F32, plane_scales=None, stream=None):
    _check("ffst_forward_batched", lib().ffst_forward_batched(batch, _ptrs(imgs), _ptrs(coeffs), int(storage),
                                                              _ptrs(plane_scales), stream))


def ffst_inverse_batched(batch: int, coeffs, storage: int, plane_scales, imgs, stream=None):
    _check("ffst_inverse_batched", lib().ffst_inverse_batched(batch, _ptrs(coeffs), int(storage), _ptrs(plane_scales),
                                                              _ptrs(imgs), stream))


def ffst_batch_destroy(batch: int):
    if batch:
        lib().ffst_batch_destroy(batch)


def ffst_batch_autotune(batch: int, storage: int = FFST_STORE_F32, reps: int = 3):
    _check("ffst_batch_autotune", lib().ffst_batch_autotune(batch, int(storage), int(reps)))


def ffst_graph_capture_batched(batch: int, what: int, imgs, coeffs, storage: int, plane_scales, out_imgs) -> int:
    out = _VP()
    _check("ffst_graph_capture_batched", lib().ffst_graph_capture_batched(
        batch, int(what), _ptrs(imgs), _ptrs(coeffs), int(storage), _ptrs(plane_scales), _ptrs(out_imgs),
        ctypes.byref(out)))
    return out.value


def ffst_graph_launch(graph_exec: int, stream=None):
    _check("ffst_graph_launch", lib().ffst_graph_launch(graph_exec, stream))


def ffst_graph_destroy(graph_exec: int):
    if graph_exec:
        lib().ffst_graph_destroy(graph_exec)


def ffst_destroy(plan: int):
    if plan:
        lib().ffst_destroy(plan)


def ffst_timing_enable(plan: int, enable: bool):
    _check("ffst_timing_enable", lib().ffst_timing_enable(plan, 1 if enable else 0))


def ffst_timing_reset(plan: int):
    _check("ffst_timing_reset", lib().ffst_timing_reset(plan))


def ffst_timing_kinds() -> int:
    return lib().ffst_timing_kinds()


def ffst_timing_read(plan: int, kind: int):
    name = ctypes.c_char_p()
    ms = ctypes.c_double()
    n = ctypes.c_longlong()
    by = ctypes.c_double()
    _check("ffst_timing_read", lib().ffst_timing_read(plan, int(kind), ctypes.byref(name), ctypes.byref(ms),
                                                      ctypes.byref(n), ctypes.byref(by)))
    return name.value.decode(), ms.value, n.value, by.value
