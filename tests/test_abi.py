"""The C-ABI library builds, loads and exports every entry point of include/ffst.h.

Host-side argument checks are exercised too: these calls return before any
CUDA work, so they run without a GPU.
"""

import ctypes
import os
import re

import pytest

from paper_1202_1773_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "ffst.h")) as fh:
        src = fh.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ffst_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 14
    for name in names:
        assert hasattr(lib, name), name
    # and the binding declares a prototype for each of them
    bound = {n for n, _, _ in _lib.SIGNATURES}
    assert set(names) <= bound, set(names) - bound


def test_status_strings(lib):
    assert _lib.status_name(0) == "FFST_OK"
    assert _lib.status_name(2) == "FFST_ERR_UNSUPPORTED_SIZE"
    assert _lib.status_name(99) == "FFST_ERR_UNKNOWN"


@pytest.mark.parametrize("rows,cols,scales", [(0, 64, 0), (64, 0, 0), (3001, 64, 0), (64, 2050, 0), (2049, 63, 0),
                                              (4, 64, 0), (64, 8192, 0), (64, 64, 9)])
def test_unsupported_sizes_rejected_on_host(lib, rows, cols, scales):
    out = ctypes.c_void_p()
    st = lib.ffst_plan(rows, cols, scales, ctypes.byref(out))
    assert st == _lib.FFST_ERR_UNSUPPORTED_SIZE
    assert out.value is None
    assert "ffst_plan" in _lib.last_error()


@pytest.mark.parametrize("rows,cols", [(63, 64), (64, 63), (131, 137), (2048, 2047), (4096, 64), (2000, 4096),
                                       (3000, 64), (2160, 3840), (64, 3087)])
def test_generic_sizes_pass_the_size_check(lib, rows, cols):
    # odd, prime and other lengths without a native FFT line (Bluestein lines
    # up to 2048, mixed-radix lines for lengths with no prime factor above 7
    # up to 4096, native lines up to 4096) are accepted: without a GPU the
    # call fails later, in CUDA, never with FFST_ERR_UNSUPPORTED_SIZE
    out = ctypes.c_void_p()
    st = lib.ffst_plan(rows, cols, 0, ctypes.byref(out))
    if st == _lib.FFST_OK:
        lib.ffst_destroy(out)
    assert st != _lib.FFST_ERR_UNSUPPORTED_SIZE, _lib.last_error()


def test_bluestein_switch_limits_generic_lengths(lib, monkeypatch):
    # with FFST_BLUESTEIN=1 every generic length runs Bluestein lines, which
    # stop at 2048: 3000 = 2^3 3 5^3 is then rejected on the host
    monkeypatch.setenv("FFST_BLUESTEIN", "1")
    out = ctypes.c_void_p()
    assert lib.ffst_plan(3000, 64, 0, ctypes.byref(out)) == _lib.FFST_ERR_UNSUPPORTED_SIZE
    assert out.value is None


def test_null_arguments_rejected_on_host(lib):
    assert lib.ffst_plan(64, 64, 0, None) == _lib.FFST_ERR_INVALID_ARG
    assert lib.ffst_plan_ex(64, 64, 0, 1, 0, 0, 0, 0, None) == _lib.FFST_ERR_INVALID_ARG
    assert lib.ffst_plan_info(None, None, None, None, None) == _lib.FFST_ERR_INVALID_ARG
    assert lib.ffst_plane_index(None, 0, None, None, None) == _lib.FFST_ERR_INVALID_ARG
    assert lib.ffst_forward(None, None, None, 0, None, None) == _lib.FFST_ERR_INVALID_ARG
    assert lib.ffst_forward_stats(None, None, None, 0, None, 0, None, None, None) == _lib.FFST_ERR_INVALID_ARG
    assert lib.ffst_forward_complex(None, None, None, None) == _lib.FFST_ERR_INVALID_ARG
    assert lib.ffst_inverse_complex(None, None, None, None) == _lib.FFST_ERR_INVALID_ARG
    assert lib.ffst_inverse(None, None, 0, None, None, None) == _lib.FFST_ERR_INVALID_ARG
    assert lib.ffst_adjoint(None, None, 0, None, None, None) == _lib.FFST_ERR_INVALID_ARG
    assert lib.ffst_spectra(None, None, None) == _lib.FFST_ERR_INVALID_ARG
    assert lib.ffst_timing_enable(None, 1) == _lib.FFST_ERR_INVALID_ARG
    assert lib.ffst_plan_set_schedule(None, 1) == _lib.FFST_ERR_INVALID_ARG
    assert lib.ffst_plan_get_schedule(None, None) == _lib.FFST_ERR_INVALID_ARG
    assert lib.ffst_plan_check(None, None) == _lib.FFST_ERR_INVALID_ARG
    assert lib.ffst_plan_schedule_info(None, None, None, None, None) == _lib.FFST_ERR_INVALID_ARG
    assert lib.ffst_plan_set_inverse_split(None, 1) == _lib.FFST_ERR_INVALID_ARG
    assert lib.ffst_plan_get_inverse_split(None, None) == _lib.FFST_ERR_INVALID_ARG
    lib.ffst_destroy(None)  # no-op
    with pytest.raises(_lib.FFSTError):
        _lib.ffst_plan(64, 2050, 0)


def test_batch_and_graph_argument_errors_on_host(lib):
    out = ctypes.c_void_p()
    rows = (ctypes.c_int * 1)(64)
    cols = (ctypes.c_int * 1)(64)
    assert lib.ffst_plan_batched(0, rows, cols, None, 4, ctypes.byref(out)) == _lib.FFST_ERR_INVALID_ARG
    assert lib.ffst_plan_batched(1, rows, cols, None, 0, ctypes.byref(out)) == _lib.FFST_ERR_INVALID_ARG
    assert lib.ffst_plan_batched(1, None, cols, None, 4, ctypes.byref(out)) == _lib.FFST_ERR_INVALID_ARG
    bad = (ctypes.c_int * 1)(3001)
    assert lib.ffst_plan_batched(1, bad, cols, None, 4, ctypes.byref(out)) == _lib.FFST_ERR_UNSUPPORTED_SIZE
    assert lib.ffst_batch_info(None, 0, None, None, None, None, None) == _lib.FFST_ERR_INVALID_ARG
    assert lib.ffst_forward_batched(None, None, None, 0, None, None) == _lib.FFST_ERR_INVALID_ARG
    assert lib.ffst_graph_launch(None, None) == _lib.FFST_ERR_INVALID_ARG
    assert lib.ffst_plan_autotune(None, 0, 1, None, None) == _lib.FFST_ERR_INVALID_ARG
    assert lib.ffst_plan_group_mb(None, None, None) == _lib.FFST_ERR_INVALID_ARG
    lib.ffst_graph_destroy(None)
    lib.ffst_batch_destroy(None)


def test_checked_build_compiles():
    # the bounds-checked debug build (-DFFST_CHECK) of the instrumented
    # transform bodies compiles for sm_103a: the fused launches hold all four
    # plane-pass bodies (the whole checked build runs on the GPU in
    # tests/test_gpu_check.py)
    import shutil
    import subprocess
    import tempfile

    from paper_1202_1773_gb300 import build

    try:
        nvcc = build.nvcc_path()
    except RuntimeError:
        pytest.skip("nvcc not available")
    with tempfile.TemporaryDirectory() as d:
        for unit in ("ffst_fused.cu",):
            src = os.path.join(build.CSRC, unit)
            cmd = [nvcc] + build._flags(["-DFFST_CHECK"]) + ["-c", src, "-o", os.path.join(d, unit + ".o")]
            r = subprocess.run(cmd, capture_output=True, text=True)
            assert r.returncode == 0, r.stderr[-3000:]
    assert shutil.which(nvcc) or os.path.exists(nvcc)
