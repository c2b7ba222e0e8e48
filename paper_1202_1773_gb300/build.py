"""Build libffst.so (the C-ABI CUDA library) in-tree for sm_103a.

Each translation unit under ``csrc/`` is compiled by its own nvcc process
(in parallel), then linked into ``_build/libffst.so``.  A unit is recompiled
only when it or a header under ``csrc/`` / ``include/`` is newer than its
object file.  Usage: ``python -m paper_1202_1773_gb300.build`` or
``build()`` from Python.
"""

from __future__ import annotations

import glob
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libffst.so")


def variant_dir(tag: str | None) -> str:
    """Build directory of a tagged variant (``_build_<tag>``), or the default."""
    return BUILD if not tag else os.path.join(PKG, "_build_" + tag)


ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc_path() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the FFST CUDA library cannot be built")


def _flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
                   "-I", os.path.join(ROOT, "include")] + list(extra)


def _headers():
    return glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(ROOT, "include", "*.h"))


def _stale(obj: str, src: str, hdr_mtime: float) -> bool:
    if not os.path.exists(obj):
        return True
    m = os.path.getmtime(obj)
    return m < os.path.getmtime(src) or m < hdr_mtime


def build(verbose: bool = False, extra_flags=(), jobs: int | None = None, tag: str | None = None) -> str:
    """Compile and link libffst.so; return its path.

    ``extra_flags`` (e.g. ``-DFFST_ROW_E_LONG=16``) with a ``tag`` build a
    variant into its own directory, loadable through ``FFST_LIB_PATH``.
    """
    nvcc = nvcc_path()
    bdir = variant_dir(tag)
    lib_path = os.path.join(bdir, "libffst.so")
    os.makedirs(bdir, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    hdr_mtime = max([os.path.getmtime(h) for h in _headers()] + [0.0])
    flags = _flags(extra_flags)

    def compile_one(src):
        obj = os.path.join(bdir, os.path.basename(src)[:-3] + ".o")
        if not _stale(obj, src, hdr_mtime):
            return obj, None
        cmd = [nvcc] + flags + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            return obj, "$ " + " ".join(cmd) + "\n" + r.stdout + r.stderr
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)
        return obj, None

    jobs = jobs or min(len(srcs), os.cpu_count() or 4)
    with ThreadPoolExecutor(max_workers=jobs) as ex:
        results = list(ex.map(compile_one, srcs))
    errors = [e for _, e in results if e]
    if errors:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errors))
    objs = [o for o, _ in results]
    if not os.path.exists(lib_path) or any(os.path.getmtime(o) > os.path.getmtime(lib_path) for o in objs):
        cmd = [nvcc] + ARCH + ["-shared", "-o", lib_path] + objs + ["-lcudart", "-ldl"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n$ " + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return lib_path


if __name__ == "__main__":
    import sys
    import time

    t0 = time.time()
    tag = None
    flags = []
    for a in sys.argv[1:]:
        if a.startswith("--tag="):
            tag = a.split("=", 1)[1]
        elif a.startswith("-D"):
            flags.append(a)
    path = build(verbose="-v" in sys.argv, extra_flags=flags, tag=tag)
    print(f"built {path} in {time.time() - t0:.1f}s")
