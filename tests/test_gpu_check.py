"""The bounds-checked debug build (-DFFST_CHECK) on the GPU.

In a checked build every global access of the native transform bodies is
tested against its buffer's extent; an access outside is skipped and
reported by ffst_plan_check as FFST_ERR_BOUNDS.  This builds that variant,
runs it in a child process (one library per process) on the native sizes
and forms, including 4096x4096 J=6 whose stack of 4.2e9 coefficients needs
64-bit indices, and requires no report and results matching the FP64 oracle
(sampled planes, relative to each plane's energy floored at 1e-3 of the
image's).
"""

import os
import subprocess
import sys
import textwrap

import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent("""
    import sys
    import numpy as np
    import torch
    sys.path.insert(0, {root!r})
    import paper_1202_1773_gb300 as ffst
    from oracle import ffst_oracle as o
    from paper_1202_1773_gb300 import inputs

    def plane_err(got, ref, f):
        return np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-3 * np.linalg.norm(f))

    cases = [((64, 64), None), ((256, 256), None), ((480, 640), None), ((128, 256), "float16"),
             ((2048, 2048), "bfloat16"), ((4096, 4096), None)]
    for (rows, cols), dt in cases:
        p = ffst.Plan(rows, cols)
        f = inputs.scaled_cartoon(rows, cols, seed=8)
        x = torch.from_numpy(f).cuda()
        if dt is None:
            c, sc = p.forward(x), None
        else:
            c, sc = p.forward(x, dtype=getattr(torch, dt))
        F = np.fft.fft2(f.astype(np.float64))
        tol = {{None: 1e-5, "float16": 2e-3, "bfloat16": 1e-2}}[dt]
        for i in sorted({{0, p.num_planes // 2, p.num_planes - 1}}):
            got = c[i].float().cpu().numpy() / (1.0 if sc is None else float(sc[i]))
            e = plane_err(got, o.forward_plane(F, p.scales, i), f)
            assert e <= tol, (rows, cols, dt, i, e)
        r = p.inverse(c, sc)
        assert float(torch.linalg.norm(r - x) / torch.linalg.norm(x)) <= tol
        st = p.check()
        assert st == 0, ("bounds report", rows, cols, st, ffst._lib.last_error())
        del c, r
        p.close()
    print("checked build: no bounds report")
""")


def test_checked_build_reports_nothing():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1202_1773_gb300 import build

    lib = build.build(extra_flags=["-DFFST_CHECK"], tag="check")
    env = dict(os.environ, FFST_LIB_PATH=lib)
    r = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT)], env=env, capture_output=True, text=True,
                       timeout=1500, cwd=ROOT)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "no bounds report" in r.stdout
