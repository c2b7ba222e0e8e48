"""The allocation-free forward entry point against the planned forward and the oracle.

ffst_forward_noalloc serves callers that cannot call cudaMalloc (processes
whose framework holds nearly all device memory, plug-ins inside a host
application that owns the allocator, hosts that forbid allocation after
start-up): it keeps its tables and intermediates in a static device array
instead of plan-owned workspace.  These tests call it through the C ABI and
compare it with ffst_forward on the same images, twice in a row, so a stale
value left in the shared array by the first call would show up in the second;
each call is also compared with the FP64 oracle plane by plane.  The file is
named to be collected last.
"""

import numpy as np
import pytest

from oracle import ffst_oracle as o
from paper_1202_1773_gb300 import inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = 1e-5  # FP32 relative L2, as in the other parity tests


@pytest.fixture(scope="module")
def ffst():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1202_1773_gb300 as pkg
    from paper_1202_1773_gb300 import build

    build.build()
    return pkg


def _rel(a, b):
    return float(torch.linalg.norm((a - b).double()) / torch.linalg.norm(b.double()))


@pytest.mark.parametrize("shape", [(64, 64), (256, 256), (128, 32), (8, 16)])
def test_noalloc_forward_matches_planned_forward(ffst, shape):
    plan = ffst.Plan(*shape)
    stream = torch.cuda.current_stream().cuda_stream
    out = torch.empty(plan.shape, dtype=torch.float32, device="cuda")
    for seed in (1, 2):  # two calls in a row on the shared scratch
        x = torch.from_numpy(inputs.scaled_cartoon(*shape, seed=seed)).cuda()
        ref = plan.forward(x)
        out.fill_(float("nan"))
        ffst.ffst_forward_noalloc(shape[0], shape[1], 0, x, out, stream)
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        assert _rel(out, ref) <= TOL
        # against the FP64 oracle, every plane relative to its own energy
        # (floored at 1e-3 of the image's, for planes that carry almost none)
        f = x.cpu().numpy().astype(np.float64)
        cref = o.forward(f)
        got = out.cpu().numpy()
        floor = 1e-3 * np.linalg.norm(f)
        for i in range(cref.shape[0]):
            err = np.linalg.norm(got[i] - cref[i]) / max(np.linalg.norm(cref[i]), floor)
            assert err <= TOL, (i, err)


def test_noalloc_rejects_sizes_beyond_the_static_limit(ffst):
    from paper_1202_1773_gb300 import _lib

    x = torch.zeros(512, 512, device="cuda")
    c = torch.empty(1, device="cuda")
    with pytest.raises(ffst.FFSTError) as ei:
        ffst.ffst_forward_noalloc(512, 512, 0, x, c, None)
    assert ei.value.status == _lib.FFST_ERR_UNSUPPORTED_SIZE
    assert "static scratch" in _lib.last_error()
    with pytest.raises(ffst.FFSTError) as ei:
        ffst.ffst_forward_noalloc(64, 64, 5, x, c, None)
    assert ei.value.status == _lib.FFST_ERR_UNSUPPORTED_SIZE
