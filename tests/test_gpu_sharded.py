"""Plane-sharded transforms through the C ABI (ffst_plan_set_planes,
ffst_inverse_partial, ffst_inverse_finish) on one GPU.

The ranks of a sharded run are emulated one after another in this process
(each with its own plan restricted to its plane range; nothing waits on
another rank): every rank's forward equals the matching planes of the
unsharded forward bit for bit (a plane's passes do not depend on which
other planes run), and the sum of the ranks' partial spectra, finished on
one plan, reconstructs the image within 1e-5 and matches the unsharded
inverse and adjoint within 1e-5 (the FP32 sums run in another order).
"""

import numpy as np
import pytest

from oracle import ffst_oracle as o
from paper_1202_1773_gb300 import inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("shape", [(256, 256), (128, 256), (480, 640), (63, 65)])
def test_sharded_matches_unsharded(ffst, shape, world):
    from paper_1202_1773_gb300 import sharded

    f = inputs.scaled_cartoon(*shape, seed=21)
    x = torch.from_numpy(f).cuda()
    full = ffst.Plan(*shape)
    c = full.forward(x)
    rec = full.inverse(c)
    adj = full.adjoint(c)
    total = None
    plans = []
    for r in range(world):
        p = ffst.Plan(*shape)
        p0, p1 = sharded.plane_range(p.num_planes, world, r)
        p.set_planes(p0, p1)
        assert p.shape == (p1 - p0,) + tuple(shape)
        local = p.forward(x)
        assert torch.equal(local, c[p0:p1]), (r, p0, p1)
        spec = p.inverse_partial(local)
        total = spec.clone() if total is None else total + spec
        plans.append(p)
    img = plans[0].inverse_finish(total.clone())
    assert _rel(img, x) <= 1e-5
    assert _rel(img, rec) <= 1e-5
    assert _rel(plans[0].inverse_finish(total.clone(), normalise=False), adj) <= 1e-5
    # against the oracle's inverse of the same stack
    ref = o.inverse(c.cpu().numpy().astype(np.float64))
    assert np.linalg.norm(img.cpu().numpy() - ref) <= 1e-5 * np.linalg.norm(ref)
    for p in plans:
        p.close()
    full.close()


def test_plane_range_checked(ffst):
    p = ffst.Plan(64, 64)
    for bad in ((0, 0), (-1, 5), (5, 3), (0, p.num_planes + 1)):
        with pytest.raises(ffst.FFSTError):
            p.set_planes(*bad)
    p.set_planes(3, 9)
    assert p.shape == (6, 64, 64)
    from paper_1202_1773_gb300 import _lib

    assert _lib.ffst_plan_get_planes(p.handle) == (3, 9)
    p.set_planes(0, p.num_planes)  # back to every plane
    x = torch.from_numpy(inputs.scaled_cartoon(64, 64, seed=2)).cuda()
    assert torch.equal(p.forward(x), ffst.Plan(64, 64).forward(x))
    p.close()
