"""GPU parity for both grid steps of non-square images (Sec. 3.5.1).

FFST_SPACING_COMMON (one step Delta for both axes, the default) and
FFST_SPACING_PER_AXIS (each axis stretched to [-X, X]) against the FP64
oracle with the same option: spectra on every plane (max abs <= 1e-6, FP32
window generation of values in [0, 1]), coefficients plane by plane (relative
L2 <= 1e-5 against the plane's own energy, floored at 1e-3 of the image's)
and reconstruction (relative L2 <= 1e-5).  The large shapes compare sampled
planes; the oracle computes each from fft2(f) on its own.
"""

import numpy as np
import pytest

from oracle import ffst_oracle as o
from paper_1202_1773_gb300 import inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def ffst():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1202_1773_gb300 as pkg
    from paper_1202_1773_gb300 import build

    build.build()
    return pkg


def _plane_err(got, ref, f):
    return np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-3 * np.linalg.norm(f))


@pytest.mark.parametrize("spacing", ["common", "per_axis"])
@pytest.mark.parametrize("shape,planes", [
    ((64, 256), None),
    ((256, 64), None),
    ((480, 640), [0, 1, 6, 13, 21, 29, 37, 45, 53, 60]),
    ((768, 1024), [0, 3, 20, 29, 45, 61, 64, 93, 100, 124]),
])
def test_spacing_matches_oracle(ffst, spacing, shape, planes):
    rows, cols = shape
    plan = ffst.Plan(rows, cols, spacing=spacing)
    j0 = plan.scales
    todo = range(plan.num_planes) if planes is None else planes
    psi = plan.spectra()
    for i in todo:
        ref = o.spectrum(rows, cols, j0, i, spacing=spacing)
        assert np.abs(psi[i].cpu().numpy() - ref).max() <= 1e-6, i
    del psi
    f = inputs.scaled_cartoon(rows, cols, seed=13)
    x = torch.from_numpy(f).cuda()
    c = plan.forward(x)
    F = np.fft.fft2(f.astype(np.float64))
    for i in todo:
        ref = o.forward_plane(F, j0, i, spacing=spacing)
        err = _plane_err(c[i].cpu().numpy(), ref, f)
        assert err <= TOL, (i, err)
    rec = plan.inverse(c)
    assert float(torch.linalg.norm(rec - x) / torch.linalg.norm(x)) <= TOL
    plan.close()


def test_readings_differ_on_gpu(ffst):
    # the two steps give different coefficients for a non-square image (and
    # the same for a square one)
    f = inputs.scaled_cartoon(128, 256, seed=14)
    x = torch.from_numpy(f).cuda()
    a = ffst.Plan(128, 256).forward(x)
    b = ffst.Plan(128, 256, spacing="per_axis").forward(x)
    assert float(torch.linalg.norm(a - b) / torch.linalg.norm(a)) > 1e-2
    g = inputs.scaled_cartoon(128, 128, seed=14)
    y = torch.from_numpy(g).cuda()
    assert torch.equal(ffst.Plan(128, 128).forward(y), ffst.Plan(128, 128, spacing="per_axis").forward(y))
