"""Construction options of ffst_plan_ex against the FP64 oracle: smooth
shearlets (Sec. 3.4), variants of v (Sec. 2.1, Sec. 3.4 remark
construction_v) and the grid extent maxScale (Sec. 3.5.1, Sec. 3.5.3).

Same bars as the classic construction: spectra 1e-6 absolute, coefficient
stack and reconstruction 1e-5 relative L2, Parseval frame on the GPU.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

SHAPES = [(64, 64, 3), (256, 256, 4), (128, 256, 4), (480, 640, 4)]


@pytest.fixture(scope="module")
def ffst():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_1202_1773_gb300 as m

    return m


@pytest.mark.parametrize("rows,cols,scales", SHAPES)
def test_smooth_spectra_match_oracle(ffst, rows, cols, scales):
    from oracle import ffst_oracle as o

    p = ffst.Plan(rows, cols, scales, smooth=True)
    psi = p.spectra().cpu().numpy().astype(np.float64)
    ref = o.spectra(rows, cols, scales, smooth=True)
    assert np.abs(psi - ref).max() <= 1e-6
    # different from the classic construction (low-pass and radial factors)
    q = ffst.Plan(rows, cols, scales)
    assert np.abs(q.spectra().cpu().numpy() - psi).max() > 1e-2
    p.close()
    q.close()


@pytest.mark.parametrize("rows,cols,scales", SHAPES)
def test_smooth_transform_matches_oracle(ffst, rows, cols, scales):
    from oracle import ffst_oracle as o
    from paper_1202_1773_gb300 import inputs

    f = inputs.scaled_cartoon(rows, cols, seed=31)
    p = ffst.Plan(rows, cols, scales, smooth=True)
    x = torch.from_numpy(f).cuda()
    c = p.forward(x)
    ref = o.forward(f.astype(np.float64), scales, smooth=True)
    err = np.linalg.norm(c.cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err <= 1e-5, err
    r = p.inverse(c)
    assert float(torch.linalg.norm(r - x) / torch.linalg.norm(x)) <= 1e-5
    # Parseval frame on the GPU: adjoint == inverse, energy preserved
    a = p.adjoint(c)
    assert float(torch.linalg.norm(a - r) / torch.linalg.norm(r)) <= 1e-5
    e = float((c.double() ** 2).sum() / (x.double() ** 2).sum())
    assert abs(e - 1.0) <= 1e-5
    p.close()


def test_smooth_stats_and_low_precision(ffst):
    from oracle import ffst_oracle as o
    from paper_1202_1773_gb300 import inputs

    f = inputs.scaled_cartoon(256, 256, seed=32)
    p = ffst.Plan(256, 256, 4, smooth=True)
    x = torch.from_numpy(f).cuda()
    c, d = p.forward_stats(x)
    ref = o.forward(f.astype(np.float64), 4, smooth=True)
    np.testing.assert_allclose(d.cpu().numpy(), o.mean_abs(ref), rtol=1e-5, atol=1e-7 * np.abs(ref).max())
    c16, s16 = p.forward(x, dtype=torch.float16)
    err = float(torch.linalg.norm(c16.float() / s16.view(-1, 1, 1) - c) / torch.linalg.norm(c))
    assert err <= 2e-3
    p.close()


def test_option_codes_checked(ffst):
    from paper_1202_1773_gb300 import _lib
    import ctypes

    out = ctypes.c_void_p()
    for args in ((7, 0, 0, 0, 0), (0, 9, 0, 0, 0), (0, 2, 0, 0, 0), (0, 2, 8, 0, 0), (0, 0, 0, 3, 0),
                 (0, 0, 0, 0, 2)):
        assert _lib.lib().ffst_plan_ex(64, 64, 0, *args, ctypes.byref(out)) == _lib.FFST_ERR_INVALID_ARG
        assert out.value is None
    with pytest.raises(ValueError):
        ffst.Plan(64, 64, vfun="cubic")
    with pytest.raises(ValueError):
        ffst.Plan(64, 64, max_scale="mid")
    with pytest.raises(ValueError):
        ffst.Plan(64, 64, spacing="isotropic")


OPTIONS = [
    dict(vfun="quadratic"), dict(vfun=("poly", 1)), dict(vfun=("poly", 5)), dict(vfun="cinf"),
    dict(max_scale="min"), dict(smooth=True, vfun="cinf", max_scale="min"),
    dict(spacing="per_axis"), dict(smooth=True, spacing="per_axis"),
]
ORACLE_KW = lambda kw: dict(smooth=kw.get("smooth", False), vfun=kw.get("vfun", "meyer"),
                            max_scale=kw.get("max_scale", "max"), spacing=kw.get("spacing", "common"))


@pytest.mark.parametrize("kw", OPTIONS, ids=lambda kw: "-".join(f"{k}={v}" for k, v in kw.items()))
@pytest.mark.parametrize("rows,cols,scales", [(64, 64, 3), (128, 256, 4)])
def test_plan_options_match_oracle(ffst, kw, rows, cols, scales):
    from oracle import ffst_oracle as o
    from paper_1202_1773_gb300 import inputs

    p = ffst.Plan(rows, cols, scales, **kw)
    psi = p.spectra().cpu().numpy().astype(np.float64)
    assert np.abs(psi - o.spectra(rows, cols, scales, **ORACLE_KW(kw))).max() <= 2e-6
    f = inputs.scaled_cartoon(rows, cols, seed=33)
    x = torch.from_numpy(f).cuda()
    c = p.forward(x)
    ref = o.forward(f.astype(np.float64), scales, **ORACLE_KW(kw))
    assert np.linalg.norm(c.cpu().numpy() - ref) <= 1e-5 * np.linalg.norm(ref)
    r = p.inverse(c)
    assert float(torch.linalg.norm(r - x) / torch.linalg.norm(x)) <= 1e-5
    p.close()
