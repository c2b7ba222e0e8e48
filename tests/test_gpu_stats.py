"""Fused per-plane statistics and shrinkage (ffst_forward_stats) against the oracle.

d(i) = 1/(MN) sum |c_i| (Sec. 3.5.2 eq. shearlet_meanvalue) and soft / hard
shrinkage of the coefficients in the row-pass epilogue, compared with the
FP64 oracle's forward, mean_abs and shrink.  Hard thresholding decides in
FP32 on the GPU and in FP64 in the oracle, so entries within a rounding band
of the threshold may go either way; they are checked to be one of the two
valid outcomes.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ffst():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_1202_1773_gb300 as m

    return m


def _case(shape, seed):
    from oracle import ffst_oracle as o
    from paper_1202_1773_gb300 import inputs

    f = inputs.scaled_cartoon(*shape, seed=seed)
    return f, o.forward(f.astype(np.float64)), o


@pytest.mark.parametrize("shape", [(64, 64), (256, 256), (128, 256)])
def test_mean_abs_matches_oracle(ffst, shape):
    f, c_ref, o = _case(shape, 21)
    p = ffst.Plan(*shape)
    c, d = p.forward_stats(torch.from_numpy(f).cuda())
    d_ref = o.mean_abs(c_ref)
    np.testing.assert_allclose(d.cpu().numpy(), d_ref, rtol=1e-5, atol=1e-7 * np.abs(d_ref).max())
    # the stack itself is the plain forward's
    assert torch.equal(c, p.forward(torch.from_numpy(f).cuda()))
    p.close()


@pytest.mark.parametrize("mode", ["soft", "hard"])
def test_shrinkage_matches_oracle(ffst, mode):
    shape = (256, 256)
    f, c_ref, o = _case(shape, 22)
    p = ffst.Plan(*shape)
    rng = np.random.default_rng(3)
    tau = (0.5 + rng.random(p.num_planes)) * o.mean_abs(c_ref)  # around each plane's mean |c|
    tau[0] = 0.0  # low-pass untouched
    c, d = p.forward_stats(torch.from_numpy(f).cuda(), shrink=mode,
                           thresh=torch.tensor(tau, dtype=torch.float32, device="cuda"))
    got = c.cpu().numpy().astype(np.float64)
    want = o.shrink(c_ref, tau, mode)
    scale = np.abs(c_ref).max()
    tau_b = np.broadcast_to(tau.reshape(-1, 1, 1), c_ref.shape)
    near = np.abs(np.abs(c_ref) - tau_b) <= 1e-5 * scale  # rounding band around the threshold
    err = np.abs(got - want)
    assert np.all(err[~near] <= 2e-5 * scale), float(err[~near].max())
    if mode == "hard":  # inside the band: kept (c) or dropped (0)
        ok = (np.abs(got - c_ref) <= 2e-5 * scale) | (got == 0.0)
        assert np.all(ok[near])
    np.testing.assert_allclose(d.cpu().numpy(), o.mean_abs(c_ref), rtol=1e-5, atol=1e-7 * scale)
    p.close()


def test_low_precision_storage_thresholds_in_coefficient_units(ffst):
    shape = (256, 256)
    f, c_ref, o = _case(shape, 23)
    p = ffst.Plan(*shape)
    tau = np.full(p.num_planes, float(o.mean_abs(c_ref)[1:].mean()))
    th = torch.tensor(tau, dtype=torch.float32, device="cuda")
    c16, d16, s16 = p.forward_stats(torch.from_numpy(f).cuda(), shrink="soft", thresh=th, dtype=torch.float16)
    c32, d32 = p.forward_stats(torch.from_numpy(f).cuda(), shrink="soft", thresh=th)
    got = (c16.float() / s16.view(-1, 1, 1)).cpu().numpy()
    ref = c32.cpu().numpy()
    assert np.linalg.norm(got - ref) <= 2e-3 * np.linalg.norm(ref)
    np.testing.assert_allclose(d16.cpu().numpy(), d32.cpu().numpy(), rtol=1e-5)
    p.close()


def test_stats_arguments(ffst):
    p = ffst.Plan(64, 64)
    x = torch.zeros(64, 64, device="cuda")
    with pytest.raises(ValueError):
        p.forward_stats(x, shrink="median", thresh=1.0)
    with pytest.raises(ValueError):
        p.forward_stats(x, shrink="soft")
    from paper_1202_1773_gb300 import _lib

    out = torch.empty(p.shape, device="cuda")
    assert _lib.lib().ffst_forward_stats(p.handle, x.data_ptr(), out.data_ptr(), 0, None, 3, None, None, None) \
        == _lib.FFST_ERR_INVALID_ARG
    assert _lib.lib().ffst_forward_stats(p.handle, x.data_ptr(), out.data_ptr(), 0, None, 1, None, None, None) \
        == _lib.FFST_ERR_INVALID_ARG
    p.close()
