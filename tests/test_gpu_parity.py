"""GPU parity: libffst (through the C ABI) against the FP64 oracle.

Tolerances (relative L2 over the compared arrays):
* spectra: max abs <= 1e-6 (FP32 generation of values in [0, 1]);
* FP32 forward / inverse / adjoint: <= 1e-5;
* FP16 storage <= 2e-3, BF16 storage <= 1e-2 (coefficients and reconstruction).
"""

import numpy as np
import pytest

from oracle import ffst_oracle as o
from paper_1202_1773_gb300 import inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)


@pytest.fixture(scope="module")
def ffst():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1202_1773_gb300 as pkg
    from paper_1202_1773_gb300 import build

    build.build()
    return pkg


def _img(rows, cols, seed=0):
    if (rows, cols) == (64, 64):
        return inputs.small_cartoon(seed).astype(np.float32)
    return inputs.scaled_cartoon(rows, cols, seed)


SHAPES = [(8, 8), (16, 16), (64, 64), (128, 128), (64, 256), (256, 64), (32, 512), (512, 512)]


@pytest.mark.parametrize("shape", [(8, 8), (16, 16), (64, 64), (64, 256), (256, 64), (128, 32)])
def test_spectra_match_oracle(ffst, shape):
    plan = ffst.Plan(*shape)
    psi = plan.spectra().cpu().numpy()
    ref = o.spectra(*shape)
    assert psi.shape == ref.shape
    assert np.abs(psi - ref).max() <= 1e-6
    # the plane table matches the oracle's index order
    assert plan.plane_table() == [tuple(t) for t in o.plane_table(plan.scales)]


@pytest.mark.parametrize("shape", SHAPES)
def test_forward_matches_oracle(ffst, shape):
    f = _img(*shape, seed=3)
    plan = ffst.Plan(*shape)
    c = plan.forward(torch.from_numpy(f).cuda())
    torch.cuda.synchronize()
    c = c.cpu().numpy()
    ref = o.forward(f.astype(np.float64))
    assert rel_l2(c, ref) <= FP32_TOL
    # every plane relative to its own energy, floored at 1e-3 of the image's
    # (a plane that carries almost none is compared at that scale)
    floor = 1e-3 * np.linalg.norm(f.astype(np.float64))
    err = np.linalg.norm((c - ref).reshape(c.shape[0], -1), axis=1)
    per_plane = err / np.maximum(np.linalg.norm(ref.reshape(ref.shape[0], -1), axis=1), floor)
    assert per_plane.max() <= FP32_TOL, (int(per_plane.argmax()), float(per_plane.max()))


@pytest.mark.parametrize("shape", SHAPES)
def test_inverse_and_adjoint_match_oracle(ffst, shape):
    rng = np.random.default_rng(5)
    eta = o.num_planes(o.default_scales(*shape))
    cnp = rng.standard_normal((eta,) + shape).astype(np.float32)
    plan = ffst.Plan(*shape)
    c = torch.from_numpy(cnp).cuda()
    inv = plan.inverse(c).cpu().numpy()
    adj = plan.adjoint(c).cpu().numpy()
    assert rel_l2(adj, o.adjoint(cnp.astype(np.float64))) <= FP32_TOL
    assert rel_l2(inv, o.inverse(cnp.astype(np.float64))) <= FP32_TOL


@pytest.mark.parametrize("shape", SHAPES)
def test_perfect_reconstruction(ffst, shape):
    f = _img(*shape, seed=9)
    plan = ffst.Plan(*shape)
    x = torch.from_numpy(f).cuda()
    rec = plan.inverse(plan.forward(x)).cpu().numpy()
    assert rel_l2(rec, f) <= FP32_TOL
    adj = plan.adjoint(plan.forward(x)).cpu().numpy()
    assert rel_l2(adj, f) <= FP32_TOL


def test_dot_product_adjoint(ffst):
    shape = (128, 256)
    rng = np.random.default_rng(21)
    plan = ffst.Plan(*shape)
    x = torch.from_numpy(rng.standard_normal(shape).astype(np.float32)).cuda()
    c = torch.from_numpy(rng.standard_normal(plan.shape).astype(np.float32)).cuda()
    lhs = float((plan.forward(x).double() * c.double()).sum())
    rhs = float((x.double() * plan.adjoint(c).double()).sum())
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def test_parseval_gpu(ffst):
    shape = (256, 256)
    f = _img(*shape, seed=2)
    plan = ffst.Plan(*shape)
    c = plan.forward(torch.from_numpy(f).cuda()).double()
    ratio = float((c**2).sum()) / float((torch.from_numpy(f).double() ** 2).sum())
    assert abs(ratio - 1.0) <= 2e-5


@pytest.mark.parametrize("dtype,tol", [("float16", 2e-3), ("bfloat16", 1e-2)])
@pytest.mark.parametrize("shape", [(64, 64), (512, 512), (128, 256)])
def test_low_precision_storage(ffst, dtype, tol, shape):
    f = _img(*shape, seed=4)
    plan = ffst.Plan(*shape)
    x = torch.from_numpy(f).cuda()
    tdt = getattr(torch, dtype)
    c, s = plan.forward(x, dtype=tdt)
    assert c.dtype == tdt
    sc = s.cpu().numpy()
    assert np.all(sc > 0) and np.all(np.log2(sc) == np.round(np.log2(sc)))  # powers of two
    cref = o.forward(f.astype(np.float64))
    deq = c.float().cpu().numpy() / sc[:, None, None]
    assert rel_l2(deq, cref) <= tol
    rec = plan.inverse(c, s).cpu().numpy()
    assert rel_l2(rec, f) <= tol
    if dtype == "float16":
        assert np.abs(c.float().cpu().numpy()).max() <= 32768.0


def test_repeat_calls_are_deterministic(ffst):
    shape = (256, 256)
    f = _img(*shape, seed=6)
    plan = ffst.Plan(*shape)
    x = torch.from_numpy(f).cuda()
    a = plan.forward(x).clone()
    b = plan.forward(x)
    assert torch.equal(a, b)
    r1 = plan.inverse(a).clone()
    r2 = plan.inverse(b)
    assert torch.equal(r1, r2)


@pytest.mark.parametrize("shape,planes", [((2048, 2048), [0, 1, 5, 13, 29, 45, 61, 93, 124]),
                                          ((1024, 2048), [0, 7, 60, 61, 124]),
                                          ((4096, 4096), [0, 125, 189, 252])])
def test_full_size_sampled_planes(ffst, shape, planes):
    # the bench workload and the largest size: sampled planes against the
    # oracle plane by plane, Parseval and reconstruction over the whole stack
    f = inputs.scaled_cartoon(*shape, seed=5)
    plan = ffst.Plan(*shape)
    x = torch.from_numpy(f).cuda()
    c = plan.forward(x)
    F = np.fft.fft2(f.astype(np.float64))
    for i in planes:
        ref = o.forward_plane(F, plan.scales, i)
        got = c[i].cpu().numpy()
        err = np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-3 * np.linalg.norm(f))
        assert err <= FP32_TOL, (i, err)
    energy = sum(float(torch.sum(c[i].double() ** 2)) for i in range(c.shape[0]))
    assert abs(energy / float(torch.sum(x.double() ** 2)) - 1.0) <= 2e-5
    rec = plan.inverse(c)
    assert float(torch.linalg.norm(rec - x) / torch.linalg.norm(x)) <= FP32_TOL


def test_errors_reported(ffst):
    from paper_1202_1773_gb300 import _lib

    with pytest.raises(ffst.FFSTError) as ei:
        ffst.Plan(2049, 64)  # no native line and above the generic lines' 2048
    assert ei.value.status == _lib.FFST_ERR_UNSUPPORTED_SIZE
    plan = ffst.Plan(64, 64)
    x = torch.zeros(64, 64, device="cuda")
    c = torch.empty(plan.shape, device="cuda")
    with pytest.raises(ffst.FFSTError) as ei:
        _lib.ffst_forward(plan.handle, x, c, 7, None, None)
    assert ei.value.status == _lib.FFST_ERR_INVALID_ARG
    with pytest.raises(ffst.FFSTError):
        _lib.ffst_forward(plan.handle, x, c.half(), _lib.FFST_STORE_F16, None, None)  # scales required
    with pytest.raises(ffst.FFSTError):
        _lib.ffst_plane_index(plan.handle, plan.num_planes)


# mixed-radix sizes (factors 3 and 5): the uneven sizes of the batched workload
@pytest.mark.parametrize("shape", [(240, 480), (480, 640), (640, 480), (320, 640), (384, 256), (64, 768)])
def test_mixed_radix_sizes_match_oracle(ffst, shape):
    f = _img(*shape, seed=11)
    plan = ffst.Plan(*shape)
    x = torch.from_numpy(f).cuda()
    c = plan.forward(x)
    ref = o.forward(f.astype(np.float64))
    assert rel_l2(c.cpu().numpy(), ref) <= FP32_TOL
    rec = plan.inverse(c).cpu().numpy()
    assert rel_l2(rec, f) <= FP32_TOL
    psi = plan.spectra().cpu().numpy()
    assert np.abs(psi - o.spectra(*shape)).max() <= 1e-6


def test_mixed_radix_768x1024_sampled(ffst):
    shape = (768, 1024)
    f = inputs.scaled_cartoon(*shape, seed=12)
    plan = ffst.Plan(*shape)
    x = torch.from_numpy(f).cuda()
    c = plan.forward(x)
    F = np.fft.fft2(f.astype(np.float64))
    for i in [0, 3, 20, 64, 100, 124]:
        ref = o.forward_plane(F, plan.scales, i)
        err = np.linalg.norm(c[i].cpu().numpy() - ref) / max(np.linalg.norm(ref), 1e-3 * np.linalg.norm(f))
        assert err <= FP32_TOL, (i, err)
    rec = plan.inverse(c)
    assert float(torch.linalg.norm(rec - x) / torch.linalg.norm(x)) <= FP32_TOL


@pytest.mark.parametrize("dtype,tol", [("float16", 2e-3), ("bfloat16", 1e-2)])
@pytest.mark.parametrize("shape,planes", [((2048, 2048), [0, 13, 61, 100, 124]),
                                          ((4096, 4096), [0, 61, 125, 200, 252])])
def test_low_precision_full_size_sampled_planes(ffst, dtype, tol, shape, planes):
    # the large low-precision workloads (2048^2 J=5, 4096^2 J=6 with 253
    # planes): dequantised sampled planes against the FP64 oracle, each
    # relative to its own energy (floored at 1e-3 of the image's), and the
    # reconstruction from the low-precision stack
    f = inputs.scaled_cartoon(*shape, seed=5)
    plan = ffst.Plan(*shape)
    x = torch.from_numpy(f).cuda()
    c, s = plan.forward(x, dtype=getattr(torch, dtype))
    sc = s.cpu().numpy()
    F = np.fft.fft2(f.astype(np.float64))
    floor = 1e-3 * np.linalg.norm(f)
    for i in planes:
        ref = o.forward_plane(F, plan.scales, i)
        got = c[i].float().cpu().numpy() / sc[i]
        err = np.linalg.norm(got - ref) / max(np.linalg.norm(ref), floor)
        assert err <= tol, (i, err)
    rec = plan.inverse(c, s)
    assert float(torch.linalg.norm(rec - x) / torch.linalg.norm(x)) <= tol
    del c, rec
    plan.close()
