"""The differentiable transform: backward = hand-written adjoint, checked
against central finite differences of the FP64 oracle and the oracle's
adjoint; double backward; the shearlet-l1 deconvolution against an FP64
run of the same iteration."""

import numpy as np
import pytest

from oracle import deconv_oracle as do
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
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("shape", [(64, 64), (128, 256)])
def test_backward_is_the_adjoint(ffst, shape):
    rng = np.random.default_rng(31)
    plan = ffst.Plan(*shape)
    x = torch.from_numpy(inputs.scaled_cartoon(*shape, seed=7)).cuda().requires_grad_(True)
    w = torch.from_numpy(rng.standard_normal(plan.shape).astype(np.float32)).cuda()
    (ffst.shearlet_transform(x, plan) * w).sum().backward()
    g = x.grad.detach()
    assert torch.equal(g, plan.adjoint(w))  # the backward pass is ffst_adjoint
    assert _rel(g.cpu().numpy(), o.adjoint(w.cpu().numpy().astype(np.float64))) <= 1e-5


@pytest.mark.parametrize("shape", [(64, 64), (32, 64)])
def test_gradient_against_central_differences(ffst, shape):
    # L(x) = <w, T x>; central differences (h = 1e-3) of the FP64 oracle
    # forward along 64 seeded directions against <GPU gradient, d>
    rng = np.random.default_rng(5)
    plan = ffst.Plan(*shape)
    x0 = inputs.scaled_cartoon(*shape, seed=1).astype(np.float64)
    w = rng.standard_normal(plan.shape)
    xt = torch.from_numpy(x0.astype(np.float32)).cuda().requires_grad_(True)
    (ffst.shearlet_transform(xt, plan) * torch.from_numpy(w.astype(np.float32)).cuda()).sum().backward()
    grad = xt.grad.double().cpu().numpy()
    h = 1e-3
    fd, an = [], []
    for _ in range(64):
        d = rng.standard_normal(shape)
        lp = np.sum(w * o.forward(x0 + h * d))
        lm = np.sum(w * o.forward(x0 - h * d))
        fd.append((lp - lm) / (2 * h))
        an.append(np.sum(grad * d))
    fd, an = np.array(fd), np.array(an)
    assert np.max(np.abs(fd - an)) <= 1e-5 * np.max(np.abs(fd))


def test_double_backward(ffst):
    # d/dw <grad_x <w, T x>, v> = T v: the backward of the backward is the forward
    shape = (64, 128)
    rng = np.random.default_rng(8)
    plan = ffst.Plan(*shape)
    x = torch.from_numpy(rng.standard_normal(shape).astype(np.float32)).cuda().requires_grad_(True)
    w = torch.from_numpy(rng.standard_normal(plan.shape).astype(np.float32)).cuda().requires_grad_(True)
    v = torch.from_numpy(rng.standard_normal(shape).astype(np.float32)).cuda()
    L = (ffst.shearlet_transform(x, plan) * w).sum()
    (g,) = torch.autograd.grad(L, x, create_graph=True)
    (g * v).sum().backward()
    assert torch.allclose(w.grad, plan.forward(v), rtol=0, atol=1e-6)


def test_deconvolution_matches_fp64_iteration(ffst):
    from paper_1202_1773_gb300 import deconv

    shape = (64, 64)
    lam, eps, steps = 5e-3, 1e-3, 30
    truth = inputs.small_cartoon(0)
    psf = deconv.gaussian_psf(*shape, sigma=2.0, radius=8)
    rng = np.random.default_rng(12)
    y = do.blur(truth, psf) + rng.normal(0.0, 0.02, shape)
    plan = ffst.Plan(*shape)
    blur = deconv.Blur(psf, "cuda")
    yt = torch.from_numpy(y.astype(np.float32)).cuda()
    x, hist = deconv.deconvolve(yt, plan, blur, lam=lam, eps=eps, steps=steps)
    xr, hr = do.deconvolve(y.astype(np.float32).astype(np.float64), psf, lam, eps, steps)
    assert _rel(x.cpu().numpy(), xr) <= 1e-4
    assert abs(hist[-1] - hr[-1]) <= 1e-4 * abs(hr[-1])
    # the objective goes down and the restoration is closer to the truth than y
    assert hist[-1] < 0.95 * hist[0]
    assert np.linalg.norm(x.cpu().numpy() - truth) < np.linalg.norm(y - truth)


def test_deconvolution_200_steps_128(ffst):
    # the full 200-step iteration on a 128x128 problem (J=3) against the FP64
    # run of the same iteration: final iterate and objective within 1e-4
    from paper_1202_1773_gb300 import deconv

    shape = (128, 128)
    lam, eps, steps = 5e-3, 1e-3, 200
    truth = inputs.scaled_cartoon(*shape, seed=16, sigma=0.0).astype(np.float64)
    psf = deconv.gaussian_psf(*shape, sigma=2.0, radius=8)
    rng = np.random.default_rng(17)
    y = (do.blur(truth, psf) + rng.normal(0.0, 0.02, shape)).astype(np.float32)
    plan = ffst.Plan(*shape)
    x, hist = deconv.deconvolve(torch.from_numpy(y).cuda(), plan, deconv.Blur(psf, "cuda"), lam=lam, eps=eps,
                                steps=steps)
    xr, hr = do.deconvolve(y.astype(np.float64), psf, lam, eps, steps)
    assert _rel(x.cpu().numpy(), xr) <= 1e-4
    assert abs(hist[-1] - hr[-1]) <= 1e-4 * abs(hr[-1])
    # the objective went down (FISTA is not monotone step by step) and the
    # restoration is closer to the truth than y
    assert hist[-1] < 0.95 * hist[0]
    assert np.linalg.norm(x.cpu().numpy() - truth) < np.linalg.norm(y - truth)


def test_deconvolution_1024_first_steps(ffst):
    # the 1024x1024 J=5 workload: the first 5 iterations (autograd through
    # ffst_forward / ffst_adjoint) against the FP64 run of the same iteration,
    # and the first gradient on its own
    from paper_1202_1773_gb300 import deconv

    shape = (1024, 1024)
    lam, eps, steps = 5e-3, 1e-3, 5
    truth = inputs.scaled_cartoon(*shape, seed=4, sigma=0.0).astype(np.float64)
    psf = deconv.gaussian_psf(*shape)
    rng = np.random.default_rng(13)
    y = (do.blur(truth, psf) + rng.normal(0.0, 0.02, shape)).astype(np.float32)
    plan = ffst.Plan(*shape)
    yt = torch.from_numpy(y).cuda()
    blur = deconv.Blur(psf, "cuda")
    x = yt.clone().requires_grad_(True)
    J = deconv.objective(x, yt, blur, plan, lam, eps)
    (g,) = torch.autograd.grad(J, x)
    y64 = y.astype(np.float64)
    psi = o.spectra(*shape)
    gr = do.gradient(y64, y64, psf, lam, eps, psi)
    assert _rel(g.cpu().numpy(), gr) <= 1e-4
    Jv = float(J.detach())
    assert abs(Jv - do.objective(y64, y64, psf, lam, eps, psi)) <= 1e-4 * abs(Jv)
    del psi
    xg, hist = deconv.deconvolve(yt, plan, blur, lam=lam, eps=eps, steps=steps)
    xr, hr = do.deconvolve(y64, psf, lam, eps, steps)
    assert _rel(xg.cpu().numpy(), xr) <= 1e-4
    for a, b in zip(hist, hr):
        assert abs(a - b) <= 1e-4 * abs(b)
