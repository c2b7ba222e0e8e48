"""Generic sizes (odd, prime, and lengths without a native FFT line) against
the FP64 oracle.

A dimension whose length has no native line runs generic lines: lengths
with no prime factor above 7 as mixed-radix (2, 3, 4, 5, 7, 8) Stockham
passes in shared memory, the others as Bluestein lines (the DFT of length n
as a chirp convolution through power-of-two FFTs of length L2 >= 2n - 1;
FFST_BLUESTEIN=1 at plan creation forces them for every length).
Everything after the line transforms (the Sec. 3.1 forward,
the Sec. 3.3 inverse and adjoint, low-precision storage, the fused
statistics and shrinkage, the one-sided complex shearlets of Sec. 3.8.2,
the plane chunks of the inverse) is the same code as at native sizes, so the
cases mix generic rows, generic columns and both.  Tolerances as in
test_gpu_parity (relative L2): FP32 1e-5, FP16 2e-3, BF16 1e-2.
"""

import numpy as np
import pytest

from oracle import ffst_oracle as o
from paper_1202_1773_gb300 import inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5

# (rows, cols): both generic, generic columns only, generic rows only,
# primes, odd x even, the smallest size, and a mixed-radix native height
SHAPES = [(8, 9), (15, 17), (63, 64), (64, 63), (100, 150), (131, 137), (127, 256), (256, 255), (240, 250),
          (97, 480)]


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module")
def ffst():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_1202_1773_gb300 as m

    return m


def _img(shape, seed):
    return inputs.scaled_cartoon(*shape, seed=seed)


@pytest.mark.parametrize("shape", SHAPES)
def test_forward_matches_oracle(ffst, shape):
    f = _img(shape, 3)
    p = ffst.Plan(*shape)
    c = p.forward(torch.from_numpy(f).cuda()).cpu().numpy()
    ref = o.forward(f.astype(np.float64))
    assert c.shape == ref.shape
    assert rel_l2(c, ref) <= FP32_TOL
    p.close()


@pytest.mark.parametrize("shape", SHAPES)
def test_inverse_and_adjoint_match_oracle(ffst, shape):
    eta = o.num_planes(o.default_scales(*shape))
    cnp = np.random.default_rng(shape[0] * 7 + shape[1]).standard_normal((eta,) + shape).astype(np.float32)
    p = ffst.Plan(*shape)
    c = torch.from_numpy(cnp).cuda()
    assert rel_l2(p.inverse(c).cpu().numpy(), o.inverse(cnp.astype(np.float64))) <= FP32_TOL
    assert rel_l2(p.adjoint(c).cpu().numpy(), o.adjoint(cnp.astype(np.float64))) <= FP32_TOL
    p.close()


@pytest.mark.parametrize("shape", [(15, 17), (131, 137), (256, 255)])
def test_reconstruction_and_parseval(ffst, shape):
    f = _img(shape, 9)
    p = ffst.Plan(*shape)
    x = torch.from_numpy(f).cuda()
    c = p.forward(x)
    assert float(torch.linalg.norm(p.inverse(c) - x) / torch.linalg.norm(x)) <= FP32_TOL
    assert float(torch.linalg.norm(p.adjoint(c) - x) / torch.linalg.norm(x)) <= FP32_TOL
    # Parseval frame: sum_i ||c_i||^2 = ||f||^2
    assert abs(float(torch.sum(c.double() ** 2)) / float(torch.sum(x.double() ** 2)) - 1.0) <= 2e-5
    p.close()


@pytest.mark.parametrize("dtype,tol", [("f16", 2e-3), ("bf16", 1e-2)])
def test_low_precision_storage(ffst, dtype, tol):
    shape = (131, 137)
    f = _img(shape, 4)
    p = ffst.Plan(*shape)
    x = torch.from_numpy(f).cuda()
    dt = torch.float16 if dtype == "f16" else torch.bfloat16
    c, sc = p.forward(x, dtype=dt)
    got = (c.float() / sc.view(-1, 1, 1)).cpu().numpy()
    ref = o.forward(f.astype(np.float64))
    assert rel_l2(got, ref) <= tol
    assert rel_l2(p.inverse(c, plane_scale=sc).cpu().numpy(), f) <= tol
    p.close()


def test_stats_and_shrinkage(ffst):
    shape = (127, 129)
    f = _img(shape, 21)
    c_ref = o.forward(f.astype(np.float64))
    p = ffst.Plan(*shape)
    x = torch.from_numpy(f).cuda()
    c, d = p.forward_stats(x)
    d_ref = o.mean_abs(c_ref)
    np.testing.assert_allclose(d.cpu().numpy(), d_ref, rtol=1e-5, atol=1e-7 * np.abs(d_ref).max())
    assert torch.equal(c, p.forward(x))
    tau = 0.8 * d_ref
    tau[0] = 0.0
    cs, _ = p.forward_stats(x, shrink="soft", thresh=torch.tensor(tau, dtype=torch.float32, device="cuda"))
    want = o.shrink(c_ref, tau, "soft")
    assert np.abs(cs.cpu().numpy() - want).max() <= 1e-5 * np.abs(c_ref).max()
    p.close()


@pytest.mark.parametrize("shape", [(63, 65), (100, 150)])
def test_complex_matches_oracle(ffst, shape):
    f = _img(shape, 8)
    p = ffst.Plan(*shape)
    x = torch.from_numpy(f).cuda()
    z = p.forward_complex(x).cpu().numpy()
    ref = o.forward_onesided(f.astype(np.float64), p.scales)
    got = z[:, 0] + 1j * z[:, 1]
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= FP32_TOL
    r = p.inverse_complex(torch.from_numpy(z).cuda())
    assert float(torch.linalg.norm(r - x) / torch.linalg.norm(x)) <= FP32_TOL
    p.close()


def test_smooth_variant(ffst):
    shape = (99, 101)
    f = _img(shape, 2)
    p = ffst.Plan(*shape, smooth=True)
    c = p.forward(torch.from_numpy(f).cuda()).cpu().numpy()
    assert rel_l2(c, o.forward(f.astype(np.float64), smooth=True)) <= FP32_TOL
    p.close()


@pytest.mark.parametrize("nsplit", [1, 3, 16])
def test_inverse_chunks(ffst, nsplit):
    shape = (131, 137)
    eta = o.num_planes(o.default_scales(*shape))
    cnp = np.random.default_rng(nsplit).standard_normal((eta,) + shape).astype(np.float32)
    p = ffst.Plan(*shape)
    p.inverse_split = nsplit
    assert rel_l2(p.inverse(torch.from_numpy(cnp).cuda()).cpu().numpy(),
                  o.inverse(cnp.astype(np.float64))) <= FP32_TOL
    p.close()


@pytest.mark.parametrize("shape,planes", [((1023, 1025), [0, 1, 7, 30, 60]), ((2047, 2048), [0, 13, 61, 124]),
                                          ((1536, 2046), [0, 5, 62, 124])])
def test_large_generic_sampled_planes(ffst, shape, planes):
    # the largest generic lines (L2 = 4096): sampled planes against the oracle
    # plane by plane, Parseval and reconstruction over the whole stack
    f = _img(shape, 5)
    p = ffst.Plan(*shape)
    x = torch.from_numpy(f).cuda()
    c = p.forward(x)
    F = np.fft.fft2(f.astype(np.float64))
    for i in planes:
        ref = o.forward_plane(F, p.scales, i)
        got = c[i].cpu().numpy()
        err = np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-3 * np.linalg.norm(f))
        assert err <= FP32_TOL, (i, err)
    energy = float(torch.sum(c.double() ** 2))
    assert abs(energy / float(torch.sum(x.double() ** 2)) - 1.0) <= 2e-5
    rec = p.inverse(c)
    assert float(torch.linalg.norm(rec - x) / torch.linalg.norm(x)) <= FP32_TOL
    p.close()


@pytest.mark.parametrize("n", [257, 384, 480])
def test_square_sizes_without_fused_launches(ffst, n):
    # square sizes whose lines are generic (257) or mixed-radix (384, 480) run
    # the standalone passes; the fused launches are for powers of two only
    shape = (n, n)
    f = _img(shape, 12)
    p = ffst.Plan(*shape)
    x = torch.from_numpy(f).cuda()
    c = p.forward(x)
    assert rel_l2(c.cpu().numpy(), o.forward(f.astype(np.float64))) <= FP32_TOL
    assert float(torch.linalg.norm(p.inverse(c) - x) / torch.linalg.norm(x)) <= FP32_TOL
    p.schedule = 1  # no persistent schedule either
    assert p.schedule == 0
    p.close()


def test_odd_square_2047_sampled_planes(ffst):
    # the bench's odd-size form: Bluestein lines of L2 = 4096 in both dimensions
    shape = (2047, 2047)
    f = _img(shape, 5)
    p = ffst.Plan(*shape)
    x = torch.from_numpy(f).cuda()
    c = p.forward(x)
    F = np.fft.fft2(f.astype(np.float64))
    for i in (0, 2, 62, 124):
        ref = o.forward_plane(F, p.scales, i)
        err = np.linalg.norm(c[i].cpu().numpy() - ref) / max(np.linalg.norm(ref), 1e-3 * np.linalg.norm(f))
        assert err <= FP32_TOL, (i, err)
    assert float(torch.linalg.norm(p.inverse(c) - x) / torch.linalg.norm(x)) <= FP32_TOL
    p.close()


def test_deterministic(ffst):
    shape = (255, 257)
    x = torch.from_numpy(_img(shape, 1)).cuda()
    p = ffst.Plan(*shape)
    c0 = p.forward(x).clone()
    r0 = p.inverse(c0).clone()
    for _ in range(2):
        assert torch.equal(p.forward(x), c0)
        assert torch.equal(p.inverse(c0), r0)
    p.close()


def test_batched_and_graph_at_generic_sizes(ffst):
    # uneven batches mixing native and generic sizes over lane streams, eager
    # and replayed from one CUDA graph, against single plans bit for bit
    shapes = [(63, 65), (100, 150), (64, 64), (131, 137), (63, 65), (256, 255)]
    imgs = [torch.from_numpy(_img(sh, 40 + i)).cuda() for i, sh in enumerate(shapes)]
    bp = ffst.BatchPlan(shapes, lanes=3)
    stacks = bp.forward(imgs)
    recs = bp.inverse(stacks)
    torch.cuda.synchronize()
    for i, sh in enumerate(shapes):
        p = ffst.Plan(*sh)
        ref = p.forward(imgs[i])
        assert torch.equal(stacks[i], ref), i
        assert torch.equal(recs[i], p.inverse(ref)), i
        p.close()
    gst = bp.empty_stacks()
    outs = [torch.empty_like(x) for x in imgs]
    g = bp.capture(imgs, gst, outs, what=3)
    g.launch()
    torch.cuda.synchronize()
    for i in range(len(bp)):
        assert torch.equal(gst[i], stacks[i]), i
        assert torch.equal(outs[i], recs[i]), i
    g.close()
    bp.close()


@pytest.mark.parametrize("shape", [(100, 150), (63, 64), (240, 250), (98, 343), (36, 1000)])
def test_smooth_lines_against_bluestein_and_oracle(ffst, shape, monkeypatch):
    # 100, 150, 63, 250, 98, 343, 36 and 1000 have no prime factor above 7:
    # mixed-radix lines by default, Bluestein lines with FFST_BLUESTEIN=1;
    # both against the oracle, and not bitwise equal (two different engines)
    f = _img(shape, 5)
    x = torch.from_numpy(f).cuda()
    p = ffst.Plan(*shape)
    monkeypatch.setenv("FFST_BLUESTEIN", "1")
    q = ffst.Plan(*shape)
    monkeypatch.delenv("FFST_BLUESTEIN")
    ref = o.forward(f.astype(np.float64))
    cp, cq = p.forward(x), q.forward(x)
    assert rel_l2(cp.cpu().numpy(), ref) <= FP32_TOL
    assert rel_l2(cq.cpu().numpy(), ref) <= FP32_TOL
    assert not torch.equal(cp, cq)
    eta = p.num_planes
    cnp = np.random.default_rng(shape[0] + shape[1]).standard_normal((eta,) + shape).astype(np.float32)
    c = torch.from_numpy(cnp).cuda()
    assert rel_l2(p.inverse(c).cpu().numpy(), o.inverse(cnp.astype(np.float64))) <= FP32_TOL
    assert rel_l2(p.adjoint(c).cpu().numpy(), o.adjoint(cnp.astype(np.float64))) <= FP32_TOL
    c16, s16 = p.forward(x, dtype=torch.float16)
    assert rel_l2((c16.float() / s16.view(-1, 1, 1)).cpu().numpy(), ref) <= 2e-3
    p.close()
    q.close()


@pytest.mark.parametrize("shape,planes", [((1080, 1920), [0, 9, 40, 77, 124]), ((700, 1000), [0, 5, 33, 60]),
                                          ((2160, 3840), [0, 61, 124])])
def test_large_smooth_sampled_planes(ffst, shape, planes):
    # 1080 = 2^3 3^3 5 and 1920 = 2^7 3 5 (columns of 1080 points, rows of
    # 1920 points as generic lines), 700 = 2^2 5^2 7 and 1000 = 2^3 5^3,
    # 2160 = 2^4 3^3 5 and 3840 = 2^8 3 5 (smooth lines above 2048 points):
    # sampled planes against the oracle, each relative to the plane's energy
    # floored at 1e-3 of the image's, and the reconstruction
    f = _img(shape, 12)
    x = torch.from_numpy(f).cuda()
    p = ffst.Plan(*shape)
    c = p.forward(x)
    F = np.fft.fft2(f.astype(np.float64))
    for i in planes:
        ref = o.forward_plane(F, p.scales, i)
        got = c[i].cpu().numpy().astype(np.float64)
        err = np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-3 * np.linalg.norm(f))
        assert err <= FP32_TOL, (i, err)
    assert float(torch.linalg.norm(p.inverse(c) - x) / torch.linalg.norm(x)) <= FP32_TOL
    del c
    p.close()
