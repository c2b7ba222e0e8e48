"""Batched transforms over uneven sizes, CUDA-graph replay and the autotuner.

Every batched result must equal (bitwise) the same image through its own
single plan: the batch only schedules the same kernels on several streams.
"""

import os

import numpy as np
import pytest

from oracle import ffst_oracle as o
from paper_1202_1773_gb300 import inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

SIZES = [(128, 128), (256, 256), (480, 640), (512, 512), (768, 1024), (1024, 1024)]


@pytest.fixture(scope="module")
def ffst():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1202_1773_gb300 as pkg
    from paper_1202_1773_gb300 import build

    build.build()
    return pkg


def _batch(n, seed):
    shapes = inputs.batch_sizes(n, seed=seed)
    imgs = [torch.from_numpy(inputs.scaled_cartoon(r, c, seed=100 + i)).cuda() for i, (r, c) in enumerate(shapes)]
    return shapes, imgs


def test_batched_equals_single_plans(ffst):
    shapes, imgs = _batch(12, seed=2)
    bp = ffst.BatchPlan(shapes, lanes=4)
    assert sorted(set(bp.lanes())) == [0, 1, 2, 3]
    stacks = bp.forward(imgs)
    recs = bp.inverse(stacks)
    torch.cuda.synchronize()
    for i, (r, c) in enumerate(shapes):
        p = ffst.Plan(r, c)
        ref = p.forward(imgs[i])
        assert torch.equal(stacks[i], ref), i
        assert torch.equal(recs[i], p.inverse(ref)), i
        assert float(torch.linalg.norm(recs[i] - imgs[i]) / torch.linalg.norm(imgs[i])) <= 1e-5


def test_batched_parity_with_oracle_small(ffst):
    shapes = [(128, 128), (64, 64), (128, 256)]
    imgs = [inputs.scaled_cartoon(r, c, seed=5 + i) for i, (r, c) in enumerate(shapes)]
    bp = ffst.BatchPlan(shapes, lanes=2)
    stacks = bp.forward([torch.from_numpy(x).cuda() for x in imgs])
    for x, s in zip(imgs, stacks):
        ref = o.forward(x.astype(np.float64))
        assert np.linalg.norm(s.cpu().numpy() - ref) / np.linalg.norm(ref) <= 1e-5


@pytest.mark.parametrize("dtype", ["float32", "float16"])
def test_graph_replay_equals_eager(ffst, dtype):
    shapes, imgs = _batch(8, seed=3)
    tdt = getattr(torch, dtype)
    bp = ffst.BatchPlan(shapes, lanes=4)
    stacks = bp.empty_stacks(tdt)
    scales = [torch.empty(bp.shape(i)[0], device="cuda") for i in range(len(bp))] if dtype != "float32" else None
    outs = [torch.empty_like(x) for x in imgs]
    g = bp.capture(imgs, stacks, outs, what=3, plane_scales=scales)
    eager = bp.forward(imgs, dtype=tdt, plane_scales=[s.clone() for s in scales] if scales else None)
    eager_stacks = eager[0] if scales else eager
    eager_scales = eager[1] if scales else None
    eager_rec = bp.inverse(eager_stacks, plane_scales=eager_scales)
    for _ in range(2):  # new inputs written into the captured buffers, replayed twice
        for x in imgs:
            x.mul_(0.5)
        g.launch()
        torch.cuda.synchronize()
    eager = bp.forward(imgs, dtype=tdt, plane_scales=eager_scales)
    eager_stacks = eager[0] if scales else eager
    eager_rec = bp.inverse(eager_stacks, plane_scales=eager_scales)
    torch.cuda.synchronize()
    for i in range(len(bp)):
        assert torch.equal(stacks[i], eager_stacks[i]), i
        assert torch.equal(outs[i], eager_rec[i]), i
    g.close()


def test_autotune_round_trip(ffst, tmp_path):
    cache = tmp_path / "ffst_tune.txt"
    os.environ["FFST_AUTOTUNE_CACHE"] = str(cache)
    try:
        x = torch.from_numpy(inputs.scaled_cartoon(512, 512, seed=1)).cuda()
        p = ffst.Plan(512, 512)
        before = p.forward(x).clone()
        rec_before = p.inverse(before).clone()
        fmb, imb = p.autotune(reps=2)
        cands = (32.0, 64.0, 96.0, 128.0, 192.0)
        assert fmb in cands and imb in cands
        assert p.group_mb == (fmb, imb)
        ff, fi, rf, ri = p.kernels
        assert ff in (0, 1) and fi in (0, 1) and rf in (0, 1) and ri == 0  # 256-point rows: no variant 2
        assert 1 <= p.inverse_split <= 16
        after = p.forward(x)
        # budgets and fusion keep the arithmetic; row variants and plane chunks change rounding only
        assert float(torch.linalg.norm(after - before) / torch.linalg.norm(before)) <= 1e-6
        rec = p.inverse(after)
        assert float(torch.linalg.norm(rec - rec_before) / torch.linalg.norm(rec_before)) <= 1e-6
        text = cache.read_text().strip().splitlines()
        assert len(text) == 1 and " 512 512 4 0 " in text[0]
        fields = text[0].split()
        assert [float(fields[-7]), float(fields[-6])] == [fmb, imb]
        assert [int(v) for v in fields[-5:]] == [ff, rf, fi, ri, p.inverse_split]
        q = ffst.Plan(512, 512)  # picks the cached configuration up
        assert q.group_mb == (fmb, imb)
        assert q.kernels == p.kernels and q.inverse_split == p.inverse_split
    finally:
        del os.environ["FFST_AUTOTUNE_CACHE"]


def test_full_256_image_batch_against_oracle(ffst):
    # the batched workload: 256 images of uneven sizes (seed 2), two seeded
    # images per size, forward + inverse replayed from one captured graph;
    # every reconstruction within 1e-5 and, for the first image of each
    # distinct size, sampled planes against the FP64 oracle plane by plane
    # (relative to the plane's energy, floored at 1e-3 of the image's)
    n = 256
    shapes = inputs.batch_sizes(n, seed=2)
    srcs = {sh: [inputs.scaled_cartoon(*sh, seed=300 + q) for q in range(2)] for sh in sorted(set(shapes))}
    dev = {sh: [torch.from_numpy(x).cuda() for x in xs] for sh, xs in srcs.items()}
    imgs = [dev[sh][i % 2] for i, sh in enumerate(shapes)]
    bp = ffst.BatchPlan(shapes, lanes=4)
    stacks = bp.empty_stacks()
    outs = [torch.empty(sh, device="cuda") for sh in shapes]
    g = bp.capture(imgs, stacks, outs, what=3)
    g.launch()
    torch.cuda.synchronize()
    for i in range(n):
        err = float(torch.linalg.norm(outs[i] - imgs[i]) / torch.linalg.norm(imgs[i]))
        assert err <= 1e-5, (i, shapes[i], err)
    seen = set()
    for i, sh in enumerate(shapes):
        if sh in seen:
            continue
        seen.add(sh)
        f = srcs[sh][i % 2].astype(np.float64)
        F = np.fft.fft2(f)
        eta = bp.shape(i)[0]
        j0 = o.default_scales(*sh)
        for q in (0, eta // 3, eta - 1):
            ref = o.forward_plane(F, j0, q)
            got = stacks[i][q].cpu().numpy()
            err = np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-3 * np.linalg.norm(f))
            assert err <= 1e-5, (sh, q, err)
    assert len(seen) == len(SIZES)
    g.close()
    bp.close()


def test_batch_autotune_keeps_results(ffst):
    # tuning a batch picks a configuration per distinct shape; the results
    # stay those of the single plans to FP32 rounding (row variants and
    # plane chunks reorder sums) and graph replay still equals eager runs
    shapes, imgs = _batch(10, seed=4)
    bp = ffst.BatchPlan(shapes, lanes=3)
    bp.autotune(reps=1)
    stacks = bp.forward(imgs)
    recs = bp.inverse(stacks)
    torch.cuda.synchronize()
    for i, (r, c) in enumerate(shapes):
        ref = ffst.Plan(r, c).forward(imgs[i])
        assert float(torch.linalg.norm(stacks[i] - ref) / torch.linalg.norm(ref)) <= 1e-6, i
        assert float(torch.linalg.norm(recs[i] - imgs[i]) / torch.linalg.norm(imgs[i])) <= 1e-5, i
    outs = [torch.empty_like(x) for x in imgs]
    g_stacks = bp.empty_stacks()
    g = bp.capture(imgs, g_stacks, outs, what=3)
    g.launch()
    torch.cuda.synchronize()
    for i in range(len(shapes)):
        assert torch.equal(g_stacks[i], stacks[i]) and torch.equal(outs[i], recs[i]), i
    g.close()
    bp.close()
