"""Kernel configurations of a plan (ffst_plan_set_kernels) against the oracle.

Fused or separate plane-pass launches, and for separate row launches every
row-FFT variant the width has (16 elements per thread; two rows per team in
packed FP32 pairs; 32 elements per thread with radix 32 x 32; the same with
its exchange by warp shuffles, bitwise equal to the shared-memory one), each checked
plane by plane against the FP64 oracle (relative to the plane's energy,
floored at 1e-3 of the image's), with the inverse, the fused per-plane
statistics and FP16 storage in every configuration.
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


def _configs(n):
    L = n // 2
    rows_fwd = [0] + ([1] if 256 <= L <= 2048 else []) + ([2] if L in (1024, 2048) else []) + ([3] if L == 1024 else [])
    rows_inv = [0] + ([2] if L in (1024, 2048) else []) + ([3] if L == 1024 else [])
    out = [(1, 1, 0, 0)]
    out += [(0, 0, rf, ri) for rf in rows_fwd for ri in rows_inv]
    return out


def _plane_err(got, ref, f):
    return np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-3 * np.linalg.norm(f))


@pytest.mark.parametrize("n,planes", [(512, None), (1024, [0, 7, 30, 61, 93, 124]),
                                      (2048, [0, 13, 61, 100, 124])])
def test_kernel_configs_match_oracle(ffst, n, planes):
    f = inputs.scaled_cartoon(n, n, seed=17)
    x = torch.from_numpy(f).cuda()
    p = ffst.Plan(n, n)
    F = np.fft.fft2(f.astype(np.float64))
    todo = range(p.num_planes) if planes is None else planes
    refs = {i: o.forward_plane(F, p.scales, i) for i in todo}
    dref = {i: float(np.abs(refs[i]).mean()) for i in todo}
    for cfg in _configs(n):
        p.set_kernels(*cfg)
        assert p.kernels == cfg
        c, d = p.forward_stats(x)
        for i in todo:
            err = _plane_err(c[i].cpu().numpy(), refs[i], f)
            assert err <= 1e-5, (cfg, i, err)
            assert abs(float(d[i]) - dref[i]) <= 1e-5 * max(dref[i], 1e-3 * float(np.abs(f).mean())), (cfg, i)
        rec = p.inverse(c)
        assert float(torch.linalg.norm(rec - x) / torch.linalg.norm(x)) <= 1e-5, cfg
        c16, s16 = p.forward(x, dtype=torch.float16)
        for i in list(todo)[:3]:
            err = _plane_err(c16[i].float().cpu().numpy() / float(s16[i]), refs[i], f)
            assert err <= 2e-3, (cfg, i, err)
        assert float(torch.linalg.norm(p.inverse(c16, s16) - x) / torch.linalg.norm(x)) <= 2e-3, cfg
        del c, c16
    p.close()


def test_shuffle_exchange_is_bitwise_shared_memory_exchange(ffst):
    # row variant 3 runs the radix 32 x 32 line of variant 2 with its one
    # exchange through warp shuffles: the same arithmetic, so the same bits
    f = inputs.scaled_cartoon(2048, 2048, seed=23)
    x = torch.from_numpy(f).cuda()
    p = ffst.Plan(2048, 2048)
    p.set_kernels(0, 0, 2, 2)
    c2 = p.forward(x)
    r2 = p.inverse(c2)
    p.set_kernels(0, 0, 3, 3)
    c3 = p.forward(x)
    r3 = p.inverse(c2)
    assert torch.equal(c2, c3)
    assert torch.equal(r2, r3)
    d = p.forward_stats(x)[1]
    p.set_kernels(0, 0, 2, 2)
    assert torch.equal(d, p.forward_stats(x)[1])
    del c2, c3
    p.close()


def test_kernel_config_checked(ffst):
    p = ffst.Plan(256, 256)  # rows of 128 points: only variant 0
    with pytest.raises(ffst.FFSTError):
        p.set_kernels(0, 0, 2, 0)
    with pytest.raises(ffst.FFSTError):
        p.set_kernels(0, 0, 0, 1)  # the paired rows are a forward (C2R) variant only
    with pytest.raises(ffst.FFSTError):
        p.set_kernels(2, 1, 0, 0)
    with pytest.raises(ffst.FFSTError):
        p.set_kernels(0, 0, 3, 0)  # the shuffle exchange exists for 1024-point rows only
    q = ffst.Plan(63, 65)  # generic rows: variant 0 only
    with pytest.raises(ffst.FFSTError):
        q.set_kernels(0, 0, 1, 0)
    p.close()
    q.close()
