"""Plane chunks of the inverse column pass (ffst_plan_set_inverse_split).

The inverse and the adjoint sum psi_hat_i times the planes' spectra over all
planes (Sec. 3.3); with nsplit chunks that sum runs as nsplit partial sums
added in chunk order.  Every split is checked against the FP64 oracle, the
splits against one another (same sum, other rounding order), and the parts
that must not move the result at all: the plane-group budgets and the
schedule mode, for a fixed split.
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
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module")
def ffst():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_1202_1773_gb300 as m

    return m


def _coeffs(shape, seed):
    eta = o.num_planes(o.default_scales(*shape))
    return np.random.default_rng(seed).standard_normal((eta,) + shape).astype(np.float32)


@pytest.mark.parametrize("shape", [(64, 64), (256, 256), (480, 640), (512, 512)])
@pytest.mark.parametrize("nsplit", [1, 2, 3, 16])
def test_split_matches_oracle(ffst, shape, nsplit):
    cnp = _coeffs(shape, seed=shape[0] + nsplit)
    p = ffst.Plan(*shape)
    p.inverse_split = nsplit
    assert p.inverse_split == nsplit
    c = torch.from_numpy(cnp).cuda()
    inv = p.inverse(c).cpu().numpy()
    adj = p.adjoint(c).cpu().numpy()
    assert rel_l2(inv, o.inverse(cnp.astype(np.float64))) <= FP32_TOL
    assert rel_l2(adj, o.adjoint(cnp.astype(np.float64))) <= FP32_TOL
    p.close()


def test_default_split_and_reset(ffst):
    big = ffst.Plan(2048, 2048)
    assert big.inverse_split == 1  # the column panels alone fill the GPU
    big.close()
    p = ffst.Plan(512, 512)
    d = p.inverse_split
    assert 2 <= d <= 16  # 33 panels of 8 columns: chunks add column blocks
    p.inverse_split = 1
    assert p.inverse_split == 1
    p.inverse_split = 0  # back to the plan's choice
    assert p.inverse_split == d
    for bad in (-1, 17):
        with pytest.raises(RuntimeError):
            p.inverse_split = bad
    assert p.inverse_split == d
    p.close()


def test_env_override(ffst, monkeypatch):
    monkeypatch.setenv("FFST_INV_SPLIT", "5")
    p = ffst.Plan(256, 256)
    assert p.inverse_split == 5
    p.close()


@pytest.mark.parametrize("n", [512, 1024])
def test_splits_agree_and_reconstruct(ffst, n):
    x = torch.from_numpy(inputs.scaled_cartoon(n, n, seed=21)).cuda()
    p = ffst.Plan(n, n)
    c = p.forward(x)
    outs = {}
    for ns in (1, 2, 4, 7, 16):
        p.inverse_split = ns
        outs[ns] = p.inverse(c).clone()
        assert float(torch.linalg.norm(outs[ns] - x) / torch.linalg.norm(x)) < 1e-5
    for ns, r in outs.items():
        assert float(torch.linalg.norm(r - outs[1]) / torch.linalg.norm(outs[1])) < 1e-6, ns
    # deterministic for a fixed split
    p.inverse_split = 7
    assert torch.equal(p.inverse(c), outs[7])
    p.close()


@pytest.mark.parametrize("nsplit", [1, 4, 16])
def test_groups_do_not_change_result(ffst, monkeypatch, nsplit):
    """Chunk boundaries are global, so the inverse group budget (one group or
    eight-plane groups with fused launches) leaves the result bit for bit."""
    x = torch.from_numpy(inputs.scaled_cartoon(512, 512, seed=4)).cuda()
    p1 = ffst.Plan(512, 512)
    monkeypatch.setenv("FFST_GROUP_MB_INV", "8")
    p2 = ffst.Plan(512, 512)
    assert p2.group_mb[1] == 8 and p1.group_mb[1] != 8
    c = p1.forward(x)
    for p in (p1, p2):
        p.inverse_split = nsplit
    assert torch.equal(p1.inverse(c), p2.inverse(c))
    assert torch.equal(p1.adjoint(c), p2.adjoint(c))
    p1.close()
    p2.close()


@pytest.mark.parametrize("nsplit", [3, 16])
def test_persistent_schedule_follows_chunks(ffst, nsplit):
    x = torch.from_numpy(inputs.scaled_cartoon(512, 512, seed=6)).cuda()
    p = ffst.Plan(512, 512)
    c = p.forward(x)
    p.inverse_split = nsplit
    r0 = p.inverse(c).clone()
    p.schedule = 1
    assert p.schedule == 1
    r1 = p.inverse(c)
    assert p.check() == 0
    assert torch.equal(r1, r0)
    p.inverse_split = 2  # rebuilds the persistent schedule's batches
    p.schedule = 0
    r2 = p.inverse(c).clone()
    p.schedule = 1
    assert torch.equal(p.inverse(c), r2)
    p.close()
