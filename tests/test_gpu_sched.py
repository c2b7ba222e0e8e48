"""Persistent schedule of the plane passes (opt-in) against the grouped launches.

Both schedules run the same per-element arithmetic in the same order (the
forward per plane, the inverse accumulation in plane order), so their
results must agree bit for bit; the oracle parity of the default schedule is
covered by test_gpu_parity.  Also checks the bounded device-side waits: in
test mode 2 the forward's first task waits on a counter nothing increments,
the wait runs out, ffst_plan_check reports FFST_ERR_TIMEOUT, and the plan
keeps working afterwards.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

SQUARE = [256, 512, 1024, 2048]


@pytest.fixture(scope="module")
def ffst():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_1202_1773_gb300 as m

    return m


def _image(n, seed):
    from paper_1202_1773_gb300 import inputs

    return torch.from_numpy(inputs.scaled_cartoon(n, n, seed=seed)).cuda()


def _run(plan, x, mode, dtype=None):
    plan.schedule = mode
    if dtype is None:
        c = plan.forward(x)
        sc = None
    else:
        c, sc = plan.forward(x, dtype=dtype)
    r = plan.inverse(c, plane_scale=sc)
    a = plan.adjoint(c, plane_scale=sc)
    assert plan.check() == 0
    return c.clone(), None if sc is None else sc.clone(), r.clone(), a.clone()


@pytest.mark.parametrize("n", SQUARE)
def test_sched_matches_grouped_bitwise(ffst, n):
    p = ffst.Plan(n, n)
    assert p.schedule == 0  # grouped launches by default
    p.schedule = 1
    assert p.schedule == 1
    info = p.schedule_info()
    assert info["blocks"] > 0 and info["fwd_tasks"] > 0 and info["inv_tasks"] > 0
    x = _image(n, seed=11 + n)
    c1, _, r1, a1 = _run(p, x, 1)
    c0, _, r0, a0 = _run(p, x, 0)
    assert torch.equal(c1, c0)
    assert torch.equal(r1, r0)
    assert torch.equal(a1, a0)
    # and the persistent result is a transform: perfect reconstruction
    assert float(torch.linalg.norm(r1 - x) / torch.linalg.norm(x)) < 1e-5
    p.close()


@pytest.mark.parametrize("dtype", ["f16", "bf16"])
def test_sched_low_precision_bitwise(ffst, dtype):
    dt = torch.float16 if dtype == "f16" else torch.bfloat16
    p = ffst.Plan(512, 512)
    x = _image(512, seed=5)
    c1, s1, r1, _ = _run(p, x, 1, dt)
    c0, s0, r0, _ = _run(p, x, 0, dt)
    assert torch.equal(s1, s0)
    assert torch.equal(c1.view(torch.int16), c0.view(torch.int16))
    assert torch.equal(r1, r0)
    p.close()


def test_sched_deterministic(ffst):
    p = ffst.Plan(1024, 1024)
    x = _image(1024, seed=7)
    outs = [_run(p, x, 1) for _ in range(3)]
    for c, _, r, a in outs[1:]:
        assert torch.equal(c, outs[0][0]) and torch.equal(r, outs[0][2]) and torch.equal(a, outs[0][3])
    p.close()


@pytest.mark.parametrize("shape", [(128, 128), (480, 640), (512, 1024)])
def test_sizes_without_persistent_schedule(ffst, shape):
    p = ffst.Plan(*shape)
    assert p.schedule == 0  # no persistent schedule: grouped or separate launches
    p.schedule = 1          # asking for it keeps the launches that exist
    assert p.schedule == 0
    p.close()


def test_schedule_mode_errors(ffst):
    p = ffst.Plan(256, 256)
    with pytest.raises(RuntimeError):
        p.schedule = 3
    with pytest.raises(RuntimeError):
        p.schedule = -1
    p.close()


def test_stuck_wait_times_out_and_plan_recovers(ffst):
    from paper_1202_1773_gb300._lib import FFST_ERR_TIMEOUT

    p = ffst.Plan(512, 512)
    x = _image(512, seed=9)
    ref = p.forward(x).clone()
    assert p.check() == 0
    p.schedule = 2
    p.forward(x)
    assert p.check() == FFST_ERR_TIMEOUT
    assert p.check() == 0  # the flag is cleared by the check that reported it
    p.schedule = 1
    c = p.forward(x)
    assert p.check() == 0
    assert torch.equal(c, ref)
    r = p.inverse(c)
    assert float(torch.linalg.norm(r - x) / torch.linalg.norm(x)) < 1e-5
    p.close()
