"""bench.py's multi-process path on the CPU: two gloo ranks.

The transform of one image has no exchange step, so N GPUs run N
independent replicas; the only collective work is the host's: a barrier
around the timed region, the slowest rank's time (max over ranks) and the
whole-job value (units all ranks processed over that time).  Under torchrun
the reference arm runs on rank 0 alone; the other ranks exit 0 without
work.  This test runs those pieces as two spawned processes on the gloo
backend (no GPU).
"""

import json
import os
import socket
import sys
from types import SimpleNamespace

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench

    w, r, _ = bench._dist()
    dist = bench._init_pg(w, "gloo")
    ms = 10.0 * (r + 1)  # rank-dependent step time: rank 1 is the slowest
    bench._barrier(w)
    ms_max = bench._max_over_ranks(ms, w, "cpu")
    value = bench._job_value(1000.0, 4, w, ms_max)
    ref = None
    if r != 0:  # the reference arm: only rank 0 runs the oracle
        ref = bench.run_reference(SimpleNamespace(steps=1, warmup=0, gpus=w))
    bench._barrier(w)
    with open(os.path.join(out_dir, f"rank{r}.json"), "w") as fh:
        json.dump({"world": w, "ms_max": ms_max, "value": value, "ref": ref}, fh)
    dist.destroy_process_group()


def test_two_replicas_on_gloo(tmp_path):
    port = _free_port()
    torch.multiprocessing.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                                          start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    for d in res:
        assert d["world"] == 2
        assert d["ms_max"] == 20.0  # every rank sees the slowest rank's time
        assert d["value"] == pytest.approx(1000.0 * 4 * 2 / 0.020)  # units of both ranks / max time
    assert res[1]["ref"] == 0  # non-zero rank of the reference arm: no work, exit status 0


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench._max_over_ranks(3.5, 1, "cpu") == 3.5
    bench._barrier(1)  # no process group: a no-op
    assert bench._job_value(10.0, 2, 1, 4.0) == pytest.approx(10.0 * 2 / 0.004)
