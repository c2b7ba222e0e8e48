"""The plane-sharded inverse's exchange on the CPU: two and three gloo ranks.

Each rank holds a contiguous range of planes (sharded.plane_range), forms
its partial spectrum sum_{i in range} psi_hat_i * fft2(c_i) and the ranks
combine them with sharded.reduce_finish (one sum-reduce, the root finishes
with ifft2 of the sum divided by sum_i psi_hat_i^2).  The partial spectra
here come from the FP64 oracle's spectra (the CUDA partials are checked on
the GPU in tests/test_gpu_sharded.py); what runs is the product's plane
partition and reduce/finish plumbing.  The root's image must equal the
single-process inverse (Sec. 3.3) to 1e-12 and the image to 1e-12.
"""

import json
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SHAPE = (32, 48)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    from oracle import ffst_oracle as o
    from paper_1202_1773_gb300 import sharded

    dist.init_process_group("gloo", rank=rank, world_size=world)
    f = np.random.default_rng(3).standard_normal(SHAPE)
    psi = o.spectra(*SHAPE)
    eta = psi.shape[0]
    p0, p1 = sharded.plane_range(eta, world, rank)
    c = o.forward_with(psi, f)[p0:p1]  # this rank's coefficients only
    part = np.zeros(SHAPE, dtype=np.complex128)
    for q, i in enumerate(range(p0, p1)):
        part += psi[i] * np.fft.fft2(c[q])
    den = (psi * psi).sum(axis=0)
    img = sharded.reduce_finish(torch.from_numpy(part),
                                lambda s: np.real(np.fft.ifft2(s.numpy() / den)))
    res = {"range": [p0, p1]}
    if img is not None:
        ref = o.inverse(o.forward(f))
        res["err_vs_inverse"] = float(np.abs(img - ref).max())
        res["err_vs_image"] = float(np.abs(img - f).max())
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as fh:
        json.dump(res, fh)
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_inverse_on_gloo(tmp_path, world):
    port = _free_port()
    torch.multiprocessing.start_processes(_worker, args=(world, port, str(tmp_path)), nprocs=world, join=True,
                                          start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    ranges = [tuple(d["range"]) for d in res]
    assert ranges[0][0] == 0 and all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
    assert ranges[-1][1] == 13  # eta = 2^(j0+2) - 3 of a 32x48 image (j0 = 2)
    assert res[0]["err_vs_inverse"] <= 1e-12
    assert res[0]["err_vs_image"] <= 1e-12
    assert all("err_vs_inverse" not in d for d in res[1:])  # only the root finishes


def test_plane_range_partition():
    sys.path.insert(0, ROOT)
    from paper_1202_1773_gb300 import sharded

    for eta in (5, 13, 29, 61, 125, 253):
        for world in range(1, 9):
            if world > eta:
                continue
            rs = [sharded.plane_range(eta, world, r) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == eta
            assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
            sizes = [b - a for a, b in rs]
            assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 1
    with pytest.raises(ValueError):
        sharded.plane_range(5, 8, 0)
    with pytest.raises(ValueError):
        sharded.plane_range(29, 2, 2)
