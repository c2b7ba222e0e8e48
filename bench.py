"""Benchmark: FFST forward + inverse throughput (shearlet coefficients / s).

Workload (one step): forward transform of one 2048x2048 float32 image with
j0 = 5 scales (eta = 125 planes, 524,288,000 coefficients, stack stored as
float32), then the inverse transform of that stack back to an image.  Inputs
are seeded synthetic cartoon images (ellipses + polygons + N(0, 0.1^2)),
already resident in device memory; the 2.1 GB coefficient stack written and
read every step is far larger than L2, so no explicit flush is needed.

Prints one JSON line.  `value` = eta*M*N*steps*ranks / (max over ranks of
the timed region); `e2e` = the same metric through the public API with the
image copied host->device and the reconstruction copied back every step;
`roofline` = the dominant kernel's algorithmic HBM bytes per launch over its
CUDA-event duration, against the measured copy bandwidth; `cpu_baseline`
= the FP64 oracle timed on this host's cores on a bounded sample.

--impl reference times the FP64 CPU oracle (the only reference this method
has) on the same workload definition, one bounded sample per step.
Multi-GPU (torchrun): every rank runs its own images (independent replicas,
weak scaling, no collective on the data path).
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

ROWS, COLS, SCALES = 2048, 2048, 5
METRIC = "fwd+inv shearlet coeffs/s (2048x2048 f32, J=5, eta=125)"
UNIT = "coeffs/s"


def _measured_traffic(kind):
    """DRAM bytes per launch of a kernel kind from the committed ncu capture
    (profiles/ffst_2048x2048_j5_dram_traffic.json), or None when the kernel
    sources changed since that capture.  The generic-length (Bluestein) line
    sources, ffst_blue*, do not enter the native kernels and are left out."""
    import glob
    import hashlib

    try:
        with open(os.path.join(ROOT, "profiles", "ffst_2048x2048_j5_dram_traffic.json")) as fh:
            d = json.load(fh)
        src = sorted([f for f in glob.glob(os.path.join(ROOT, "paper_1202_1773_gb300", "csrc", "*"))
                      if not os.path.basename(f).startswith("ffst_blue")] +
                     glob.glob(os.path.join(ROOT, "include", "*.h")))
        h = hashlib.sha256(b"".join(open(f, "rb").read() for f in src)).hexdigest()[:16]
        if h != d["source_hash"]:
            return None
        return d["kernels"][kind]["traffic_bytes_per_launch"]
    except Exception:
        return None


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """Samples SM clocks / throttle reasons with nvidia-smi while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _init_pg(world, backend):
    import torch.distributed as dist

    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return dist


def _max_over_ranks(x: float, world: int, device):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _job_value(units_per_step: float, steps: int, world: int, ms_max: float) -> float:
    """Whole-job throughput: the units every rank processed (each rank runs
    its own replica of the workload) over the slowest rank's time."""
    return units_per_step * steps * world / (ms_max / 1e3)


def _barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


# ---------------------------------------------------------------------------
# CPU oracle (baseline / reference arm)
# ---------------------------------------------------------------------------

ORACLE_STEP_PLANES = 1      # planes per worker per sample (~5 s of CPU each)
ORACLE_BASELINE_PLANES = 2  # single-core leg of the GPU arm's cpu_baseline
ORACLE_REPEATS = 3          # samples per leg (median)


def oracle_sample_seconds(f64, planes, first=0):
    """Time the FP64 oracle on a bounded sample of one step: fft2 of the image,
    `planes` forward planes (indices first, first + 1, ...), the inverse
    contributions of those planes and the final ifft2.  Returns (seconds,
    coefficients processed)."""
    from oracle import ffst_oracle as o

    M, N = f64.shape
    eta = o.num_planes(SCALES)
    t0 = time.perf_counter()
    F = np.fft.fft2(f64)
    acc = np.zeros((M, N), dtype=np.complex128)
    den = np.zeros((M, N))
    for q in range(planes):
        i = (first + q) % eta
        c = o.forward_plane(F, SCALES, i)
        s = o.spectrum(M, N, SCALES, i)
        acc += s * np.fft.fft2(c)
        den += s * s
    np.real(np.fft.ifft2(acc / np.where(den > 0, den, 1.0)))
    return time.perf_counter() - t0, planes * M * N


_WORKER_IMG = None


def _oracle_worker_init(seed):
    global _WORKER_IMG
    from paper_1202_1773_gb300 import inputs

    _WORKER_IMG = inputs.scaled_cartoon(ROWS, COLS, seed=seed).astype(np.float64)


def _oracle_worker(first):
    return oracle_sample_seconds(_WORKER_IMG, ORACLE_STEP_PLANES, first)


def host_identity():
    """Logical core count and CPU model name of this host (lscpu)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.split(":")[0].strip() in ("Model name", "Model Name"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model}


class OraclePool:
    """The FP64 oracle on every host core: one spawned process per core, each
    running the oracle as it stands on its own planes of the same image (the
    planes of the transform are independent).  Spawned, not forked, so it is
    safe to start after CUDA."""

    def __init__(self, seed, workers=None):
        import multiprocessing as mp

        self.workers = workers or os.cpu_count() or 1
        self.pool = mp.get_context("spawn").Pool(self.workers, initializer=_oracle_worker_init, initargs=(seed,))
        self.pool.map(_oracle_worker, range(self.workers))  # warm: imports, image, first FFTs

    def sample(self, first=0):
        """One all-core sample: wall seconds and coefficients processed."""
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_worker, [first + w * ORACLE_STEP_PLANES for w in range(self.workers)])
        return time.perf_counter() - t0, sum(c for _, c in res)

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_baseline_numbers(seed, f64):
    """cpu_baseline of the GPU arm: the oracle on all host cores and on one
    core, each the median rate of ORACLE_REPEATS bounded samples."""
    pool = OraclePool(seed)
    try:
        rates = []
        for r in range(ORACLE_REPEATS):
            s, c = pool.sample(first=r * pool.workers)
            rates.append(c / s)
    finally:
        pool.close()
    oracle_sample_seconds(f64, planes=1)
    single = []
    for r in range(ORACLE_REPEATS):
        s, c = oracle_sample_seconds(f64, ORACLE_BASELINE_PLANES, first=r * ORACLE_BASELINE_PLANES)
        single.append(c / s)
    host = host_identity()
    sample = (f"per sample: each of {pool.workers} worker processes runs fft2 + {ORACLE_STEP_PLANES} plane(s) "
              f"forward and inverse + ifft2 of the 2048x2048 J=5 workload (FP64 NumPy oracle, one process per "
              f"core); median of {ORACLE_REPEATS} samples, rate scaled to coefficients/s")
    return {"value": statistics.median(rates), "unit": UNIT, "cores": pool.workers, "kind": "oracle",
            "sample": sample, "host": host,
            "single_core": {"value": statistics.median(single), "unit": UNIT, "cores": 1,
                            "sample": f"fft2 + {ORACLE_BASELINE_PLANES} of 125 planes fwd+inv + ifft2 in one "
                                      f"process, median of {ORACLE_REPEATS}"}}


def run_reference(args):
    world, rank, local = _dist()
    if world > 1 and rank != 0:
        return 0
    from paper_1202_1773_gb300 import inputs

    pool = OraclePool(seed=5)
    try:
        for w in range(args.warmup):
            pool.sample(first=w)
        tot_s, tot_c = 0.0, 0
        for q in range(args.steps):
            s, c = pool.sample(first=q * pool.workers)
            tot_s += s
            tot_c += c
    finally:
        pool.close()
    value = tot_c / tot_s
    sample = (f"per step: each of {pool.workers} worker processes (one per host core) runs fft2 + "
              f"{ORACLE_STEP_PLANES} plane(s) forward and inverse + ifft2 of the 2048x2048 J=5 workload "
              f"(FP64 NumPy oracle), rate scaled to coefficients/s")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": "FFST fwd+inv, 2048x2048 f32 image, J=5, eta=125", "rows": ROWS, "cols": COLS,
                       "scales": SCALES},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.workers, "kind": "oracle",
                             "sample": sample, "host": host_identity()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_gpu(args):
    import torch

    import paper_1202_1773_gb300 as ffst
    from paper_1202_1773_gb300 import build, inputs

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    _init_pg(world, "nccl")
    build.build()

    ffst.Plan(64, 64, device=dev).close()  # context and module loading outside the plan timing
    torch.cuda.synchronize(dev)
    tp = time.perf_counter()
    plan = ffst.Plan(ROWS, COLS, SCALES, device=dev)
    plan_ms = 1e3 * (time.perf_counter() - tp)
    eta = plan.num_planes
    coeffs_per_step = eta * ROWS * COLS
    pool = [torch.from_numpy(inputs.scaled_cartoon(ROWS, COLS, seed=100 + 8 * rank + q)).to(dev) for q in range(4)]
    stack = torch.empty(plan.shape, dtype=torch.float32, device=dev)
    rec = torch.empty((ROWS, COLS), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(q):
        plan.forward(pool[q % len(pool)], out=stack)
        plan.inverse(stack, out=rec)

    for q in range(args.warmup):
        step(q)
    torch.cuda.synchronize(dev)

    # timed region (the headline value): no per-kernel instrumentation
    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.5)
    _barrier(world)
    torch.cuda.synchronize(dev)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for q in range(args.steps):
        step(q)
    t1.record(stream)
    torch.cuda.synchronize(dev)
    _barrier(world)
    clocks = sampler.stop() if sampler else None
    ms = t0.elapsed_time(t1)
    ms_max = _max_over_ranks(ms, world, dev)
    value = _job_value(coeffs_per_step, args.steps, world, ms_max)

    # the same number of steps again with every kernel bracketed by CUDA
    # events on the launch stream: per-kernel durations for the roofline
    plan.timing_reset()
    plan.timing(True)
    for q in range(args.steps):
        step(q)
    torch.cuda.synchronize(dev)
    plan.timing(False)
    kernels = plan.timing_read()

    # forward / inverse split (untimed loop, events only)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    fwd_ms = inv_ms = 0.0
    for q in range(max(3, args.steps // 2)):
        e[0].record(stream)
        plan.forward(pool[q % len(pool)], out=stack)
        e[1].record(stream)
        plan.inverse(stack, out=rec)
        e[2].record(stream)
        torch.cuda.synchronize(dev)
        fwd_ms += e[0].elapsed_time(e[1])
        inv_ms += e[1].elapsed_time(e[2])
    nsplit = max(3, args.steps // 2)

    # end to end through the public API with host buffers
    host_img = [torch.from_numpy(inputs.scaled_cartoon(ROWS, COLS, seed=200 + q)).pin_memory() for q in range(2)]
    host_out = torch.empty((ROWS, COLS), dtype=torch.float32).pin_memory()
    dimg = torch.empty((ROWS, COLS), dtype=torch.float32, device=dev)

    def e2e_step(q):
        dimg.copy_(host_img[q % 2], non_blocking=True)
        plan.forward(dimg, out=stack)
        plan.inverse(stack, out=rec)
        host_out.copy_(rec, non_blocking=True)

    for q in range(2):
        e2e_step(q)
    torch.cuda.synchronize(dev)
    _barrier(world)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    tw = time.perf_counter()
    a.record(stream)
    for q in range(args.steps):
        e2e_step(q)
    b.record(stream)
    torch.cuda.synchronize(dev)
    wall_ms = _max_over_ranks(1e3 * (time.perf_counter() - tw), world, dev)  # host launch cost included
    e2e_ms = _max_over_ranks(a.elapsed_time(b), world, dev)
    e2e_value = _job_value(coeffs_per_step, args.steps, world, e2e_ms)
    e2e_wall_value = _job_value(coeffs_per_step, args.steps, world, wall_ms)

    forms = None if args.no_forms else run_forms(plan, pool, stack, rec, value, args, dev)

    if rank != 0:
        return 0

    # roofline of the dominant kernel (largest total time in the timed region)
    peak, peak_kind = _peaks()
    name, (kms, kn, kbytes) = max(kernels.items(), key=lambda kv: kv[1][0])
    step_bytes = 2.0 * coeffs_per_step * 4 + 8.0 * ROWS * COLS
    if kbytes > 0 and kn > 0:
        achieved = (kbytes / kn) / ((kms / kn) / 1e3) / 1e9
        roof = {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": _measured_traffic(name), "peak_source": peak_kind,
                "algorithmic_bytes_per_launch": kbytes / kn, "launches": kn, "avg_ms": kms / kn}
    else:
        roof = {"kernel": name, "bound": "alu", "achieved": None, "peak": None, "unit": "GB/s", "frac": None,
                "traffic": None, "launches": kn, "avg_ms": kms / max(kn, 1),
                "note": "intermediates stay in L2: no algorithmic HBM bytes"}
    step_gbs = step_bytes * args.steps / (ms_max / 1e3) / 1e9

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline_numbers(100 + 8 * rank, pool[0].double().cpu().numpy())

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "FFST fwd+inv, 2048x2048 f32 image, J=5, eta=125, f32 stack",
                   "rows": ROWS, "cols": COLS, "scales": SCALES, "planes": eta,
                   "coeffs_per_step": coeffs_per_step,
                   "l2": "inputs larger than L2 (2.10 GB coefficient stack written and read per step)",
                   "parallelism": f"replicas x{world}"},
        "fwd_ms": fwd_ms / nsplit, "inv_ms": inv_ms / nsplit, "plan_ms": plan_ms,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 4 * ROWS * COLS,
                "d2h_bytes_per_step": 4 * ROWS * COLS,
                "wall_clock": {"value": e2e_wall_value, "ms_per_step": wall_ms / args.steps,
                               "note": "host time.perf_counter() around the same loop and its final "
                                       "synchronize: launch and API cost on the host included"}},
        "roofline": roof,
        "roofline_step": {"bound": "hbm", "achieved": step_gbs, "peak": peak, "unit": "GB/s",
                          "frac": step_gbs / peak, "bytes_per_step": step_bytes, "peak_source": peak_kind},
        "kernels": {k: {"ms_per_step": v[0] / args.steps, "launches_per_step": v[1] / args.steps,
                        "alg_bytes_per_step": v[2] / args.steps} for k, v in kernels.items() if v[1]},
        "gpu_launches": int(sum(v[1] for v in kernels.values())),
        "forms": forms,
        "clocks": clocks,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_sharded(args):
    """--shard planes: one image per step, its planes split over the ranks
    (strong scaling).  Each rank runs the forward of its plane range (it
    recomputes fft2 of the image) and its partial inverse spectrum; one
    NCCL sum-reduce of the M x (N/2+1) complex64 spectrum onto rank 0, which
    finishes the inverse.  value = the image's coefficients per step / the
    slowest rank's time."""
    import torch

    from paper_1202_1773_gb300 import build, inputs, sharded

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    _init_pg(world, "nccl")
    build.build()
    sp = sharded.ShardedPlan(ROWS, COLS, SCALES, device=dev)
    eta = sp.plan.num_planes
    coeffs_per_step = eta * ROWS * COLS
    pool = [torch.from_numpy(inputs.scaled_cartoon(ROWS, COLS, seed=100 + q)).to(dev) for q in range(2)]
    stack = torch.empty(sp.shape, dtype=torch.float32, device=dev)
    rec = torch.empty((ROWS, COLS), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(q):
        sp.forward(pool[q % 2], out=stack)
        sp.inverse(stack, out=rec)

    for q in range(args.warmup):
        step(q)
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.5)
    _barrier(world)
    torch.cuda.synchronize(dev)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for q in range(args.steps):
        step(q)
    b.record(stream)
    torch.cuda.synchronize(dev)
    _barrier(world)
    clocks = sampler.stop() if sampler else None
    ms_max = _max_over_ranks(a.elapsed_time(b), world, dev)
    value = coeffs_per_step * args.steps / (ms_max / 1e3)
    err = None
    if rank == 0:
        err = float(torch.linalg.norm(rec - pool[(args.steps - 1) % 2]) / torch.linalg.norm(pool[(args.steps - 1) % 2]))
    # end to end: every rank copies the image up, rank 0 copies the result down
    host_img = torch.from_numpy(inputs.scaled_cartoon(ROWS, COLS, seed=200)).pin_memory()
    host_out = torch.empty((ROWS, COLS), dtype=torch.float32).pin_memory()
    dimg = torch.empty((ROWS, COLS), dtype=torch.float32, device=dev)

    def e2e_step(q):
        dimg.copy_(host_img, non_blocking=True)
        sp.forward(dimg, out=stack)
        sp.inverse(stack, out=rec)
        if rank == 0:
            host_out.copy_(rec, non_blocking=True)

    e2e_step(0)
    torch.cuda.synchronize(dev)
    _barrier(world)
    a.record(stream)
    for q in range(args.steps):
        e2e_step(q)
    b.record(stream)
    torch.cuda.synchronize(dev)
    e2e_ms = _max_over_ranks(a.elapsed_time(b), world, dev)
    if rank != 0:
        return 0
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "FFST fwd+inv, 2048x2048 f32 image, J=5, eta=125, f32 stack, planes split over ranks",
                   "rows": ROWS, "cols": COLS, "scales": SCALES, "planes": eta,
                   "coeffs_per_step": coeffs_per_step,
                   "l2": "inputs larger than L2 (2.10 GB coefficient stack per step over all ranks)",
                   "parallelism": f"planes x{world} (one sum-reduce of the partial inverse spectrum)"},
        "e2e": {"value": coeffs_per_step * args.steps / (e2e_ms / 1e3), "unit": UNIT,
                "h2d_bytes_per_step": 4 * ROWS * COLS * world, "d2h_bytes_per_step": 4 * ROWS * COLS},
        "accuracy": {"reconstruction_rel_l2": err},
        "clocks": clocks,
        "cpu_baseline": None,
    }
    print(json.dumps(line), flush=True)
    return 0


def _time_steps(fn, steps, dev):
    import torch

    stream = torch.cuda.current_stream(dev)
    for q in range(3):
        fn(q)
    torch.cuda.synchronize(dev)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for q in range(steps):
        fn(q)
    b.record(stream)
    torch.cuda.synchronize(dev)
    return a.elapsed_time(b) / steps


def run_forms(plan, pool, stack, rec, plain_value, args, dev):
    """The forms beside the plain FP32 round trip, each timed like the plain
    step and with its accuracy measured on the GPU against the plain FP32
    path (reconstruction error; coefficient error of low-precision storage
    against the FP32 stack; d(i) against the stored stack)."""
    import torch

    import paper_1202_1773_gb300 as ffst
    from paper_1202_1773_gb300 import inputs

    steps = max(3, args.steps // 2)
    eta = plan.num_planes
    cps = eta * ROWS * COLS
    out = {}
    x0 = pool[0]
    ref = plan.forward(x0).clone()
    xnorm = float(torch.linalg.norm(x0))

    # adjoint: forward + ffst_adjoint (the backward of the differentiable layer)
    ms = _time_steps(lambda q: (plan.forward(pool[q % len(pool)], out=stack), plan.adjoint(stack, out=rec)), steps, dev)
    plan.forward(x0, out=stack)
    err = float(torch.linalg.norm(plan.adjoint(stack) - x0)) / xnorm
    out["adjoint"] = {"value": cps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "vs_plain": cps / (ms / 1e3) / plain_value,
                      "accuracy": {"reconstruction_rel_l2": err}}

    # low-precision stack storage (FP32 arithmetic)
    for name, dt, tol in (("f16", torch.float16, 2e-3), ("bf16", torch.bfloat16, 1e-2)):
        lp = torch.empty(plan.shape, dtype=dt, device=dev)
        sc = torch.empty(eta, device=dev)
        ms = _time_steps(lambda q: (plan.forward(pool[q % len(pool)], out=lp, plane_scale=sc),
                                    plan.inverse(lp, plane_scale=sc, out=rec)), steps, dev)
        plan.forward(x0, out=lp, plane_scale=sc)
        cerr = 0.0
        for i in range(eta):  # plane by plane, no full-size temporaries
            d = lp[i].float() / sc[i] - ref[i]
            cerr += float((d.double() ** 2).sum())
        cerr = (cerr / sum(float((ref[i].double() ** 2).sum()) for i in range(eta))) ** 0.5
        rerr = float(torch.linalg.norm(plan.inverse(lp, plane_scale=sc) - x0)) / xnorm
        byts = 2.0 * cps * 2 + 8.0 * ROWS * COLS
        out[name] = {"value": cps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
                     "vs_plain": cps / (ms / 1e3) / plain_value, "stack_bytes_saved": cps * 2,
                     "roofline_step_frac": byts / (ms / 1e3) / 1e9 / _peaks()[0],
                     "accuracy": {"coeff_rel_l2_vs_f32": cerr, "reconstruction_rel_l2": rerr, "tolerance": tol}}
        del lp

    # fused per-plane statistics + soft shrinkage in the forward's row pass,
    # then the inverse (one denoising round trip), against the plain round trip
    d0 = plan.forward_stats(x0, out=stack)[1]
    thr = (1.5 * d0).contiguous()
    thr[0] = 0.0
    ms = _time_steps(lambda q: (plan.forward_stats(pool[q % len(pool)], shrink="soft", thresh=thr, out=stack),
                                plan.inverse(stack, out=rec)), steps, dev)
    plan.forward_stats(x0, shrink="soft", thresh=thr, out=stack)
    kept = float(sum(int(torch.count_nonzero(stack[i])) for i in range(eta))) / cps
    dref = torch.stack([ref[i].double().abs().mean() for i in range(eta)])  # plane by plane
    dmax = float(((d0.double() - dref).abs() / dref.clamp_min(1e-30)).max())
    out["stats_soft"] = {"value": cps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
                         "vs_plain": cps / (ms / 1e3) / plain_value, "threshold": "1.5 d(i) per plane, low-pass kept",
                         "kept_fraction": kept, "accuracy": {"mean_abs_rel_vs_stack_max": dmax}}

    # one-sided complex shearlets (Sec. 3.8.2): planar complex stack, both parts and the inverse
    zst = torch.empty((eta, 2, ROWS, COLS), device=dev)
    ms = _time_steps(lambda q: (plan.forward_complex(pool[q % len(pool)], out=zst), plan.inverse_complex(zst, out=rec)),
                     steps, dev)
    plan.forward_complex(x0, out=zst)
    err = float(torch.linalg.norm(plan.inverse_complex(zst) - x0)) / xnorm
    out["complex"] = {"value": cps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "vs_plain": cps / (ms / 1e3) / plain_value,
                      "stack_bytes": 2 * cps * 4, "accuracy": {"reconstruction_rel_l2": err}}
    del zst

    # smooth shearlets (Sec. 3.4): a plan of the same size, same round trip
    sp = ffst.Plan(ROWS, COLS, SCALES, device=dev, smooth=True)
    ms = _time_steps(lambda q: (sp.forward(pool[q % len(pool)], out=stack), sp.inverse(stack, out=rec)), steps, dev)
    sp.forward(x0, out=stack)
    err = float(torch.linalg.norm(sp.inverse(stack) - x0)) / xnorm
    out["smooth"] = {"value": cps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "vs_plain": cps / (ms / 1e3) / plain_value,
                     "accuracy": {"reconstruction_rel_l2": err}}
    sp.close()

    # odd size: 2047x2047 (no native FFT line: Bluestein lines of L2 = 4096 in
    # both dimensions), same scales, same round trip
    on = ROWS - 1
    op = ffst.Plan(on, on, SCALES, device=dev)
    opool = [torch.from_numpy(inputs.scaled_cartoon(on, on, seed=400 + q)).to(dev) for q in range(2)]
    ost = torch.empty(op.shape, device=dev)
    orec = torch.empty(on, on, device=dev)
    ms = _time_steps(lambda q: (op.forward(opool[q % 2], out=ost), op.inverse(ost, out=orec)), steps, dev)
    op.forward(opool[0], out=ost)
    err = float(torch.linalg.norm(op.inverse(ost) - opool[0]) / torch.linalg.norm(opool[0]))
    ocps = op.num_planes * on * on
    out["odd_2047"] = {"value": ocps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
                       "vs_plain": ocps / (ms / 1e3) / plain_value, "size": f"{on}x{on}", "lines": "Bluestein, L2 = 4096",
                       "accuracy": {"reconstruction_rel_l2": err}}
    del ost, orec, opool
    op.close()

    # large low-precision storage: 4096x4096, J=6 (253 planes), the FP32 stack
    # and the FP16 / BF16 stacks with per-plane scales, each as one round trip
    del ref
    out.update(_forms_4096(args, dev))

    # differentiable layer: 200 FISTA steps of shearlet-l1 deconvolution at
    # 1024x1024 J=5 (each step one forward and one adjoint through autograd)
    out["deconv_1024"] = _form_deconv(plain_value, dev)

    # batched: 256 images of uneven sizes, forward + inverse replayed from one CUDA graph
    n = 256
    shapes = inputs.batch_sizes(n, seed=2)
    srcs = {}
    for (r, c) in sorted(set(shapes)):
        srcs[(r, c)] = [torch.from_numpy(inputs.scaled_cartoon(r, c, seed=300 + q)).to(dev) for q in range(2)]
    imgs = [srcs[sh][i % 2] for i, sh in enumerate(shapes)]
    bp = ffst.BatchPlan(shapes, lanes=8, device=dev)
    stacks = bp.empty_stacks()
    outs = [torch.empty(sh, device=dev) for sh in shapes]
    graph = bp.capture(imgs, stacks, outs, what=3)
    total = sum(bp.shape(i)[0] * shapes[i][0] * shapes[i][1] for i in range(n))
    ms = _time_steps(lambda q: graph.launch(), max(2, args.steps // 5), dev)
    errs = [float(torch.linalg.norm(outs[i] - imgs[i]) / torch.linalg.norm(imgs[i])) for i in range(n)]
    byts = 2.0 * total * 4 + 8.0 * sum(r * c for r, c in shapes)
    # the same 256 round trips one after another through single plans (one
    # per shape, eager launches on one stream): what the batch saves
    singles = {sh: ffst.Plan(*sh, device=dev) for sh in sorted(set(shapes))}
    s_stk = {sh: torch.empty(singles[sh].shape, device=dev) for sh in singles}
    s_rec = {sh: torch.empty(sh, device=dev) for sh in singles}

    def _sequential(q):
        for i, sh in enumerate(shapes):
            singles[sh].forward(imgs[i], out=s_stk[sh])
            singles[sh].inverse(s_stk[sh], out=s_rec[sh])

    seq_ms = _time_steps(_sequential, 2, dev)
    for p_ in singles.values():
        p_.close()
    del s_stk, s_rec
    out["batched"] = {"value": total / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
                      "vs_plain": total / (ms / 1e3) / plain_value,
                      "sequential_single_plans_ms": seq_ms, "vs_sequential": seq_ms / ms, "images": n,
                      "sizes": {f"{r}x{c}": shapes.count((r, c)) for (r, c) in sorted(set(shapes))},
                      "coeffs_per_step": total, "lanes": 8, "graph": True,
                      "roofline_step_frac": byts / (ms / 1e3) / 1e9 / _peaks()[0],
                      "accuracy": {"reconstruction_rel_l2_max": max(errs)}}
    graph.close()
    bp.close()
    return out


def _forms_4096(args, dev):
    """4096x4096 J=6 round trips: FP32 stack, then FP16 and BF16 stacks with
    per-plane power-of-two scales (FP32 arithmetic), each against the FP32
    round trip of the same size; accuracy of the dequantised coefficients
    against the FP32 stack of the same image, plane by plane."""
    import torch

    import paper_1202_1773_gb300 as ffst
    from paper_1202_1773_gb300 import inputs

    n, j = 4096, 6
    p = ffst.Plan(n, n, j, device=dev)
    eta = p.num_planes
    cps = eta * n * n
    imgs = [torch.from_numpy(inputs.scaled_cartoon(n, n, seed=6 + q)).to(dev) for q in range(2)]
    rec = torch.empty(n, n, device=dev)
    steps = max(2, args.steps // 5)
    out = {}
    st = torch.empty(p.shape, device=dev)
    ms32 = _time_steps(lambda q: (p.forward(imgs[q % 2], out=st), p.inverse(st, out=rec)), steps, dev)
    p.forward(imgs[0], out=st)
    xnorm = float(torch.linalg.norm(imgs[0]))
    err = float(torch.linalg.norm(p.inverse(st) - imgs[0])) / xnorm
    b32 = 2.0 * cps * 4 + 8.0 * n * n
    out["f32_4096"] = {"value": cps / (ms32 / 1e3), "unit": UNIT, "ms_per_step": ms32, "size": "4096x4096, J=6",
                       "planes": eta, "roofline_step_frac": b32 / (ms32 / 1e3) / 1e9 / _peaks()[0],
                       "accuracy": {"reconstruction_rel_l2": err}}
    for name, dt, tol in (("f16_4096", torch.float16, 2e-3), ("bf16_4096", torch.bfloat16, 1e-2)):
        lp = torch.empty(p.shape, dtype=dt, device=dev)
        sc = torch.empty(eta, device=dev)
        ms = _time_steps(lambda q: (p.forward(imgs[q % 2], out=lp, plane_scale=sc),
                                    p.inverse(lp, plane_scale=sc, out=rec)), steps, dev)
        p.forward(imgs[0], out=lp, plane_scale=sc)
        num = den = 0.0
        for i in range(eta):
            d = lp[i].float() / sc[i] - st[i]
            num += float((d.double() ** 2).sum())
            den += float((st[i].double() ** 2).sum())
        rerr = float(torch.linalg.norm(p.inverse(lp, plane_scale=sc) - imgs[0])) / xnorm
        blp = 2.0 * cps * 2 + 8.0 * n * n
        out[name] = {"value": cps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "size": "4096x4096, J=6",
                     "vs_f32_same_size": ms32 / ms, "stack_bytes_saved": cps * 2,
                     "roofline_step_frac": blp / (ms / 1e3) / 1e9 / _peaks()[0],
                     "accuracy": {"coeff_rel_l2_vs_f32": (num / den) ** 0.5, "reconstruction_rel_l2": rerr,
                                  "tolerance": tol}}
        del lp
    del st
    p.close()
    return out


def _form_deconv(plain_value, dev):
    """200 FISTA steps of the shearlet-l1 deconvolution at 1024x1024, J=5
    (Gaussian blur sigma = 2 px, noise sigma = 0.02): time per step, the
    shearlet coefficients moved per second (one forward and one adjoint per
    step) and the restoration's error against the unblurred image."""
    import torch

    import paper_1202_1773_gb300 as ffst
    from paper_1202_1773_gb300 import deconv, inputs

    n, steps = 1024, 200
    truth = inputs.scaled_cartoon(n, n, seed=4, sigma=0.0).astype(np.float32)
    psf = deconv.gaussian_psf(n, n)
    blur = deconv.Blur(psf, dev)
    tt = torch.from_numpy(truth).to(dev)
    g = torch.Generator(device=dev).manual_seed(13)
    y = blur(tt) + 0.02 * torch.randn(tt.shape, device=dev, generator=g)
    p = ffst.Plan(n, n, 5, device=dev)
    deconv.deconvolve(y, p, blur, steps=3)  # warm-up
    torch.cuda.synchronize(dev)
    stream = torch.cuda.current_stream(dev)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    x, hist = deconv.deconvolve(y, p, blur, steps=steps)
    b.record(stream)
    torch.cuda.synchronize(dev)
    ms = a.elapsed_time(b) / steps
    cps = 2 * p.num_planes * n * n
    e_y = float(torch.linalg.norm(y - tt) / torch.linalg.norm(tt))
    e_x = float(torch.linalg.norm(x - tt) / torch.linalg.norm(tt))
    p.close()
    return {"value": 1e3 / ms, "unit": "FISTA steps/s", "ms_per_step": ms, "steps": steps,
            "size": "1024x1024, J=5", "transform_coeffs_per_s": cps / (ms / 1e3),
            "vs_plain": cps / (ms / 1e3) / plain_value,
            "note": "per step: objective with one forward, gradient by autograd (ffst_adjoint), blur by torch.fft",
            "objective": {"first": hist[0], "last": hist[-1]},
            "accuracy": {"rel_l2_to_truth_observed": e_y, "rel_l2_to_truth_restored": e_x}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the adjoint / f16 / bf16 / stats / complex / smooth / odd-size / batched forms")
    ap.add_argument("--shard", default="replicas", choices=["replicas", "planes"],
                    help="N > 1: independent replicas per GPU (weak scaling, default) or one image with its planes "
                         "split over the GPUs (strong scaling, one sum-reduce per inverse)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.shard == "planes" and _dist()[0] > 1:
        return run_sharded(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
