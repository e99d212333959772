#!/usr/bin/env python3
"""Benchmark of the MLBA hot path on GB300.

Workload (default): 64 independent deblurring problems of mixed size
n in {128, 192, 256, 384, 512, 768, 1024}, PSF (Gaussian / disk / motion),
boundary treatment (periodic / reflective / rectangular) and noise, FP32 with
FP64 norms / denominators / alpha_n, 2-level framelets; BC problems run
Algorithm 4-NS and rectangular ones Algorithm 1.  All problems advance
together: one step = one CUDA-graph launch = one MLBA iteration (residual and
stop test, preconditioner, adjoint, fused framelet update) of every problem.
The discrepancy rule is evaluated every step but does not stop the timed run,
so every step does the same work.  The working set (~2.7 GB of Bregman
variable alone) is far larger than L2.

Metric: megapixel-iterations per second (sum of observed n^2 per step).
`python bench.py --gpus N --steps K --warmup W [--impl reference]`.

`--config {1,2,3,5,l4}` measures one of the single-image workloads instead
(64x64 FP64; 256x256 reflective 4-NS to the discrepancy stop; 1024x1024
rectangular Rect1/2/3 with BF16 z; 4096x4096 rectangular 500 nonstationary
iterations; the 4096x4096 image with 4 framelet levels) and prints its own
line.  The default run also appends a compact record of those workloads
(`per_config`) to its one line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import mlba_inputs as I  # noqa: E402

METRIC = "MLBA megapixel-iterations/s and % HBM roofline, FP32-batched vs FP64 plain at equal RRE"
UNIT = "Mpix-it/s"
WORKLOAD = ("batch of 64 problems, n in {128..1024}, mixed Gaussian/disk/motion PSF, "
            "periodic/reflective/rectangular, FP32 + FP64 islands, L=2, Alg 4-NS (BC) / Alg-Rect1")


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def problems_for_rank(rank: int, count: int = 64):
    """Each rank gets its own independent batch (weak scaling, no exchange)."""
    return I.batch_problems(count=count, seed=4 + 1000 * rank)


def reduce_rank_metrics(ms: float, mpix: float, dist=None, device="cpu"):
    """(max elapsed ms over ranks, total megapixels per step over ranks)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return ms, mpix
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    m = torch.tensor([mpix], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(m, op=dist.ReduceOp.SUM)
    return float(t.item()), float(m.item())


# framelet tile shape: 2 = timed at create on the batch's own buffers (the
# shapes compute the same values; set by --autotune)
AUTOTUNE = 2
LAST_TILES = {}       # framelet tiles of the last single-problem run


def descs(probs):
    return [dict(psf=p.psf, g=p.g.astype(np.float32), delta=p.delta, bc=p.bc, precond=p.precond,
                 mu=p.mu, alpha=p.alpha) for p in probs]


def frame_bytes(probs, zbytes=4, tbytes=4, levels=2):
    """Algorithmic bytes of one fused framelet launch: z read + write, u read,
    f write, per problem."""
    tot = 0
    for p in probs:
        nb = 8 * levels + 1
        nf2 = p.nf * p.nf
        u = (p.n + p.p - 1) ** 2 if p.bc == "rect" else p.n * p.n
        tot += 2 * nb * zbytes * nf2 + tbytes * u + tbytes * nf2
    return tot


def step_min_bytes(probs, zbytes=4, b=4, levels=2):
    """Minimal HBM bytes of one iteration of the fused schedule:
    2 B bz Nf^2 (z) + 2 b Nf^2 (f) + b n^2 (g) + 6 b n^2 (transform passes, t)."""
    tot = 0
    for p in probs:
        nb = 8 * levels + 1
        tot += 2 * nb * zbytes * p.nf ** 2 + 2 * b * p.nf ** 2 + b * p.n ** 2 + 6 * b * p.n ** 2
    return tot


def src_hash(*names):
    h = hashlib.sha256()
    for nme in names:
        with open(os.path.join(ROOT, "paper_1504_07234_gb300", "csrc", nme), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi samples during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def ncu_traffic(kernel_hash, shape=0):
    """DRAM bytes of one frame-kernel launch from the committed ncu summary,
    scaled to the bench workload; null if the kernel changed since or the
    launch uses another tile shape than the captured one."""
    path = os.path.join(ROOT, "profiles", "frame_traffic.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    if d.get("kernel_hash") != kernel_hash or d.get("tile_shape", 0) != shape:
        return None
    return d.get("bytes_per_launch_bench")


def cpu_model():
    """The host CPU's model string and logical core count."""
    name = None
    try:
        for line in open("/proc/cpuinfo"):
            key = line.split(":")[0].strip().lower()
            if key in ("model name", "cpu model", "hardware"):
                name = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    if not name:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.lower().startswith("model name"):
                    name = line.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    return name or "unknown", os.cpu_count() or 1


def _oracle_job(args):
    """One worker's share of the oracle sample: run the oracle as it stands on
    problem i for `iters` iterations; returns (i, seconds)."""
    i, seed, count, iters = args
    from oracle import mlba_oracle as O
    p = I.batch_problems(count=count, seed=seed)[i]
    t0 = time.perf_counter()
    O.mlba(p.g, p.psf, p.delta, p.bc, p.precond, p.mu, p.alpha, p.levels, iters, stop=False,
           q=p.q, rho=p.rho)
    return i, time.perf_counter() - t0


def oracle_pool(jobs, workers):
    """Run oracle jobs on `workers` host processes (spawned: no state of this
    process, GPU context included, is inherited)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        return pool.map(_oracle_job, jobs, chunksize=1)


def oracle_sample(probs, seed, count, iters=2, budget_s=20.0):
    """Time the oracle as it stands on the host cores: one process per core,
    each running whole problems of the batch for `iters` iterations.  The
    sample is the whole batch when it fits the budget (estimated from the
    first wave), else the first problems."""
    name, ncpu = cpu_model()
    workers = max(1, min(ncpu, 16, len(probs)))
    t0 = time.perf_counter()
    first = oracle_pool([(i, seed, count, iters) for i in range(workers)], workers)
    el = time.perf_counter() - t0
    per_mpix = el / max(sum(probs[i].n ** 2 for i, _ in first) / 1e6, 1e-9)
    rest = []
    spent = el
    for i in range(workers, len(probs)):
        cost = per_mpix * probs[i].n ** 2 / 1e6 / workers
        if spent + cost > budget_s:
            break
        rest.append(i)
        spent += cost
    if rest:
        t1 = time.perf_counter()
        oracle_pool([(i, seed, count, iters) for i in rest], workers)
        el += time.perf_counter() - t1
    used = list(range(workers)) + rest
    mpix_it = sum(probs[i].n ** 2 for i in used) * iters / 1e6
    return {"value": mpix_it / el, "unit": UNIT, "cores": workers, "kind": "oracle",
            "cpu": name, "nproc": ncpu,
            "sample": f"oracle (FP64 numpy) {iters} iterations of {len(used)} of the "
                      f"{len(probs)} problems, one process per core, {el:.1f} s"}


def run_reference(args):
    """The oracle as it stands, on the same 64-problem workload, spread over
    the host cores (one process per core, whole problems each).  Iterations
    W .. W + K of every problem of the sample are timed as the difference of a
    W-iteration and a (W + K)-iteration run.  The sample is the whole batch
    when that fits about a minute, else the first problems."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    seed, count = 4, 64
    probs = problems_for_rank(0)
    name, ncpu = cpu_model()
    workers = max(1, min(ncpu, 16))
    W, K = args.warmup, args.steps
    # calibrate on one wave, then size the sample
    t0 = time.perf_counter()
    oracle_pool([(i, seed, count, 1) for i in range(workers)], workers)
    cal = (time.perf_counter() - t0) / max(sum(probs[i].n ** 2 for i in range(workers)), 1)
    used, cost = [], 0.0
    for i in range(count):
        c = cal * probs[i].n ** 2 * (2 * W + K) / workers
        if used and cost + c > 60.0:
            break
        used.append(i)
        cost += c
    t0 = time.perf_counter()
    oracle_pool([(i, seed, count, W) for i in used], workers)
    t1 = time.perf_counter()
    oracle_pool([(i, seed, count, W + K) for i in used], workers)
    t2 = time.perf_counter()
    el = max((t2 - t1) - (t1 - t0), 1e-9)
    mpix = sum(probs[i].n ** 2 for i in used) / 1e6
    value = mpix * K / el
    sample = (f"oracle (FP64 numpy) iterations {W}..{W + K} of {len(used)} of the {count} problems "
              f"(every problem when it fits), {workers} processes")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": K, "warmup": W, "ms_per_step": 1e3 * el / K,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "problems": count},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle",
                             "cpu": name, "nproc": ncpu, "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="mlba", choices=["mlba", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle baseline leg")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 plain comparison")
    ap.add_argument("--one-group", action="store_true",
                    help="advance the whole batch launch by launch (no two-group schedule)")
    ap.add_argument("--persistent", action="store_true",
                    help="the K steps as one persistent cooperative launch (grid barriers "
                         "between the stages) instead of the captured graphs")
    ap.add_argument("--blur-path", default="direct", choices=["direct", "fft", "auto"],
                    help="how A and A^T are applied: direct stencils (default), FFT convolution, "
                         "or per problem the faster of the two (timed at create)")
    ap.add_argument("--autotune", type=int, default=2, choices=[0, 1, 2],
                    help="framelet tile shape: 0 built-in, 1 timed at create or read from the "
                         "on-disk cache, 2 timed at create (default)")
    ap.add_argument("--problems", type=int, default=64,
                    help="first K problems of the batch (small cases for profiling)")
    ap.add_argument("--config", default="4", choices=["4", "1", "2", "3", "5", "l4"],
                    help="workload: 4 = the 64-problem batch (default); 1, 2, 3, 5, l4 = the "
                         "single-image workloads")
    ap.add_argument("--size", type=int, default=None,
                    help="single-image workloads: run at this n instead (profiling)")
    ap.add_argument("--iters", type=int, default=None,
                    help="single-image workloads 1, 3, 5, l4: iteration budget (profiling)")
    ap.add_argument("--no-configs", action="store_true",
                    help="default run: skip the per-config record of the single-image workloads")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    global AUTOTUNE, SIZE
    AUTOTUNE = args.autotune
    SIZE = args.size
    if args.impl == "reference":
        return run_reference(args)
    if args.config != "4":
        return run_single_config(args)

    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    from paper_1504_07234_gb300.build import build
    if rank == 0:
        build()
    if dist is not None:
        dist.barrier()
    import paper_1504_07234_gb300 as M

    probs = problems_for_rank(rank)[: args.problems]
    mpix = sum(p.n * p.n for p in probs) / 1e6
    K, W = args.steps, args.warmup
    reps_prof = 20
    max_iter = W + K + 2 * reps_prof + 20
    batch = M.Batch(descs(probs), dtype="f32", levels=2, stop=False, max_iter=max_iter,
                    rect_ns_hybrid=True, two_group=not args.one_group,
                    persistent=args.persistent, autotune=AUTOTUNE, blur_path=args.blur_path)
    stream = batch.stream
    # warm-up
    batch.iterate(W)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    batch.iterate(K)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    ck = clocks.stop()
    ms = e0.elapsed_time(e1)
    ms, mpix_all = reduce_rank_metrics(ms, mpix, dist, device="cuda")
    ms_step = ms / K
    value = mpix_all * K / (ms / 1e3)

    # per-kernel timing of the dominant kernel (fused framelet) and the others
    batch.reset()
    stage_ms = {}
    for stage, name in ((4, "frame"), (3, "adjoint_corr"), (2, "preconditioner"), (1, "residual")):
        batch.reset()
        stage_ms[name] = batch.profile(stage, reps_prof)
    batch.reset()
    kernels = batch.graph_kernels()
    tiles = batch.tiles()
    shape = tiles["frame_shape"]
    hbm, peak_kind = measured_peaks()
    fb = frame_bytes(probs)
    achieved = fb / (stage_ms["frame"] / 1e3) / 1e9
    khash = src_hash("k_frame.cu")
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": ncu_traffic(khash, shape),
                "kernel": f"k_frame3<float, float, 2> (tile shape {shape})",
                "peak_kind": peak_kind, "algorithmic_bytes_per_launch": fb}
    bmin = step_min_bytes(probs)
    step_frac = bmin / (ms_step / 1e3) / 1e9 / hbm

    # end to end through the public API with host buffers (pinned)
    pinned_g = [torch.from_numpy(d["g"]).pin_memory() for d in descs(probs)]
    pinned_f = [torch.empty((p.nf, p.nf), dtype=torch.float32).pin_memory() for p in probs]
    h2d = sum(x.numel() * 4 for x in pinned_g)
    d2h = sum(x.numel() * 4 for x in pinned_f)
    gs, fs, deltas = [x.numpy() for x in pinned_g], [x.numpy() for x in pinned_f], [p.delta for p in probs]
    # host-timed, so the median of three identical call sequences
    reps = []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        batch.set_data_all(gs, deltas)
        batch.reset()
        batch.iterate(K)
        batch.result_all(fs)
        torch.cuda.synchronize()
        reps.append(time.perf_counter() - t0)
    e2e_s = sorted(reps)[1]
    # whole job: every rank's pixels over the slowest rank's time
    e2e_ms, e2e_mpix = reduce_rank_metrics(e2e_s * 1e3, mpix, dist, device="cuda")
    e2e_s = e2e_ms / 1e3
    e2e = {"value": e2e_mpix * K / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d / K,
           "d2h_bytes_per_step": d2h / K,
           "note": f"median of 3 call sequences, each = upload of every g (one call), reset, "
                   f"{K} iterations, download of every f (one call)",
           "sequences_s": reps}
    batch.close()

    extra = {}
    if rank == 0 and not args.no_fp64:
        extra["fp64_plain"] = fp64_plain_vs_fp32(M, probs, torch)
    if rank == 0 and not args.no_configs and len(probs) == 64:
        extra["per_config"] = {c: measure_config(M, torch, c, compact=True)
                               for c in ("1", "2", "3", "5", "l4")}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = oracle_sample(probs, seed=4, count=64)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": W,
                "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD if len(probs) == 64 else f"first {len(probs)} problems of: " + WORKLOAD,
                           "problems": len(probs), "mpix_per_step_per_gpu": mpix,
                           "l2": "inputs larger than L2 (Bregman variable ~2.7 GB)",
                           "parallelism": f"replicas x{ws}, problems sharded",
                           "schedule": "one persistent launch for the K steps" if args.persistent
                           else "one group" if args.one_group else
                           "two groups half a step apart on two streams",
                           "frame_tiles": tiles, "blur_path": args.blur_path},
                "clocks": ck, "e2e": e2e, "gpu_launches": 1 if args.persistent else kernels * K,
                "roofline": roofline,
                "step_roofline": {"min_bytes": bmin, "frac": step_frac, "peak": hbm},
                "stage_ms": stage_ms, "cpu_baseline": cpu}
        line.update(extra)
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# single-image workloads 1, 2, 3 and 5, and workload 5 at four levels

def frame_bytes_one(p, levels, zbytes, tbytes):
    """Algorithmic bytes of one framelet launch for one problem: z read and
    written, u read (the correlation for rectangular A, t otherwise), f
    written."""
    nb = 8 * levels + 1
    nf2 = p.nf * p.nf
    u = (p.n + p.p - 1) ** 2 if p.bc == "rect" else p.n * p.n
    return 2 * nb * zbytes * nf2 + tbytes * u + tbytes * nf2


def stage_bytes_one(p, tbytes):
    """Algorithmic bytes of the other launches of one step for one problem:
    residual (f, g read, r written), correlation (t read, the (n+p-1)^2
    correlation written), spectral preconditioner (rows: r read, spectrum
    written; columns: spectrum read and written, sigma read; rows: spectrum
    read, t written; the half spectrum is n (n/2+1) complex for the DFT, n^2
    real for the DCT, i.e. about n^2 values either way)."""
    n2, ne2 = p.n * p.n, (p.n + p.p - 1) ** 2
    out = {"residual": tbytes * (p.nf * p.nf + 2 * n2)}
    # Algorithm 4 / 4-NS with a BC apply C^T inside the preconditioner: no A^T
    if p.bc == "rect" or p.precond not in ("tikh", "tikh_ns"):
        out["adjoint_corr"] = tbytes * (n2 + ne2)
    if p.precond != "none":
        out["preconditioner"] = tbytes * (n2 + n2 + 3 * n2 + n2 + n2)
    return out


SIZE = None          # --size: a single-image workload at another n (profiling)


def _single_problem(c, variant=None):
    if c == "l4":
        pr = I.config(5, n=SIZE)
        pr.levels = 4
        pr.name = "C5-L4"
        return pr
    return I.config(int(c), variant=variant, n=SIZE)


def _run_batch(M, torch, pr, dtype, iters, z_store=None, warm=0, stop=None, profile=False):
    """One problem as a batch of one: device time of `iters` steps after
    `warm` steps (CUDA events on the library stream), the result and stats;
    optionally the per-stage launch times."""
    d = dict(psf=pr.psf, g=pr.g.astype(np.float32 if dtype == "f32" else np.float64),
             delta=pr.delta, bc=pr.bc, precond=pr.precond, mu=pr.mu, alpha=pr.alpha,
             transform=pr.transform, max_iter=warm + iters)
    b = M.Batch([d], dtype=dtype, z_store=z_store, levels=pr.levels,
                stop=pr.stop if stop is None else stop, max_iter=warm + iters, gamma=pr.gamma,
                q=pr.q, rho=pr.rho, rect_ns_hybrid=pr.rect_ns_hybrid, autotune=AUTOTUNE)
    steps = iters + 1             # the last step only evaluates the final residual
    if stop:
        # time exactly the steps up to the discrepancy stop (found by an
        # untimed run), not the idle launches after it
        b.iterate(steps)
        steps = b.stats(0)["iter"] + 1
        b.reset()
    if warm:
        b.iterate(warm)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(b.stream)
    b.iterate(steps)
    e1.record(b.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    st = b.stats(0)
    f = b.result(0).astype(np.float64)
    stages = None
    if profile:
        stages = {}
        for stage, name in ((4, "frame"), (3, "adjoint_corr"), (2, "preconditioner"), (1, "residual")):
            b.reset()
            stages[name] = b.profile(stage, 10)
    kern = b.graph_kernels()
    LAST_TILES.clear()
    LAST_TILES.update(b.tiles())
    b.close()
    return ms, st, f, stages, kern


def _e2e(M, torch, pr, dtype, iters, z_store=None):
    """The same run through the public API with host buffers: pinned g
    uploaded, iterations, f downloaded, all inside the timed region."""
    npd = np.float32 if dtype == "f32" else np.float64
    g = torch.from_numpy(pr.g.astype(npd)).pin_memory()
    fo = torch.empty((pr.nf, pr.nf), dtype=torch.float32 if dtype == "f32" else torch.float64).pin_memory()
    d = dict(psf=pr.psf, g=g.numpy(), delta=pr.delta, bc=pr.bc, precond=pr.precond, mu=pr.mu,
             alpha=pr.alpha, transform=pr.transform, max_iter=iters)
    b = M.Batch([d], dtype=dtype, z_store=z_store, levels=pr.levels, stop=pr.stop,
                max_iter=iters, gamma=pr.gamma, q=pr.q, rho=pr.rho, rect_ns_hybrid=pr.rect_ns_hybrid,
                autotune=AUTOTUNE)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.set_data(0, g.numpy(), pr.delta)
    b.reset()
    b.iterate(iters + 1)
    b.result(0, out=fo.numpy())
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    done = b.stats(0)["iter"]
    b.close()
    return {"value": pr.n * pr.n * max(done, 1) / 1e6 / el, "unit": UNIT,
            "h2d_bytes_per_step": g.numel() * g.element_size() / max(done, 1),
            "d2h_bytes_per_step": fo.numel() * fo.element_size() / max(done, 1)}


def _quality(f, pr):
    t = pr.truth_in_fov()
    return {"rre": float(np.linalg.norm(f - t) / np.linalg.norm(t)),
            "psnr": float(20 * np.log10(t.shape[0] / np.linalg.norm(f - t)))}


def measure_config(M, torch, c, compact=False, iters=None, warm=5):
    """Measure one single-image workload; returns its record (value in
    Mpix-it/s of the observed image, roofline of the framelet launch, per
    stage fractions, and the precision comparison the workload asks for)."""
    hbm, peak_kind = measured_peaks()
    out = {"workload": I.CONFIG_NAMES.get(int(c), "") if c != "l4" else
           "rect 4096x4096, 31x31 Gaussian sigma=5, DCT + NS alpha, L=4 (the paper's level count)"}
    if SIZE:
        out["workload"] += f" (run at n = {SIZE})"
    if c == "1":
        pr = _single_problem(c)
        it = iters or pr.max_iter
        ms, st, f, stg, kern = _run_batch(M, torch, pr, "f64", it, profile=not compact)
        out["frame_tiles"] = dict(LAST_TILES)
        out.update(dtype="f64", iters=it, value=pr.n ** 2 * it / 1e6 / (ms / 1e3),
                   ms_per_iter=ms / (it + 1), quality=_quality(f, pr), graph_kernels=kern,
                   note="launch-latency bound (1.06 MB of compulsory traffic per iteration)")
        fp32 = _run_batch(M, torch, pr, "f32", it)
        out["fp32"] = {"value": pr.n ** 2 * it / 1e6 / (fp32[0] / 1e3),
                       "rre_diff_vs_fp64": abs(_quality(fp32[2], pr)["rre"] - out["quality"]["rre"])}
        main = ("f64", pr, it, None)
    elif c == "2":
        pr = _single_problem(c)
        ms, st, f, stg, kern = _run_batch(M, torch, pr, "f32", pr.max_iter, stop=True, profile=not compact)
        out["frame_tiles"] = dict(LAST_TILES)
        it = max(st["iter"], 1)
        ms64, st64, f64, _, _ = _run_batch(M, torch, pr, "f64", pr.max_iter, stop=True)
        q32, q64 = _quality(f, pr), _quality(f64, pr)
        out.update(dtype="f32", iters=st["iter"], stop_iter=st["stop_iter"],
                   value=pr.n ** 2 * it / 1e6 / (ms / 1e3), ms_per_iter=ms / (it + 1),
                   quality=q32, graph_kernels=kern,
                   fp64={"stop_iter": st64["stop_iter"], "quality": q64,
                         "value": pr.n ** 2 * max(st64["iter"], 1) / 1e6 / (ms64 / 1e3)},
                   rre_diff_vs_fp64=abs(q32["rre"] - q64["rre"]),
                   psnr_diff_vs_fp64=abs(q32["psnr"] - q64["psnr"]))
        main = ("f32", pr, pr.max_iter, None)
    elif c == "3":
        res = {}
        it = iters or 200
        main_ms = main_kern = None
        for v in ("rect1", "rect2", "rect3"):
            pr = _single_problem(c, v)
            ms, st, f, stg, kern = _run_batch(M, torch, pr, "f32", it, warm=0)
            msb, stb, fb, _, kernb = _run_batch(M, torch, pr, "f32", it, z_store="bf16", warm=0)
            if v == "rect1":
                main_ms, main_kern = msb, kernb
                out["frame_tiles"] = dict(LAST_TILES)
            ms64, _, f64, _, _ = _run_batch(M, torch, pr, "f64", it, warm=0)
            q, qb, q64 = _quality(f, pr), _quality(fb, pr), _quality(f64, pr)
            res[v] = {"value_fp32z": pr.n ** 2 * it / 1e6 / (ms / 1e3),
                      "value_bf16z": pr.n ** 2 * it / 1e6 / (msb / 1e3),
                      "value_fp64": pr.n ** 2 * it / 1e6 / (ms64 / 1e3),
                      "quality_fp32z": q, "quality_bf16z": qb, "quality_fp64": q64,
                      "bf16z_rel_f_err_vs_fp64": float(np.abs(fb - f64).max() / np.abs(f64).max()),
                      "fp32z_rel_f_err_vs_fp64": float(np.abs(f - f64).max() / np.abs(f64).max())}
        out.update(dtype="f32 (bf16 z)", iters=it, variants=res,
                   value=res["rect1"]["value_bf16z"], ms_per_iter=main_ms / (it + 1),
                   graph_kernels=main_kern,
                   note="equal budget of 200 iterations; Rect1 = BCCB (DFT), Rect2 = PCG, "
                        "Rect3 = symmetrised PSF (DCT); the FP64 reference is the library's FP64 "
                        "path (pinned to the oracle at smaller sizes)")
        pr = _single_problem(c, "rect1")
        main = ("f32", pr, it, "bf16")
    else:   # "5", "l4"
        pr = _single_problem(c)
        it = iters or (pr.max_iter if c == "5" else 50)
        ms, st, f, stg, kern = _run_batch(M, torch, pr, "f32", it, warm=0, profile=True)
        out["frame_tiles"] = dict(LAST_TILES)
        out.update(dtype="f32", iters=it, value=pr.n ** 2 * it / 1e6 / (ms / 1e3),
                   ms_per_iter=ms / (it + 1), quality=_quality(f, pr), stop_iter=st["stop_iter"],
                   graph_kernels=kern)
        if c == "5":
            ms64, st64, f64, _, _ = _run_batch(M, torch, pr, "f64", it, warm=0)
            q64 = _quality(f64, pr)
            out["fp64"] = {"quality": q64, "value": pr.n ** 2 * it / 1e6 / (ms64 / 1e3)}
            out["rre_diff_vs_fp64"] = abs(out["quality"]["rre"] - q64["rre"])
            out["rel_f_err_vs_fp64"] = float(np.abs(f - f64).max() / np.abs(f64).max())
        main = ("f32", pr, it, None)
    dtype, pr, it, zst = main
    if stg is None:
        _, _, _, stg, _ = _run_batch(M, torch, pr, dtype, 8, z_store=zst, warm=0, profile=True)
    tb = 8 if dtype == "f64" else 4
    zb = 8 if dtype == "f64" else (2 if zst == "bf16" else 4)
    fb = frame_bytes_one(pr, pr.levels, zb, tb)
    ach = fb / (stg["frame"] / 1e3) / 1e9
    out["roofline"] = {"bound": "hbm", "kernel": "k_frame3" if pr.levels <= 2 else "k_lowpass + k_frame_lev (per level)",
                       "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                       "peak_kind": peak_kind, "algorithmic_bytes_per_launch": fb}
    sb = stage_bytes_one(pr, tb)
    out["stage_ms"] = {k: v for k, v in stg.items() if k in sb or k == "frame"}
    out["stage_frac"] = {k: sb[k] / (stg[k] / 1e3) / 1e9 / hbm for k in sb if stg.get(k)}
    if not compact:
        out["e2e"] = _e2e(M, torch, pr, dtype, it, z_store=zst)
    return out


def run_single_config(args):
    import torch
    ws, rank, local = dist_env()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    from paper_1504_07234_gb300.build import build
    build()
    import paper_1504_07234_gb300 as M
    c = args.config
    cpu = None
    if not args.no_cpu:
        cpu = oracle_config_sample(c)
    clocks = ClockSampler(local)
    clocks.start()
    rec = measure_config(M, torch, c, iters=args.iters)
    ck = clocks.stop()
    pr = _single_problem(c, "rect1" if c == "3" else None)
    line = {"metric": METRIC, "value": rec["value"], "unit": UNIT, "n_gpus": 1,
            "steps": rec["iters"], "warmup": 0,
            "ms_per_step": rec.get("ms_per_iter"), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": rec["dtype"], "data": "synthetic",
            "config": {"workload": rec["workload"], "n": pr.n, "p": pr.p, "levels": pr.levels,
                       "l2": "inputs larger than L2" if pr.n >= 1024 else "inputs fit in L2"},
            "clocks": ck, "e2e": rec.get("e2e"), "gpu_launches": rec.get("graph_kernels", 0) * rec["iters"],
            "roofline": rec["roofline"], "cpu_baseline": cpu, "record": rec}
    print(json.dumps(line))
    return 0


def oracle_config_sample(c):
    """The oracle as it stands on a bounded sample of a single-image workload
    (two iterations; the 4096 x 4096 images are sampled at 512 x 512)."""
    from oracle import mlba_oracle as O
    name, ncpu = cpu_model()
    if c in ("5", "l4"):
        pr = I.config(5, n=512)
        if c == "l4":
            pr.levels = 4
    elif c == "3":
        pr = I.config(3, variant="rect1", n=256)
    else:
        pr = I.config(int(c))
    iters = 2
    t0 = time.perf_counter()
    O.mlba(pr.g, pr.psf, pr.delta, pr.bc, pr.precond, pr.mu, pr.alpha, pr.levels, iters,
           stop=False, q=pr.q, rho=pr.rho, transform=pr.transform, rect_ns_hybrid=pr.rect_ns_hybrid)
    el = time.perf_counter() - t0
    return {"value": pr.n ** 2 * iters / 1e6 / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "cpu": name, "nproc": ncpu,
            "sample": f"oracle (FP64 numpy, one process) {iters} iterations of the workload at "
                      f"{pr.n}x{pr.n}, {el:.1f} s"}


def fp64_plain_vs_fp32(M, probs, torch, count=4, iters=40):
    """FP64 plain per-image GPU path vs the FP32 batched path on the same
    problems at a fixed iteration budget: iterations/s and RRE."""
    def rre(f, t):
        return float(np.linalg.norm(f - t) / np.linalg.norm(t))

    sel = sorted(range(len(probs)), key=lambda i: probs[i].n)[:: max(1, len(probs) // count)][:count]
    out = {"problems": sel, "iters": iters}
    rre32, rre64, t64 = [], [], 0.0
    sub = [probs[i] for i in sel]
    b = M.Batch(descs(sub), dtype="f32", levels=2, stop=False, max_iter=iters, rect_ns_hybrid=True)
    torch.cuda.synchronize()
    s0 = time.perf_counter()
    b.iterate(iters + 1)
    torch.cuda.synchronize()
    t32 = time.perf_counter() - s0
    for k, p in enumerate(sub):
        rre32.append(rre(b.result(k).astype(np.float64), p.truth_in_fov()))
    b.close()
    for p in sub:
        c = M.Context(p.psf, p.n, p.bc, p.precond, dtype="f64", mu=p.mu, alpha=p.alpha, levels=2,
                      max_iter=iters, stop=False, rect_ns_hybrid=True)
        c.set_data(p.g, p.delta)
        torch.cuda.synchronize()
        s0 = time.perf_counter()
        c.iterate(iters + 1)
        c.stream.synchronize()
        t64 += time.perf_counter() - s0
        rre64.append(rre(c.result(), p.truth_in_fov()))
        c.close()
    mp = sum(p.n * p.n for p in sub) / 1e6
    out["fp32_batched_mpix_it_s"] = mp * iters / t32
    out["fp64_plain_mpix_it_s"] = mp * iters / t64
    out["max_abs_rre_diff"] = float(max(abs(a - b_) for a, b_ in zip(rre32, rre64)))
    return out


if __name__ == "__main__":
    sys.exit(main())
