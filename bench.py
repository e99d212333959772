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


def ncu_traffic(kernel_hash):
    """DRAM bytes of one frame-kernel launch from the committed ncu summary,
    scaled to the bench workload; null if the kernel changed since."""
    path = os.path.join(ROOT, "profiles", "frame_traffic.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    if d.get("kernel_hash") != kernel_hash:
        return None
    return d.get("bytes_per_launch_bench")


def oracle_sample(probs, seconds=15.0, iters=2):
    """Time the oracle as it stands on the first problems of the batch."""
    from oracle import mlba_oracle as O
    t0 = time.perf_counter()
    mpix_it = 0.0
    used = []
    for i, p in enumerate(probs):
        O.mlba(p.g, p.psf, p.delta, p.bc, p.precond, p.mu, p.alpha, p.levels, iters, stop=False,
               q=p.q, rho=p.rho)
        mpix_it += p.n * p.n * iters / 1e6
        used.append(i)
        if time.perf_counter() - t0 > seconds:
            break
    el = time.perf_counter() - t0
    return mpix_it / el, el, used


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import mlba_oracle as O
    probs = problems_for_rank(0)
    smallest = min(range(len(probs)), key=lambda i: probs[i].n)
    p = probs[smallest]
    kw = dict(stop=False, q=p.q, rho=p.rho)
    t0 = time.perf_counter()
    O.mlba(p.g, p.psf, p.delta, p.bc, p.precond, p.mu, p.alpha, p.levels, args.warmup, **kw)
    t1 = time.perf_counter()
    O.mlba(p.g, p.psf, p.delta, p.bc, p.precond, p.mu, p.alpha, p.levels, args.warmup + args.steps, **kw)
    t2 = time.perf_counter()
    el = (t2 - t1) - (t1 - t0)
    el = max(el, 1e-9)
    value = p.n * p.n * args.steps / 1e6 / el
    sample = (f"oracle (FP64 numpy) iterations {args.warmup}..{args.warmup + args.steps} of problem "
              f"{smallest} ({p.n}x{p.n}, {p.bc}, {p.precond}) of the 64-problem batch")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "problems": 64},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
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
    ap.add_argument("--problems", type=int, default=64,
                    help="first K problems of the batch (small cases for profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

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
                    rect_ns_hybrid=True, two_group=not args.one_group)
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
    hbm, peak_kind = measured_peaks()
    fb = frame_bytes(probs)
    achieved = fb / (stage_ms["frame"] / 1e3) / 1e9
    khash = src_hash("k_frame.cu")
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": ncu_traffic(khash), "kernel": "k_frame3<float,float,2>",
                "peak_kind": peak_kind, "algorithmic_bytes_per_launch": fb}
    bmin = step_min_bytes(probs)
    step_frac = bmin / (ms_step / 1e3) / 1e9 / hbm

    # end to end through the public API with host buffers (pinned)
    pinned_g = [torch.from_numpy(d["g"]).pin_memory() for d in descs(probs)]
    pinned_f = [torch.empty((p.nf, p.nf), dtype=torch.float32).pin_memory() for p in probs]
    h2d = sum(x.numel() * 4 for x in pinned_g)
    d2h = sum(x.numel() * 4 for x in pinned_f)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i, p in enumerate(probs):
        batch.set_data(i, pinned_g[i].numpy(), p.delta)
    batch.reset()
    batch.iterate(K)
    for i in range(len(probs)):
        batch.result(i, out=pinned_f[i].numpy())
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e = {"value": mpix * K / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d / K,
           "d2h_bytes_per_step": d2h / K,
           "note": f"one call sequence = upload 64 g, reset, {K} iterations, download 64 f"}
    batch.close()

    extra = {}
    if rank == 0 and not args.no_fp64:
        extra["fp64_plain"] = fp64_plain_vs_fp32(M, probs, torch)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        v, el, used = oracle_sample(probs)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"oracle (FP64 numpy, 1 thread) 2 iterations of problems {used[0]}..{used[-1]} "
                         f"of the batch, {el:.1f} s"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": W,
                "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD if len(probs) == 64 else f"first {len(probs)} problems of: " + WORKLOAD,
                           "problems": len(probs), "mpix_per_step_per_gpu": mpix,
                           "l2": "inputs larger than L2 (Bregman variable ~2.7 GB)",
                           "parallelism": f"replicas x{ws}, problems sharded",
                           "schedule": "one group" if args.one_group else
                           "two groups half a step apart on two streams"},
                "clocks": ck, "e2e": e2e, "gpu_launches": kernels * K, "roofline": roofline,
                "step_roofline": {"min_bytes": bmin, "frac": step_frac, "peak": hbm},
                "stage_ms": stage_ms, "cpu_baseline": cpu}
        line.update(extra)
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


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
