"""Benchmark of the GCP-Adam sampled-gradient path on one GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload: dense 100x100x100x100 FP32 tensor (1e8 entries, 400 MB), planted
rank 10 plus N(0, 0.01) noise; Gaussian loss; uniform sampling with 1e5
sampled entries per iteration; loss estimate on a fixed set of 1e5 entries.
One step is one GCP-Adam epoch (Alg. 4): tau = 100 iterations of (fused
sample + gradient, Adam step), the loss estimate, accept-or-revert; the epoch
is captured once as a CUDA graph and replayed.  Metric: sampled-gradient
entries processed per second (tau * s per step).

Rank r of an N-rank run (torchrun) fits its own replica (seed + r): the path
has no exchange step between independent decompositions ("replicas only").
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "sampled-gradient entries/s"
UNIT = "entries/s"
WORKLOAD = "dense-100x100x100x100-r10-gaussian-uniform-s1e5"
DIMS, RANK, S_DRAWS, EST_DRAWS, TAU = (100, 100, 100, 100), 10, 100_000, 100_000, 100
# Algorithmic bytes per draw of the gradient kernel: generated indices (0 B),
# the dense value (4 B), the d row gathers and the d row updates of r FP32
# entries each: 4 + d*r*4 + d*r*4.
BYTES_PER_DRAW = 4 + 2 * len(DIMS) * RANK * 4


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = []
        for line in (self.out or "").strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), max=float(parts[2]), power=float(parts[3]),
                                 hw=parts[5], hwt=parts[6], swt=parts[7], cap=parts[8]))
            except ValueError:
                continue
        if not rows:
            return None
        reasons = set()
        for r in rows:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("cap", "sw_power_cap")):
                if r[key].lower() == "active":
                    reasons.add(name)
        loaded = [r["sm"] for r in rows if r["power"] > 200] or [r["sm"] for r in rows]
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(r["max"] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows)}


# ---------------------------------------------------------------------------
# the FP64 oracle on the host cores (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------

def oracle_tensor(X32):
    import oracle
    return oracle.Tensor(DIMS, dense=X32.astype(np.float64).reshape(-1))


def oracle_epoch_rate(XO, A0, budget_s=12.0, seed=1687):
    """Entries/s of the oracle doing the same epoch: tau iterations of
    (sample, gradient, Adam) plus one loss estimate, extrapolated from a
    bounded number of iterations and one estimate."""
    import oracle
    A = oracle.concat_factors([a.astype(np.float64) for a in A0])
    B, C = np.zeros_like(A), np.zeros_like(A)
    t0 = time.perf_counter()
    est = oracle.sample(XO, oracle.UNIFORM, 0, EST_DRAWS, 7, 2**64 - 1)
    oracle.loss_estimate(DIMS, oracle.split_factors(A, DIMS, RANK), oracle.GAUSSIAN, est)
    t_est = time.perf_counter() - t0
    iters, t_it = 0, 0.0
    while t_it < budget_s and iters < TAU:
        t0 = time.perf_counter()
        S = oracle.sample(XO, oracle.UNIFORM, 0, S_DRAWS, seed, iters)
        G = oracle.concat_factors(oracle.grad(DIMS, oracle.split_factors(A, DIMS, RANK), oracle.GAUSSIAN, S))
        oracle.adam_step(A, B, C, G, 1e-3, t=iters)
        t_it += time.perf_counter() - t0
        iters += 1
    per_it = t_it / iters
    rate = TAU * S_DRAWS / (TAU * per_it + t_est)
    sample = (f"{iters} oracle iterations of {S_DRAWS} draws (sample + gradient + Adam) and one "
              f"{EST_DRAWS}-entry loss estimate, scaled to a {TAU}-iteration epoch")
    return rate, sample


def reference_arm(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    from paper_1906_01687_gb300 import synth
    X32, _ = synth.dense_100_4()
    A0 = synth.initial_guess(DIMS, RANK, seed=3, target_norm=float(np.linalg.norm(X32)))
    XO = oracle_tensor(X32)
    budget = max(1.0, min(20.0, 100.0 / max(1, args.steps + args.warmup)))
    rates = []
    for step in range(args.warmup + args.steps):
        rate, sample = oracle_epoch_rate(XO, A0, budget_s=budget)
        if step >= args.warmup:
            rates.append(rate)
    value = statistics.median(rates)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": TAU * S_DRAWS / value * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded planted model)",
            "config": {"workload": WORKLOAD, "dims": list(DIMS), "rank": RANK, "samples_per_iter": S_DRAWS,
                       "tau": TAU, "est_samples": EST_DRAWS},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# the CUDA path
# ---------------------------------------------------------------------------

def time_grad_kernel(torch, gcp, h, F, G, spec, stream, launches=200):
    """Average device duration of one gradient launch, from CUDA events on the
    launching stream around each launch, all queued behind a sleep so that
    the launches run back to back."""
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(launches)]
    with torch.cuda.stream(stream):
        torch.cuda._sleep(200_000_000)
        for i, (a, b) in enumerate(evs):
            s = gcp.Sampling(spec.kind, spec.p, spec.q, spec.seed, 10_000 + i, spec.problem, spec.oversample)
            a.record(stream)
            gcp.gcp_grad(h, F, gcp.LOSS_GAUSSIAN, G, S=s, stream=stream)
            b.record(stream)
    stream.synchronize()
    times = [a.elapsed_time(b) for a, b in evs]
    for g in G:
        g.zero_()
    return statistics.mean(times) * 1e-3, statistics.median(times) * 1e-3


def ours_arm(args):
    import torch
    from paper_1906_01687_gb300 import gcp, synth
    from paper_1906_01687_gb300.adam import GcpAdam

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)

    X32, _ = synth.dense_100_4()
    A0 = synth.initial_guess(DIMS, RANK, seed=3 + rank, target_norm=float(np.linalg.norm(X32)))
    XT = gcp.DataTensor.dense(X32, device=dev)
    seed = 1687 + rank
    with torch.cuda.stream(stream):
        run = GcpAdam(XT, A0, gcp.LOSS_GAUSSIAN, gcp.SAMPLER_UNIFORM, 0, S_DRAWS, 0, EST_DRAWS, seed=seed,
                      est_seed=7, alpha=1e-3, tau=TAU, kappa=1_000_000, stream=stream, autotune=not args.no_autotune)
        run.capture()
    for _ in range(args.warmup):
        run.run_epoch()
    stream.synchronize()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    # device-resident timed region: K replayed epochs
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        barrier()
        start.record(stream)
        for _ in range(args.steps):
            run.run_epoch()
        end.record(stream)
        barrier()
    elapsed = start.elapsed_time(end) * 1e-3
    st = run.status()
    if world > 1:
        t = torch.tensor([elapsed], device=dev, dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        elapsed = float(t.item())
    entries = args.steps * TAU * S_DRAWS * world
    value = entries / elapsed

    # end to end through the public API with host buffers: H2D of X and of the
    # initial factors from pinned memory, the epoch, D2H of F-hat and the factors
    X_pin = torch.from_numpy(X32.reshape(-1)).pin_memory()
    A_pin = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in A0]
    F_out = [torch.empty(a.shape, dtype=torch.float32).pin_memory() for a in A0]
    state_out = torch.empty(8, dtype=torch.float64).pin_memory()
    h2d = X_pin.numel() * 4 + sum(a.numel() * 4 for a in A_pin)
    d2h = state_out.numel() * 8 + sum(a.numel() * 4 for a in F_out)
    e_start, e_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e_start.record(stream)
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            XT.vals.copy_(X_pin, non_blocking=True)
            for a_dev, a_host in zip(run.F.A, A_pin):
                a_dev[:, :RANK].copy_(a_host, non_blocking=True)
            run.run_epoch()
            state_out.copy_(run.state, non_blocking=True)
            for a_host, a_dev in zip(F_out, run.F.A):
                a_host.copy_(a_dev[:, :RANK], non_blocking=True)
    e_end.record(stream)
    barrier()
    e2e_elapsed = e_start.elapsed_time(e_end) * 1e-3
    if world > 1:
        t = torch.tensor([e2e_elapsed], device=dev, dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_elapsed = float(t.item())
    e2e_value = entries / e2e_elapsed

    # the dominant kernel (the fused sampled gradient), timed alone
    G = run.F.like()
    mean_s, median_s = time_grad_kernel(torch, gcp, run.h, run.F, G, run.spec, stream)
    peak, peak_kind = peaks()
    achieved = BYTES_PER_DRAW * S_DRAWS / mean_s / 1e9
    launch = gcp.gcp_get_launch(run.h, run.F, S_DRAWS)

    if rank != 0:
        return 0
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded planted rank-10 model + N(0,0.01) noise)",
            "config": {"workload": WORKLOAD, "dims": list(DIMS), "rank": RANK, "loss": "gaussian",
                       "sampler": "uniform", "samples_per_iter": S_DRAWS, "tau": TAU, "est_samples": EST_DRAWS,
                       "step": "one GCP-Adam epoch (tau iterations + loss estimate + accept/revert), CUDA graph",
                       "l2": "inputs larger than L2 (X = 400 MB, gathered at random)",
                       "parallelism": f"replicas{world}", "grad_launch": launch,
                       "autotuned": run.tuned},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": args.steps * ((3 if any(r > 1 for r in launch["replicas"]) else 2) * TAU + 2),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "kernel": "gcp_grad (fused sampled gradient)",
                         "bytes_per_draw": BYTES_PER_DRAW, "draws_per_launch": S_DRAWS,
                         "launch_us_mean": mean_s * 1e6, "launch_us_median": median_s * 1e6,
                         "peak_source": f"{peak_kind} hbm_gbs"},
            "final_state": {k: st[k] for k in ("F", "t", "iter", "alpha", "bad")}}
    clocks = clk.summary()
    line["clocks"] = clocks
    if not args.no_cpu_baseline:
        rate, sample = oracle_epoch_rate(oracle_tensor(X32), A0, budget_s=args.cpu_budget)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample}
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        return reference_arm(args)
    return ours_arm(args)


if __name__ == "__main__":
    sys.exit(main())
