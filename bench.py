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


KERNEL_SOURCES = ("gcp_grad_impl.cuh", "gcp_draw.cuh", "gcp_device.cuh", "gcp_kernels.cuh")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "grad_kernel_dense100_r10_s1e5.json")


def kernel_source_hash():
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1906_01687_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(launch):
    """DRAM bytes per launch of grad_kernel from the committed ncu summary, if
    the kernel sources and the kernel instance (lanes x chunks, draw layout,
    early draws) are those the counters were taken with; otherwise None.
    The block size is not compared: it changes neither the kernel's code nor
    its DRAM traffic, which is the random gathers of X."""
    try:
        with open(TRAFFIC_FILE) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    if rec.get("source_hash") != kernel_source_hash():
        return None
    keys = ("lanes", "chunks", "group_draws", "prefetch", "early_draws")
    if any(rec.get("launch_shape", {}).get(k) != launch.get(k) for k in keys):
        return None
    return rec.get("dram_bytes_per_launch")


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


def max_over_ranks(value, world, device="cpu"):
    """The slowest rank's time: every rank's value, all-reduced with MAX."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_seeds(rank):
    """Rank r fits its own replica: initial-guess seed 3 + r, draw seed 1687 + r
    (the estimate set, seed 7, is shared by all replicas)."""
    return 3 + rank, 1687 + rank


def whole_job_rate(units_per_rank, world, seconds):
    """Units all ranks processed per second of the slowest rank."""
    return units_per_rank * world / seconds


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

def time_grad_kernel(torch, gcp, run, stream, launches=200):
    """Average device duration of the fused-gradient kernel: the library
    records CUDA events on the launching stream around each kernel launch of
    `launches` GCP-Adam iterations, queued behind a sleep so that they run
    back to back as in the replayed epochs."""
    gcp.gcp_profile(run.h, True, launches)
    with torch.cuda.stream(stream):
        torch.cuda._sleep(200_000_000)
        for _ in range(launches):
            run.iteration()
    stream.synchronize()
    ms, n = gcp.gcp_profile_read(run.h, 0)
    ms_adam, n_adam = gcp.gcp_profile_read(run.h, 1)
    gcp.gcp_profile(run.h, False)
    return ms * 1e-3 / n, n, ms_adam * 1e-3 / max(n_adam, 1)


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
    # the end-to-end section's copy stream, taken now: torch hands out streams
    # round-robin from a small pool, and one taken after the autotuner's
    # captures can be the compute stream itself
    copy_stream = torch.cuda.Stream(device=dev)
    assert copy_stream.cuda_stream != stream.cuda_stream

    X32, _ = synth.dense_100_4()
    init_seed, seed = replica_seeds(rank)
    A0 = synth.initial_guess(DIMS, RANK, seed=init_seed, target_norm=float(np.linalg.norm(X32)))
    XT = gcp.DataTensor.dense(X32, device=dev)
    with torch.cuda.stream(stream):
        run = GcpAdam(XT, A0, gcp.LOSS_GAUSSIAN, gcp.SAMPLER_UNIFORM, 0, S_DRAWS, 0, EST_DRAWS, seed=seed,
                      est_seed=7, alpha=1e-3, tau=TAU, kappa=1_000_000, stream=stream,
                      autotune=not (args.no_autotune or args.tuning))
        if args.tuning:
            gcp.gcp_set_tuning(run.h, **json.loads(args.tuning))
            run.tuned = {"best": json.loads(args.tuning), "given": True}
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
    elapsed = max_over_ranks(start.elapsed_time(end) * 1e-3, world, dev)
    st = run.status()
    entries = args.steps * TAU * S_DRAWS * world
    value = whole_job_rate(args.steps * TAU * S_DRAWS, world, elapsed)

    # end to end through the public API with host buffers: every step copies X
    # and the initial factors from pinned memory, runs the epoch and reads
    # F-hat and the factors back.  X is double-buffered: step e + 1's copy (on
    # a copy stream, into the other device buffer, read by a second handle
    # and graph) runs while step e computes.  All host-to-device copies go
    # through the copy stream in step order (factors of step e, then X of step
    # e + 1), so that the small copies never queue behind a large one.
    X_pin = torch.from_numpy(X32.reshape(-1)).pin_memory()
    A_pin = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in A0]
    F_out = [torch.empty(a.shape, dtype=torch.float32).pin_memory() for a in A0]
    state_out = torch.empty(8, dtype=torch.float64).pin_memory()
    h2d = X_pin.numel() * 4 + sum(a.numel() * 4 for a in A_pin)
    d2h = state_out.numel() * 8 + sum(a.numel() * 4 for a in F_out)
    XT2 = gcp.DataTensor.dense(X32, device=dev)
    handles, graphs, xbufs = [run.h], [run.graph], [XT.vals, XT2.vals]
    with torch.cuda.stream(stream):
        h2 = gcp.Handle(XT2, stream=stream)
        gcp.gcp_set_tuning(h2, **(run.tuned["best"] if run.tuned else {"early_draws": 1}))
        run.h = h2
        run.capture()
    handles.append(h2)
    graphs.append(run.graph)
    run.h, run.graph = handles[0], graphs[0]
    copied = [torch.cuda.Event(), torch.cuda.Event()]
    step_done = [torch.cuda.Event(), torch.cuda.Event()]
    factors_in = torch.cuda.Event()
    e_start, e_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e_start.record(stream)
    copy_stream.wait_stream(stream)
    with torch.cuda.stream(copy_stream):
        xbufs[0].copy_(X_pin, non_blocking=True)
        copied[0].record(copy_stream)
    for e in range(args.steps):
        buf = e % 2
        with torch.cuda.stream(copy_stream):
            if e >= 1:  # step e - 1 has read its results back and is done with buffer 1 - buf
                copy_stream.wait_event(step_done[1 - buf])
            for a_dev, a_host in zip(run.F.A, A_pin):
                a_dev[:, :RANK].copy_(a_host, non_blocking=True)
            factors_in.record(copy_stream)
            if e + 1 < args.steps:
                xbufs[1 - buf].copy_(X_pin, non_blocking=True)
                copied[1 - buf].record(copy_stream)
        with torch.cuda.stream(stream):
            stream.wait_event(factors_in)
            stream.wait_event(copied[buf])
            graphs[buf].replay()
            state_out.copy_(run.state, non_blocking=True)
            for a_host, a_dev in zip(F_out, run.F.A):
                a_host.copy_(a_dev[:, :RANK], non_blocking=True)
            step_done[buf].record(stream)
    e_end.record(stream)
    barrier()
    e2e_elapsed = max_over_ranks(e_start.elapsed_time(e_end) * 1e-3, world, dev)
    e2e_value = entries / e2e_elapsed

    # the dominant kernel (the fused sampled gradient), timed alone
    mean_s, n_timed, adam_s = time_grad_kernel(torch, gcp, run, stream)
    peak, peak_kind = peaks()
    achieved = BYTES_PER_DRAW * S_DRAWS / mean_s / 1e9
    launch = gcp.gcp_get_launch(run.h, run.F, S_DRAWS)

    if rank != 0:
        torch.distributed.destroy_process_group()
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
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "overlap": "X double-buffered: step e+1's H2D copy runs during step e"},
            "gpu_launches": args.steps * (2 * TAU + 2),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": recorded_traffic(launch), "kernel": "grad_kernel (fused sample/gather/model/derivative/MTTKRP scatter)",
                         "bytes_per_draw": BYTES_PER_DRAW, "draws_per_launch": S_DRAWS,
                         "launch_us_mean": mean_s * 1e6, "launches_timed": n_timed,
                         "adam_us_mean": adam_s * 1e6,
                         "share_of_iteration_kernels": mean_s / (mean_s + adam_s),
                         "peak_source": f"{peak_kind} hbm_gbs"},
            "final_state": {k: st[k] for k in ("F", "t", "iter", "alpha", "bad")}}
    clocks = clk.summary()
    line["clocks"] = clocks
    # the single-GPU characterisations and the CPU baseline belong to the
    # one-GPU line; with N replicas they would only hold the N GPUs longer
    single = world == 1
    if single and not args.no_sweep:
        line["sweep"] = sweep_draws(torch, gcp, run, stream, peak)
    if single and not args.no_large:
        line["large_sparse"] = large_sparse(torch, gcp, synth, stream, peak)
    if single and not args.no_forms:
        line["forms"] = {"bf16": forms_bf16(torch, gcp, synth, stream),
                         "batched": forms_batched(torch, gcp, synth, stream)}
    if single and not args.no_cpu_baseline:
        rate, sample = oracle_epoch_rate(oracle_tensor(X32), A0, budget_s=args.cpu_budget)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample}
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# the other forms, each beside the plain FP32 single-problem path
# ---------------------------------------------------------------------------

def _time_calls(torch, fn, stream, reps):
    """Median device time of fn() from CUDA events around each call, queued behind a sleep."""
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    with torch.cuda.stream(stream):
        torch.cuda._sleep(100_000_000)
        for a, b in evs:
            a.record(stream)
            fn()
            b.record(stream)
    stream.synchronize()
    return statistics.median(a.elapsed_time(b) for a, b in evs) * 1e-3


def sweep_draws(torch, gcp, run, stream, peak, sizes=(100_000, 1_000_000, 10_000_000)):
    """Whole GCP-Adam iterations (gradient + Adam) on the benchmark tensor at
    larger draw counts per iteration, each size captured as a CUDA graph of
    back-to-back iterations on throwaway copies of the factors: the
    bandwidth-bound reading of the same kernels."""
    out = []
    with torch.cuda.stream(stream):
        F = gcp.Factors([a[:, :RANK] for a in run.F.A])
        G, B, C = F.like(), F.like(), F.like()
        st = gcp.new_state()
        gcp.gcp_state_init(st, 1e-4, stream=stream)
    from paper_1906_01687_gb300.autotune import side_stream
    cap = side_stream(stream)
    for s in sizes:
        spec = gcp.Sampling(gcp.SAMPLER_UNIFORM, 0, s, 99, 0)
        iters = max(3, min(50, 5_000_000 // s))

        def one(strm):
            gcp.gcp_iteration(run.h, F, gcp.LOSS_GAUSSIAN, spec, G, B, C, st, stream_dev=st[3:4], stream=strm)
        with torch.cuda.stream(stream):
            one(stream)
        stream.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=cap):
            for _ in range(iters):
                one(cap)
        with torch.cuda.stream(stream):
            g.replay()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(3):
                g.replay()
            b.record(stream)
        stream.synchronize()
        us = a.elapsed_time(b) * 1e3 / (3 * iters)
        gbs = BYTES_PER_DRAW * s / us / 1e3
        out.append({"draws_per_iteration": s, "us_per_iteration": us, "entries_per_s": s / us * 1e6,
                    "algorithmic_gbs": gbs, "frac_of_measured_hbm": gbs / peak})
        del g
    return {"what": "whole iterations (gradient + Adam), CUDA graph, dense 100^4 rank 10, Gaussian, uniform",
            "points": out}


def large_sparse(torch, gcp, synth, stream, peak, iters=10):
    """The largest sparse workload: the 1e5 x 1e5 x 1e4 binary tensor with 1e8
    nonzeros, rank 32, Bernoulli-logit, semi-stratified 1e6 + 1e6 draws per
    iteration, whole GCP-Adam iterations (gradient + Adam over all 2.1e5 x 32
    factor entries) captured in a CUDA graph; FP32 and BF16 factor storage.
    Algorithmic bytes per iteration: nonzero draws 16 B (packed record) +
    d r b_f B rows + d r 4 B updates (784 B in FP32, 592 B with BF16 rows),
    "zero" draws the same without the record (no value read), plus the Adam
    pass (32 B per factor entry, + 2 B for the BF16 copy)."""
    t0 = time.time()
    dims, rank, p, q = (100_000, 100_000, 10_000), 32, 1_000_000, 1_000_000
    idx, _, _ = synth.binary_tensor(device=stream.device)
    h = gcp.Handle(gcp.DataTensor.coo(dims, idx, None, device=stream.device), stream=stream)
    gen_s = time.time() - t0
    A = [(a / math.sqrt(rank) ** (1 / 3)).astype(np.float32) for a in synth.initial_guess(dims, rank, 5)]
    entries = sum(dims) * rank
    out = {"workload": "coo-1e5x1e5x1e4-nnz1e8-r32-bernoullilogit-semistratified-1e6+1e6",
           "what": "whole iterations (gradient + Adam), CUDA graph", "generation_s": gen_s}
    from paper_1906_01687_gb300.autotune import side_stream
    cap = side_stream(stream)
    for name, bf16 in (("fp32", False), ("bf16", True)):
        b_f = 2 if bf16 else 4
        grad_bytes = p * (16 + len(dims) * rank * (b_f + 4)) + q * (len(dims) * rank * (b_f + 4))
        adam_bytes = entries * (32 + (2 if bf16 else 0))
        with torch.cuda.stream(stream):
            F = gcp.Factors(A, bf16=bf16)
            G, B, C = F.like(), F.like(), F.like()
            st = gcp.new_state()
            gcp.gcp_state_init(st, 1e-4, stream=stream)
        spec = gcp.Sampling(gcp.SAMPLER_SEMI_STRATIFIED, p, q, 1687, 0)
        gcp.gcp_set_tuning(h, early_draws=1)

        def one(strm):
            gcp.gcp_iteration(h, F, gcp.LOSS_BERNOULLI_LOGIT, spec, G, B, C, st, stream_dev=st[3:4], stream=strm)
        with torch.cuda.stream(stream):
            one(stream)
        stream.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=cap):
            for _ in range(iters):
                one(cap)
        with torch.cuda.stream(stream):
            g.replay()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(3):
                g.replay()
            b.record(stream)
        stream.synchronize()
        us = a.elapsed_time(b) * 1e3 / (3 * iters)
        gbs = (grad_bytes + adam_bytes) / us / 1e3
        out[name] = {"us_per_iteration": us, "entries_per_s": (p + q) / us * 1e6,
                     "algorithmic_bytes_per_iteration": grad_bytes + adam_bytes, "algorithmic_gbs": gbs,
                     "frac_of_measured_hbm": gbs / peak}
        del g
    return out


def forms_bf16(torch, gcp, synth, stream):
    """FP32 vs BF16 factor storage on the count tensor (6186x24x77x32, 5.33M
    nonzeros, rank 10, Poisson-log, stratified 1e5 + 1e5 draws): gradient
    throughput, and the gradient's and the loss estimate's errors against the
    FP64 oracle (at the FP32 factors) on the same draws."""
    import oracle
    from paper_1906_01687_gb300.autotune import autotune, candidates
    dims = (6186, 24, 77, 32)
    idx, vals, _ = synth.count_tensor()
    h = gcp.Handle(gcp.DataTensor.coo(dims, idx, vals))
    A = [(a * 0.3).astype(np.float32) for a in synth.initial_guess(dims, 10, 4, positive=True)]
    spec = gcp.Sampling(gcp.SAMPLER_STRATIFIED, 100_000, 100_000, 1687, 0)
    XO = oracle.Tensor(dims, coo=np.stack([i.astype(np.int64) for i in idx], axis=1), vals=vals.astype(np.float64))
    SO = oracle.sample(XO, oracle.STRATIFIED, 100_000, 100_000, 1687, 0)
    ref = oracle.grad(dims, [a.astype(np.float64) for a in A], oracle.POISSON_LOG, SO)
    # the fixed loss-estimate list (stratified 1e5 + 1e5, the estimate stream)
    est_spec = gcp.Sampling(gcp.SAMPLER_STRATIFIED, 100_000, 100_000, 7, gcp.STREAM_EST)
    SOe = oracle.sample(XO, oracle.STRATIFIED, 100_000, 100_000, 7, gcp.STREAM_EST)
    F_ref = oracle.loss_estimate(dims, [a.astype(np.float64) for a in A], oracle.POISSON_LOG, SOe)
    out = {"workload": "coo-6186x24x77x32-nnz5330673-r10-poissonlog-stratified-1e5+1e5",
           "metric": "entries/s of gcp_grad (zero pass + gradient)"}
    for name, bf16 in (("fp32", False), ("bf16", True)):
        F = gcp.Factors(A, bf16=bf16)
        tuned = autotune(h, F, gcp.LOSS_POISSON_LOG, spec, launches=10, stream=stream,
                         configs=[dict(c, early_draws=1) for c in candidates(10)])
        G = F.like()
        t = _time_calls(torch, lambda: gcp.gcp_grad(h, F, gcp.LOSS_POISSON_LOG, G, S=spec, stream=stream), stream, 50)
        for x in G:
            x.zero_()
        gcp.gcp_grad(h, F, gcp.LOSS_POISSON_LOG, G, S=spec, stream=stream)
        stream.synchronize()
        got = [x[:, :10].double().cpu().numpy() for x in G]
        err = math.sqrt(sum(np.linalg.norm(a - b) ** 2 for a, b in zip(got, ref)) /
                        sum(np.linalg.norm(b) ** 2 for b in ref))
        out[name] = {"value": 200_000 / t, "us_per_call": t * 1e6, "grad_rel_err_vs_fp64_oracle": err,
                     "launch": gcp.gcp_get_launch(h, F, 200_000), "tuning": tuned["best"]}
        try:
            est = gcp.gcp_sample(h, est_spec, stream=stream)
            F_dev = torch.zeros(1, dtype=torch.float64, device=G[0].device)
            gcp.gcp_loss_est(h, F, gcp.LOSS_POISSON_LOG, est, F_dev, stream=stream)
            stream.synchronize()
            out[name]["loss_rel_err_vs_fp64_oracle"] = abs(F_dev.item() - F_ref) / abs(F_ref)
        except Exception as e:  # a reporting extra: record the failure, keep the line
            out[name]["loss_rel_err_vs_fp64_oracle"] = None
            out[name]["loss_error"] = repr(e)
    out["bf16_over_fp32"] = out["bf16"]["value"] / out["fp32"]["value"]
    return out


def forms_batched(torch, gcp, synth, stream, tau=20, epochs=3):
    """64 independent dense problems (d in {3,4}, dims U[50,2000] with at most
    2e7 entries, ranks {4,8,16,32,64}, mixed losses, 1e4-1e5 draws/iteration):
    one batched launch per step under one CUDA graph, against the same 64
    problems run one after another (each its own graph-replayed epoch)."""
    from paper_1906_01687_gb300.adam import GcpAdam
    from paper_1906_01687_gb300.batch import GcpAdamBatch
    shapes = synth.batched_problems()
    specs = []
    gen = torch.Generator(device="cuda")
    for i, sh in enumerate(shapes):
        gen.manual_seed(1911 + i)
        d, r = len(sh["dims"]), sh["rank"]
        fac = [torch.randn((n, r), generator=gen, device="cuda") * (1.0 / r) ** (1.0 / (2 * d)) for n in sh["dims"]]
        letters = "ijkl"[:d]
        M = torch.einsum(",".join(f"{c}z" for c in letters) + "->" + letters, *fac)
        if sh["loss"] == "gaussian":
            X = M + 0.1 * torch.randn(M.shape, generator=gen, device="cuda")
        elif sh["loss"] == "bernoulli_logit":
            X = (torch.rand(M.shape, generator=gen, device="cuda") < torch.sigmoid(M)).float()
        else:
            X = torch.poisson(torch.exp(M.clamp(max=10.0)), generator=gen)
        X = gcp.DataTensor(tuple(sh["dims"]), vals=X.reshape(-1).contiguous())
        A0 = synth.initial_guess(sh["dims"], r, 500 + i, target_norm=float(torch.linalg.vector_norm(X.vals)))
        specs.append(dict(X=X, A0=A0, loss=gcp.LOSSES[sh["loss"]], s=sh["s"], est=10_000, seed=1687 + i,
                          est_seed=7, problem=i))
    draws = sum(sp["s"] for sp in specs)
    torch.cuda.synchronize()
    batch = GcpAdamBatch(specs, tau=tau, alpha=1e-3, kappa=1_000_000, stream=stream, autotune=True)
    batch.capture()
    batch.run_epoch()
    stream.synchronize()
    t_batch = _time_calls(torch, batch.run_epoch, stream, epochs)
    singles = []
    for i, sp in enumerate(specs):
        run = GcpAdam(sp["X"], sp["A0"], sp["loss"], gcp.SAMPLER_UNIFORM, 0, sp["s"], 0, sp["est"], seed=sp["seed"],
                      est_seed=7, alpha=1e-3, tau=tau, kappa=1_000_000, problem=i, stream=stream)
        run.capture()
        singles.append(run)
    for run in singles:
        run.run_epoch()
    stream.synchronize()
    t_seq = _time_calls(torch, lambda: [run.run_epoch() for run in singles], stream, epochs)
    # accuracy: after the same number of epochs, each batched problem vs its single run
    errs = []
    batch2 = GcpAdamBatch(specs, tau=tau, alpha=1e-3, kappa=1_000_000, stream=stream)
    for _ in range(2):
        batch2.run_epoch()
    for i in range(0, len(specs), 8):
        single = GcpAdam(specs[i]["X"], specs[i]["A0"], specs[i]["loss"], gcp.SAMPLER_UNIFORM, 0, specs[i]["s"], 0,
                         specs[i]["est"], seed=specs[i]["seed"], est_seed=7, alpha=1e-3, tau=tau, kappa=1_000_000,
                         problem=i, stream=stream)
        single.run_epoch()
        single.run_epoch()
        a, b = batch2.factors(i), single.factors()
        errs.append(math.sqrt(sum(np.linalg.norm(x - y) ** 2 for x, y in zip(a, b)) /
                              sum(np.linalg.norm(y) ** 2 for y in b)))
    entries = tau * draws
    return {"workload": f"64 dense problems, d 3-4, dims 50-2000 (<= 2e7 entries), ranks 4-64, mixed losses, "
                        f"{draws} draws/iteration in total, tau {tau}",
            "metric": "sampled-gradient entries/s over one epoch (all problems)",
            "batched": {"value": entries / t_batch, "ms_per_epoch": t_batch * 1e3, "launches_per_iteration": 2,
                        "tuning": batch.tuned},
            "sequential": {"value": entries / t_seq, "ms_per_epoch": t_seq * 1e3,
                           "launches_per_iteration": 2 * len(specs)},
            "batched_over_sequential": t_seq / t_batch,
            "factor_rel_diff_vs_single_runs_after_2_epochs_max": max(errs)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the BF16 and batched form comparisons")
    ap.add_argument("--no-sweep", action="store_true", help="skip the draws-per-iteration sweep")
    ap.add_argument("--no-large", action="store_true", help="skip the 1e8-nonzero sparse workload")
    ap.add_argument("--tuning", default=None, help="JSON gcp_tuning fields to use instead of autotuning")
    ap.add_argument("--only-forms", action="store_true",
                    help="run only the BF16 and batched form comparisons (one JSON object; for profiling them)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        return reference_arm(args)
    if args.only_forms:
        return forms_only()
    return ours_arm(args)


def forms_only():
    import torch
    from paper_1906_01687_gb300 import gcp, synth
    stream = torch.cuda.Stream()
    print(json.dumps({"forms": {"bf16": forms_bf16(torch, gcp, synth, stream),
                                "batched": forms_batched(torch, gcp, synth, stream)}}), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
