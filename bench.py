"""Benchmark of the GCP-Adam sampled-gradient path on one GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload: a sparse binary 3-way tensor of 1e5 x 1e5 x 1e4 with 1e8 nonzeros
in COO (int32 indices), drawn from a planted rank-32 logistic model;
Bernoulli-logit loss; semi-stratified sampling (Alg. 3) with 1e6 nonzero and
1e6 "zero" draws per iteration; rank 32; FP32 factors; the loss estimate on a
fixed semi-stratified set of 1e5 + 1e5 entries.  One step is one GCP-Adam
epoch (Alg. 4): tau = 1000 iterations of (fused sample + gradient, Adam
step; Section 5.1's epoch length), the loss estimate and the accept-or-revert
decision, captured once as a CUDA graph and replayed.  Metric: sampled-gradient entries processed per
second (tau (p + q) per step).

The same line carries the other workloads as forms, each beside the plain
FP32 path with its roofline fraction: BF16-stored factors on this tensor;
the dense 100^4 Gaussian tensor (uniform sampling, rank 10); the count tensor
shaped like the Chicago crime data (stratified, Poisson-log, FP32 and BF16);
64 batched problems; a draws-per-iteration sweep.

Rank r of an N-rank run (torchrun) fits its own replica (seed + r): the
benchmark's ranks are independent decompositions ("replicas only"; the
sample-parallel split of one problem is in paper_1906_01687_gb300/parallel.py).
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
from concurrent.futures import ThreadPoolExecutor

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "sampled-gradient entries/s"
UNIT = "entries/s"
WORKLOAD = "coo-1e5x1e5x1e4-nnz1e8-r32-bernoullilogit-semistratified-1e6+1e6"
DIMS, NNZ, RANK = (100_000, 100_000, 10_000), 100_000_000, 32
P_DRAWS, Q_DRAWS, EST_P, EST_Q, TAU = 1_000_000, 1_000_000, 100_000, 100_000, 1000  # tau: Section 5.1's default
ALPHA = 0.01  # Adam's learning rate, Section 5.1's default
RECORD_BYTES = 16  # packed record of a nonzero of a 3-way tensor: three indices and the value's bits

KERNEL_SOURCES = ("gcp_grad_impl.cuh", "gcp_draw.cuh", "gcp_device.cuh", "gcp_kernels.cuh")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "grad_kernel_coo1e8_r32_semi2e6.json")


def row_bytes(d, rank, b_f):
    """Per draw: d factor rows of rank entries gathered (b_f bytes each) and
    d rows of rank FP32 updates added into G."""
    return d * rank * (b_f + 4)


def grad_bytes(p, q, d, rank, b_f, nz_extra=RECORD_BYTES, zero_extra=0):
    """Algorithmic bytes of one gradient launch: p nonzero draws reading
    nz_extra bytes each (their packed record), q zero draws reading
    zero_extra bytes (0 when their indices are generated), and the rows."""
    return p * (nz_extra + row_bytes(d, rank, b_f)) + q * (zero_extra + row_bytes(d, rank, b_f))


def stratified_call_bytes(dims, nnz, p, q, rank, b_f, rho=1.1):
    """Algorithmic bytes of a stratified gcp_grad call (Alg. 2): nonzero draws
    read a 32-byte record (4 indices and the value, padded); each accepted
    zero costs rho * omega / zeta candidates' 8-byte hash probes (zeta =
    omega - nnz zeros); no zero list is read or written (the gradient kernel
    walks the accepted candidates it draws); every draw gathers and updates
    its d rows."""
    omega = float(np.prod(dims))
    cand_per_zero = rho * omega / (omega - nnz)
    return grad_bytes(p, q, len(dims), rank, b_f, nz_extra=32, zero_extra=8 * cand_per_zero)


def adam_bytes(dims, rank, bf16=False):
    """Algorithmic bytes of one Adam step: A, B, C, G read and written (32 B
    per factor entry), plus the BF16 copy written."""
    return sum(dims) * rank * (32 + (2 if bf16 else 0))


def code_hash(texts):
    """Hash of C++/CUDA source texts with comments and blank space removed:
    a change of code changes it, a change of comments does not."""
    import hashlib
    import re
    h = hashlib.sha256()
    for text in texts:
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def kernel_source_hash():
    """code_hash of the gradient kernel's sources: the key of the recorded traffic."""
    texts = []
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1906_01687_gb300", "csrc", name)) as f:
            texts.append(f.read())
    return code_hash(texts)


def recorded_traffic(launch, path=None):
    """DRAM bytes per launch of grad_kernel from the committed ncu summary, if
    the kernel sources and the kernel instance (lanes x chunks, draw layout,
    early draws) are those the counters were taken with; otherwise None.
    The block size is not compared: it changes neither the kernel's code nor
    its DRAM traffic."""
    try:
        with open(path or TRAFFIC_FILE) as f:
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


def host_cores():
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


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
# inputs
# ---------------------------------------------------------------------------

def large_input(init_seed=3):
    """The benchmark tensor's nonzero positions (host int32 SoA; generated
    with torch's seeded generator on the GPU when there is one), the initial
    factors -- entries uniform in (0, 1), scaled so that the model's norm
    equals the data's, sqrt(nnz) (the paper's initial guesses for its binary
    problems, Sections 5.4-5.5) -- and the planted factors."""
    import torch
    from paper_1906_01687_gb300 import synth
    device = "cuda" if torch.cuda.is_available() else "cpu"
    idx, _, planted = synth.binary_tensor(DIMS, NNZ, RANK, device=device)
    A0 = synth.initial_guess(DIMS, RANK, seed=init_seed, target_norm=math.sqrt(NNZ), positive=True)
    return idx, A0, planted


def near_fitted(planted):
    """Factors near a fitted model of the benchmark tensor: the planted
    model with its first column a constant c, c^3 = log(1e-6) (the density),
    so that sigma(m) of a zero is about 1e-6 and a zero draw's y, (omega/q)
    sigma(m) ~ 100, nearly cancels a nonzero draw's, -(eta/p) = -100."""
    c = -(-math.log(1e-6)) ** (1.0 / 3.0)
    A = [np.array(a, dtype=np.float32) for a in planted]
    for a in A:
        a[:, 0] = c
    return A


# ---------------------------------------------------------------------------
# the FP64 oracle on the host cores (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------

def oracle_large_tensor(idx):
    import oracle
    return oracle.Tensor(DIMS, coo=np.stack([np.asarray(i, np.int64) for i in idx], axis=1), vals=None)


def _slices(S, parts):
    import oracle
    cuts = [S.n * i // parts for i in range(parts + 1)]
    return [oracle.Samples(S.idx[a:b], S.x[a:b], S.w[a:b], S.cls[a:b]) for a, b in zip(cuts[:-1], cuts[1:])]


def oracle_grad_threads(dims, A, loss, S, cores):
    """The oracle's sampled gradient over S on `cores` host threads: the draws
    split into contiguous slices, one oracle call per slice on its own thread
    (the C oracle runs without the interpreter lock), the partial gradients
    summed in slice order."""
    import oracle
    if cores <= 1:
        return oracle.grad(dims, A, loss, S)
    with ThreadPoolExecutor(cores) as ex:
        parts = list(ex.map(lambda s: oracle.grad(dims, A, loss, s), _slices(S, cores)))
    out = [p.copy() for p in parts[0]]
    for part in parts[1:]:
        for k in range(len(dims)):
            out[k] += part[k]
    return out


def oracle_loss_threads(dims, A, loss, S, cores):
    """The oracle's loss estimate over S, split over `cores` host threads like the gradient."""
    import oracle
    if cores <= 1:
        return oracle.loss_estimate(dims, A, loss, S)
    with ThreadPoolExecutor(cores) as ex:
        return sum(ex.map(lambda s: oracle.loss_estimate(dims, A, loss, s), _slices(S, cores)))


def oracle_epoch_rate(XO, A0, cores, iters=1, seed=1687):
    """Entries/s of the FP64 oracle doing the benchmark's epoch on `cores`
    host threads: per iteration the draws (one thread: the oracle's sampler
    has no draw range), the gradient split over the threads and summed, and
    the Adam step; one loss estimate per epoch (split the same way).  Timed
    over `iters` iterations and one estimate, scaled to a tau-iteration epoch."""
    import oracle
    A = [np.asarray(a, np.float64) for a in A0]
    flat = oracle.concat_factors(A)
    B, C = np.zeros_like(flat), np.zeros_like(flat)
    est = oracle.sample(XO, oracle.SEMI_STRATIFIED, EST_P, EST_Q, 7, 2**64 - 1)
    t0 = time.perf_counter()
    oracle_loss_threads(DIMS, oracle.split_factors(flat, DIMS, RANK), oracle.BERNOULLI_LOGIT, est, cores)
    t_est = time.perf_counter() - t0
    t_it = 0.0
    for it in range(iters):
        t0 = time.perf_counter()
        S = oracle.sample(XO, oracle.SEMI_STRATIFIED, P_DRAWS, Q_DRAWS, seed, it)
        G = oracle_grad_threads(DIMS, oracle.split_factors(flat, DIMS, RANK), oracle.BERNOULLI_LOGIT, S, cores)
        oracle.adam_step(flat, B, C, oracle.concat_factors(G), 1e-3, t=it)
        t_it += time.perf_counter() - t0
    per_it = t_it / iters
    rate = TAU * (P_DRAWS + Q_DRAWS) / (TAU * per_it + t_est)
    sample = (f"{iters} oracle iteration(s) of {P_DRAWS}+{Q_DRAWS} semi-stratified draws (sample on one thread, "
              f"gradient on {cores} thread(s), Adam) and one {EST_P}+{EST_Q}-entry loss estimate, "
              f"scaled to a {TAU}-iteration epoch")
    return rate, sample


def cpu_baseline(XO, A0, budget_iters=(1, 2)):
    """The oracle on one host core and on all of them (threads over draw slices)."""
    cores = host_cores()
    rate1, sample1 = oracle_epoch_rate(XO, A0, 1, iters=budget_iters[0])
    rate_n, sample_n = oracle_epoch_rate(XO, A0, cores, iters=budget_iters[1])
    return {"value": rate_n, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample_n,
            "value_1core": rate1, "sample_1core": sample1, "cores_from": "os.sched_getaffinity(0)"}


def reference_arm(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    idx, A0, _ = large_input()
    XO = oracle_large_tensor(idx)
    cores = host_cores()
    rates = []
    for step in range(args.warmup + args.steps):
        rate, sample = oracle_epoch_rate(XO, A0, cores, iters=1, seed=1687 + step)
        if step >= args.warmup:
            rates.append(rate)
    value = statistics.median(rates)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": TAU * (P_DRAWS + Q_DRAWS) / value * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded planted rank-32 logistic model)",
            "config": {"workload": WORKLOAD, "dims": list(DIMS), "nnz": NNZ, "rank": RANK,
                       "samples_per_iter": [P_DRAWS, Q_DRAWS], "tau": TAU, "est_samples": [EST_P, EST_Q]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# the CUDA path
# ---------------------------------------------------------------------------

def time_grad_kernel(torch, gcp, h, iterate, stream, launches=50):
    """Average device duration of the fused-gradient kernel and of the Adam
    kernel: the library records CUDA events on the launching stream around
    each kernel launch of `launches` GCP-Adam iterations (iterate()), queued
    behind a sleep so that they run back to back."""
    gcp.gcp_profile(h, True, launches)
    with torch.cuda.stream(stream):
        torch.cuda._sleep(200_000_000)
        for _ in range(launches):
            iterate()
    stream.synchronize()
    ms, n = gcp.gcp_profile_read(h, 0)
    ms_adam, n_adam = gcp.gcp_profile_read(h, 1)
    gcp.gcp_profile(h, False)
    return ms * 1e-3 / n, n, ms_adam * 1e-3 / max(n_adam, 1)


def time_iterations(torch, gcp, h, F, loss, spec, stream, iters=10, replays=3):
    """Device time (s) per whole GCP-Adam iteration (gradient + Adam) of a
    captured sequence of iterations on throwaway optimizer state."""
    from paper_1906_01687_gb300.autotune import side_stream
    with torch.cuda.stream(stream):
        G, B, C = F.like(), F.like(), F.like()
        st = gcp.new_state(F.A[0].device)
        gcp.gcp_state_init(st, 1e-4, stream=stream)

    def one(strm):
        gcp.gcp_iteration(h, F, loss, spec, G, B, C, st, stream_dev=st[3:4], stream=strm)
    with torch.cuda.stream(stream):
        one(stream)
    stream.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side_stream(stream)):
        for _ in range(iters):
            one(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        g.replay()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(replays):
            g.replay()
        b.record(stream)
    stream.synchronize()
    del g
    return a.elapsed_time(b) * 1e-3 / (replays * iters)


def adam_only_time(torch, gcp, F, stream, iters=50, replays=3):
    """Device time (s) per Adam step (gcp_adam_step) of a captured sequence of
    steps on throwaway state: subtracted from a captured whole iteration it
    bounds the gradient kernel's time inside the iteration from above (the
    standalone step folds no replica slabs, so it is the cheaper Adam)."""
    from paper_1906_01687_gb300.autotune import side_stream
    with torch.cuda.stream(stream):
        Ft = gcp.Factors([a[:, :F.rank] for a in F.A])
        G, B, C = Ft.like(), Ft.like(), Ft.like()
        st = gcp.new_state(Ft.A[0].device)
        gcp.gcp_state_init(st, 1e-4, stream=stream)
        gcp.gcp_adam_step(Ft, G, B, C, st, stream=stream)
    stream.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side_stream(stream)):
        for _ in range(iters):
            gcp.gcp_adam_step(Ft, G, B, C, st, stream=torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        g.replay()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(replays):
            g.replay()
        b.record(stream)
    stream.synchronize()
    del g
    return a.elapsed_time(b) * 1e-3 / (replays * iters)


def grad_launch_time(torch, gcp, h, F, loss, spec, stream, launches=50):
    """Per-launch device time of the gradient kernel inside GCP-Adam
    iterations on throwaway state (events around each gradient launch)."""
    with torch.cuda.stream(stream):
        G, B, C = F.like(), F.like(), F.like()
        st = gcp.new_state(F.A[0].device)
        gcp.gcp_state_init(st, 1e-4, stream=stream)

    def it():
        gcp.gcp_iteration(h, F, loss, spec, G, B, C, st, stream_dev=st[3:4], stream=stream)
    with torch.cuda.stream(stream):
        it()
    return time_grad_kernel(torch, gcp, h, it, stream, launches)


def rel_err(got, ref):
    return math.sqrt(sum(float(np.linalg.norm(a - b)) ** 2 for a, b in zip(got, ref)) /
                     sum(float(np.linalg.norm(b)) ** 2 for b in ref))


def ours_arm(args):
    import torch
    from paper_1906_01687_gb300 import gcp
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

    init_seed, seed = replica_seeds(rank)
    t_gen = time.time()
    idx, A0, planted = large_input(init_seed)
    gen_s = time.time() - t_gen
    XT = gcp.DataTensor.coo(DIMS, idx, None, device=dev)
    with torch.cuda.stream(stream):
        run = GcpAdam(XT, A0, gcp.LOSS_BERNOULLI_LOGIT, gcp.SAMPLER_SEMI_STRATIFIED, P_DRAWS, Q_DRAWS, EST_P, EST_Q,
                      seed=seed, est_seed=7, alpha=ALPHA, tau=TAU, kappa=1_000_000, stream=stream,
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
    per_step = TAU * (P_DRAWS + Q_DRAWS)
    entries = args.steps * per_step * world
    value = whole_job_rate(args.steps * per_step, world, elapsed)

    # end to end through the public API with host buffers: every step copies
    # the COO index arrays (1.2 GB) and the initial factors from pinned
    # memory, re-packs the nonzero records (gcp_refresh, first node of the
    # step's graph), runs the epoch and reads F-hat and the factors back.
    # The tensor is double-buffered: step e + 1's copy (on a copy stream,
    # into the other device buffer, read by a second handle and graph) runs
    # while step e computes.  All host-to-device copies go through the copy
    # stream in step order (factors of step e, then the tensor of step e + 1).
    idx_pin = [torch.from_numpy(np.ascontiguousarray(i)).pin_memory() for i in idx]
    A_pin = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in A0]
    F_out = [torch.empty(a.shape, dtype=torch.float32).pin_memory() for a in A0]
    state_out = torch.empty(8, dtype=torch.float64).pin_memory()
    h2d = sum(i.numel() * 4 for i in idx_pin) + sum(a.numel() * 4 for a in A_pin)
    d2h = state_out.numel() * 8 + sum(a.numel() * 4 for a in F_out)
    XT2 = gcp.DataTensor.coo(DIMS, idx, None, device=dev)
    tuning = dict(run.tuned["best"]) if run.tuned else {"early_draws": 1}
    with torch.cuda.stream(stream):
        h1 = run.h
        run.capture(refresh=True)
        g1 = run.graph
        h2 = gcp.Handle(XT2, stream=stream)
        gcp.gcp_set_tuning(h2, **tuning)
        run.h = h2
        run.capture(refresh=True)
        g2 = run.graph
        run.h = h1
    handles, graphs, xbufs = [h1, h2], [g1, g2], [XT.idx, XT2.idx]
    # the host-to-device rate of this machine for the step's tensor copy (pinned memory, the copy stream alone)
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(copy_stream):
        c0.record(copy_stream)
        for dst, src in zip(xbufs[1], idx_pin):
            dst.copy_(src, non_blocking=True)
        c1.record(copy_stream)
    copy_stream.synchronize()
    h2d_gbs = sum(i.numel() * 4 for i in idx_pin) / (c0.elapsed_time(c1) * 1e-3) / 1e9
    copied = [torch.cuda.Event(), torch.cuda.Event()]
    step_done = [torch.cuda.Event(), torch.cuda.Event()]
    factors_in = torch.cuda.Event()
    e_start, e_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e_start.record(stream)
    copy_stream.wait_stream(stream)
    with torch.cuda.stream(copy_stream):
        for dst, src in zip(xbufs[0], idx_pin):
            dst.copy_(src, non_blocking=True)
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
                for dst, src in zip(xbufs[1 - buf], idx_pin):
                    dst.copy_(src, non_blocking=True)
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
    e2e_state = gcp.read_state(state_out)
    del graphs, g1, g2

    # the dominant kernel (the fused sampled gradient), timed on its stream
    peak, peak_kind = peaks()
    mean_s, n_timed, adam_s = time_grad_kernel(torch, gcp, run.h, run.iteration, stream)
    bytes_launch = grad_bytes(P_DRAWS, Q_DRAWS, len(DIMS), RANK, 4)
    achieved = bytes_launch / mean_s / 1e9
    launch = gcp.gcp_get_launch(run.h, run.F, P_DRAWS + Q_DRAWS)
    iter_s = time_iterations(torch, gcp, run.h, run.F, run.loss, run.spec, stream)

    if rank != 0:
        torch.distributed.destroy_process_group()
        return 0
    ms_per_step = elapsed / args.steps * 1e3
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded planted rank-32 logistic model; COO int32)",
            "config": {"workload": WORKLOAD, "dims": list(DIMS), "nnz": NNZ, "rank": RANK,
                       "loss": "bernoulli_logit", "sampler": "semi_stratified",
                       "samples_per_iter": [P_DRAWS, Q_DRAWS], "tau": TAU, "est_samples": [EST_P, EST_Q],
                       "factors": "fp32",
                       "step": "one GCP-Adam epoch (tau iterations + loss estimate + accept/revert), CUDA graph",
                       "l2": "inputs larger than L2 (1.6 GB of packed nonzero records gathered at random; "
                             "factors and gradients, 27 MB each, L2-resident)",
                       "parallelism": f"replicas{world}", "grad_launch": launch, "autotuned": run.tuned,
                       "generation_s": gen_s},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "overlap": "tensor double-buffered: step e+1's H2D copy runs during step e; each step "
                               "re-packs its records (gcp_refresh) inside its graph",
                    "h2d_gbs_alone": h2d_gbs, "final_F": e2e_state["F"]},
            "gpu_launches": args.steps * (2 * TAU + 2),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": recorded_traffic(launch),
                         "kernel": "grad_kernel (fused sample/gather/model/derivative/MTTKRP scatter)",
                         "bytes_per_launch": bytes_launch,
                         "bytes_per_draw": {"nonzero": RECORD_BYTES + row_bytes(3, RANK, 4),
                                            "zero": row_bytes(3, RANK, 4)},
                         "draws_per_launch": P_DRAWS + Q_DRAWS,
                         "launch_us_mean": mean_s * 1e6, "launches_timed": n_timed,
                         "adam_us_mean": adam_s * 1e6,
                         "iteration_us_in_graph": iter_s * 1e6,
                         "in_step_check": {"grad_ms_per_step": TAU * mean_s * 1e3, "ms_per_step": ms_per_step,
                                           "fits": TAU * mean_s * 1e3 <= ms_per_step},
                         "peak_source": f"{peak_kind} hbm_gbs"},
            "final_state": {k: st[k] for k in ("F", "t", "iter", "alpha", "bad")}}
    clocks = clk.summary()
    line["clocks"] = clocks
    # the single-GPU characterisations and the CPU baseline belong to the
    # one-GPU line; with N replicas they would only hold the N GPUs longer
    single = world == 1
    XO = None
    if single and not (args.no_cpu_baseline and args.no_forms):
        XO = oracle_large_tensor(idx)
    if single and not args.no_forms:
        forms = {}
        for name, fn in (("bf16", lambda: form_large_bf16(torch, gcp, run, XO, A0, planted, stream, peak)),
                         ("dense100", lambda: form_dense100(torch, gcp, stream, peak, args)),
                         ("count", lambda: form_count(torch, gcp, stream, peak)),
                         ("batched", lambda: form_batched(torch, gcp, stream, peak))):
            try:
                forms[name] = fn()
            except Exception as e:  # a reporting extra: record the failure, keep the line
                forms[name] = {"error": repr(e)}
            torch.cuda.empty_cache()
        line["forms"] = forms
    if single and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(XO, A0)
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


def form_large_bf16(torch, gcp, run, XO, A0, planted, stream, peak):
    """FP32 vs BF16 factor storage on the benchmark tensor: per-launch
    gradient kernel time and roofline fraction of each, whole-iteration time,
    and the gradient's and the loss estimate's errors against the FP64
    oracle on the same draws (at the FP32 factors; for BF16 also at the
    BF16-rounded factors, which separates storage from arithmetic error)."""
    import oracle
    out = {"workload": WORKLOAD, "metric": "entries/s of the gradient kernel; whole GCP-Adam iterations"}
    spec = gcp.Sampling(gcp.SAMPLER_SEMI_STRATIFIED, P_DRAWS, Q_DRAWS, 4242, 0)
    SO = oracle.sample(XO, oracle.SEMI_STRATIFIED, P_DRAWS, Q_DRAWS, 4242, 0)
    cores = host_cores()
    A64 = [np.asarray(a, np.float32).astype(np.float64) for a in A0]
    G_ref = oracle_grad_threads(DIMS, A64, oracle.BERNOULLI_LOGIT, SO, cores)
    estO = oracle.sample(XO, oracle.SEMI_STRATIFIED, EST_P, EST_Q, 7, gcp.STREAM_EST)
    F_ref = oracle_loss_threads(DIMS, A64, oracle.BERNOULLI_LOGIT, estO, cores)
    from paper_1906_01687_gb300.autotune import autotune, candidates
    fp32_tuning = (run.tuned or {}).get("best")
    for name, bf16 in (("fp32", False), ("bf16", True)):
        b_f = 2 if bf16 else 4
        with torch.cuda.stream(stream):  # the timing steps its own copy of the factors
            F_t = gcp.Factors(A0, bf16=bf16)
        tuned = None
        if bf16 and fp32_tuning is not None:
            # BF16 rows get a launch shape of their own, timed as GCP-Adam times
            # them: whole iterations captured in a CUDA graph
            with torch.cuda.stream(stream):
                Gt, Bt, Ct = F_t.like(), F_t.like(), F_t.like()
                st_t = gcp.new_state(F_t.A[0].device)
                gcp.gcp_state_init(st_t, 1e-4, stream=stream)

            def call(sp, strm):
                gcp.gcp_iteration(run.h, F_t, run.loss, sp, Gt, Bt, Ct, st_t, stream_dev=st_t[3:4], stream=strm)
            tuned = autotune(run.h, F_t, run.loss, spec, launches=5, stream=stream, call=call, graph=True,
                             configs=[dict(c, early_draws=1) for c in candidates(RANK)])
            del Gt, Bt, Ct, st_t
        mean_s, n, adam_s = grad_launch_time(torch, gcp, run.h, F_t, run.loss, spec, stream)
        iter_s = time_iterations(torch, gcp, run.h, F_t, run.loss, spec, stream)
        del F_t
        gb = grad_bytes(P_DRAWS, Q_DRAWS, len(DIMS), RANK, b_f)
        ab = adam_bytes(DIMS, RANK, bf16)
        with torch.cuda.stream(stream):  # the error check: the initial factors A0
            F = gcp.Factors(A0, bf16=bf16)
            G = F.like()
            gcp.gcp_grad(run.h, F, run.loss, G, S=spec, stream=stream)
            F_dev = torch.zeros(1, dtype=torch.float64, device=G[0].device)
            gcp.gcp_loss_est(run.h, F, run.loss, run.est, F_dev, stream=stream)
        stream.synchronize()
        got = [x[:, :RANK].double().cpu().numpy() for x in G]
        rec = {"grad_kernel_us": mean_s * 1e6, "entries_per_s": (P_DRAWS + Q_DRAWS) / mean_s,
               "grad_bytes_per_launch": gb, "grad_frac_of_measured_hbm": gb / mean_s / 1e9 / peak,
               "iteration_us": iter_s * 1e6, "iteration_frac_of_measured_hbm": (gb + ab) / iter_s / 1e9 / peak,
               "grad_rel_err_vs_fp64_oracle": rel_err(got, G_ref),
               "loss_rel_err_vs_fp64_oracle": abs(F_dev.item() - F_ref) / abs(F_ref),
               "launch": gcp.gcp_get_launch(run.h, F, P_DRAWS + Q_DRAWS),
               "tuning": tuned["best"] if tuned else fp32_tuning}
        if tuned:
            gcp.gcp_set_tuning(run.h, **fp32_tuning)
        if bf16:
            Ab = [a.double().cpu().numpy()[:, :RANK] for a in F.A_bf16]
            G_rb = oracle_grad_threads(DIMS, Ab, oracle.BERNOULLI_LOGIT, SO, cores)
            rec["grad_rel_err_vs_fp64_oracle_at_bf16_factors"] = rel_err(got, G_rb)
        out[name] = rec
    # near a fitted model: the terms of opposite sign that nearly cancel in FP32
    An = near_fitted(planted)
    Gn_ref = oracle_grad_threads(DIMS, [a.astype(np.float64) for a in An], oracle.BERNOULLI_LOGIT, SO, cores)
    near = {}
    for name, bf16 in (("fp32", False), ("bf16", True)):
        with torch.cuda.stream(stream):
            F = gcp.Factors(An, bf16=bf16)
            G = F.like()
            gcp.gcp_grad(run.h, F, run.loss, G, S=spec, stream=stream)
        stream.synchronize()
        got = [x[:, :RANK].double().cpu().numpy() for x in G]
        near[name] = {"grad_rel_err_vs_fp64_oracle": rel_err(got, Gn_ref)}
        if bf16:
            Ab = [a.double().cpu().numpy()[:, :RANK] for a in F.A_bf16]
            near[name]["grad_rel_err_vs_fp64_oracle_at_bf16_factors"] = rel_err(
                got, oracle_grad_threads(DIMS, Ab, oracle.BERNOULLI_LOGIT, SO, cores))
    out["near_fitted"] = dict(near, what="planted factors with a constant column, c^3 = log(1e-6): "
                                         "zero and nonzero draws' terms of about +-100 nearly cancel")
    out["bf16_over_fp32_grad_kernel"] = out["fp32"]["grad_kernel_us"] / out["bf16"]["grad_kernel_us"]
    out["bound"] = ("L2: the gathered rows and the row updates of both forms are L2 hits (factors 27 MB); "
                    "BF16 halves the gathered bytes, not the L2 vector reductions of the updates")
    return out


def form_dense100(torch, gcp, stream, peak, args, tau=100, epochs=5):
    """The dense 100^4 FP32 tensor (planted rank 10 + N(0, 0.01) noise),
    Gaussian loss, uniform 1e5 draws per iteration: graph-replayed epochs,
    the gradient kernel per launch, and a draws-per-iteration sweep."""
    from paper_1906_01687_gb300 import synth
    from paper_1906_01687_gb300.adam import GcpAdam
    dims, rank, s = (100, 100, 100, 100), 10, 100_000
    X32, _ = synth.dense_100_4()
    A0 = synth.initial_guess(dims, rank, seed=3, target_norm=float(np.linalg.norm(X32)))
    XT = gcp.DataTensor.dense(X32, device=stream.device)
    with torch.cuda.stream(stream):
        run = GcpAdam(XT, A0, gcp.LOSS_GAUSSIAN, gcp.SAMPLER_UNIFORM, 0, s, 0, 100_000, seed=1687, est_seed=7,
                      alpha=1e-3, tau=tau, kappa=1_000_000, stream=stream, autotune=not args.no_autotune)
        run.capture()
    run.run_epoch()
    stream.synchronize()
    t_epoch = _time_calls(torch, run.run_epoch, stream, epochs)
    mean_s, n, adam_s = time_grad_kernel(torch, gcp, run.h, run.iteration, stream)
    launch = gcp.gcp_get_launch(run.h, run.F, s)
    iter_s = time_iterations(torch, gcp, run.h, run.F, run.loss, run.spec, stream, iters=50)
    # the same iteration with the Adam step in a launch of its own and as the
    # gradient kernel's tail work, for comparison
    best = dict((run.tuned or {}).get("best") or {"early_draws": 1})
    iters_by_tail = {}
    for tw in (0, 1):
        gcp.gcp_set_tuning(run.h, **dict(best, tail_work=tw))
        iters_by_tail[tw] = time_iterations(torch, gcp, run.h, run.F, run.loss, run.spec, stream, iters=50)
    gcp.gcp_set_tuning(run.h, **best)
    iter_sep_s = iters_by_tail[0]
    adam_s = adam_only_time(torch, gcp, run.F, stream)
    grad_in_graph = iter_sep_s - adam_s
    gb = s * (4 + row_bytes(4, rank, 4))
    ab = adam_bytes(dims, rank)
    out = {"workload": "dense-100x100x100x100-r10-gaussian-uniform-s1e5", "tau": tau,
           "entries_per_s": tau * s / t_epoch, "ms_per_epoch": t_epoch * 1e3,
           "grad_bytes_per_launch": gb, "adam_bytes_per_step": ab, "grad_kernel_us": mean_s * 1e6,
           "grad_frac_of_measured_hbm": gb / mean_s / 1e9 / peak,
           "kernels_per_iteration": 1 if launch["adam_tail_blocks"] else 2,
           "iteration_us_in_graph": iter_s * 1e6,
           "iteration_frac_of_measured_hbm": (gb + ab) / iter_s / 1e9 / peak,
           "iteration_us_in_graph_separate_adam_launch": iter_sep_s * 1e6,
           "iteration_us_in_graph_adam_in_gradient_kernel": iters_by_tail[1] * 1e6,
           "adam_only_us_in_graph": adam_s * 1e6,
           "grad_us_in_graph_at_most": grad_in_graph * 1e6,
           "grad_frac_in_graph_at_least": gb / grad_in_graph / 1e9 / peak,
           "launch": launch, "autotuned": run.tuned,
           "notes": "grad_kernel_us: CUDA events around each launch (with the Adam step when it is in the kernel); "
                    "grad_us_in_graph_at_most: the iteration with a separate Adam launch minus a captured Adam step "
                    "alone; factors and G are 16 KB: rows and updates are L2 hits, DRAM traffic is the X gathers"}
    if not args.no_sweep:
        out["sweep"] = sweep_draws(torch, gcp, run, stream, peak, rank)
    return out


def sweep_draws(torch, gcp, run, stream, peak, rank, sizes=(100_000, 1_000_000, 10_000_000)):
    """Whole GCP-Adam iterations (gradient + Adam) on the dense tensor at
    larger draw counts per iteration: the bandwidth-bound reading of the same
    kernels."""
    out = []
    F = gcp.Factors([a[:, :rank] for a in run.F.A])
    # the tuned walk (lanes, chunks, block, layout) with the grid and the
    # replica slabs automatic: both were fitted to 1e5 draws per iteration
    best = dict((run.tuned or {}).get("best") or {"early_draws": 1})
    for key in ("grid_blocks", "max_replicas", "replica_target"):
        best.pop(key, None)
    gcp.gcp_set_tuning(run.h, **best)
    for s in sizes:
        spec = gcp.Sampling(gcp.SAMPLER_UNIFORM, 0, s, 99, 0)
        iters = max(3, min(50, 5_000_000 // s))
        us = time_iterations(torch, gcp, run.h, F, gcp.LOSS_GAUSSIAN, spec, stream, iters=iters) * 1e6
        gbs = s * (4 + row_bytes(4, rank, 4)) / us / 1e3
        out.append({"draws_per_iteration": s, "us_per_iteration": us, "entries_per_s": s / us * 1e6,
                    "algorithmic_gbs": gbs, "frac_of_measured_hbm": gbs / peak,
                    "launch": gcp.gcp_get_launch(run.h, F, s)})
    if run.tuned:
        gcp.gcp_set_tuning(run.h, **run.tuned["best"])
    return out


def count_problem(gcp):
    """The count tensor's gcp_grad workload: (dims, rank, p, q, idx, vals,
    handle, initial factors, stratified spec)."""
    from paper_1906_01687_gb300 import synth
    dims, rank, p, q = (6186, 24, 77, 32), 10, 100_000, 100_000
    idx, vals, _ = synth.count_tensor()
    h = gcp.Handle(gcp.DataTensor.coo(dims, idx, vals))
    A = [(a * 0.3).astype(np.float32) for a in synth.initial_guess(dims, rank, 4, positive=True)]
    spec = gcp.Sampling(gcp.SAMPLER_STRATIFIED, p, q, 1687, 0)
    return dims, rank, p, q, idx, vals, h, A, spec


def form_count(torch, gcp, stream, peak):
    """FP32 vs BF16 factor storage on the count tensor (6186x24x77x32, 5.33M
    nonzeros, rank 10, Poisson-log, stratified 1e5 + 1e5 draws): the whole
    gcp_grad call (ordered zero rejection + gradient + fold), its roofline fraction, and
    the gradient's and the loss estimate's errors against the FP64 oracle (at
    the FP32 factors) on the same draws."""
    import oracle
    from paper_1906_01687_gb300.autotune import autotune, candidates, with_grids
    dims, rank, p, q, idx, vals, h, A, spec = count_problem(gcp)
    XO = oracle.Tensor(dims, coo=np.stack([i.astype(np.int64) for i in idx], axis=1), vals=vals.astype(np.float64))
    SO = oracle.sample(XO, oracle.STRATIFIED, p, q, 1687, 0)
    ref = oracle.grad(dims, [a.astype(np.float64) for a in A], oracle.POISSON_LOG, SO)
    est_spec = gcp.Sampling(gcp.SAMPLER_STRATIFIED, p, q, 7, gcp.STREAM_EST)
    SOe = oracle.sample(XO, oracle.STRATIFIED, p, q, 7, gcp.STREAM_EST)
    F_ref = oracle.loss_estimate(dims, [a.astype(np.float64) for a in A], oracle.POISSON_LOG, SOe)
    call_bytes = {b_f: stratified_call_bytes(dims, len(vals), p, q, rank, b_f) for b_f in (4, 2)}
    out = {"workload": "coo-6186x24x77x32-nnz5330673-r10-poissonlog-stratified-1e5+1e5",
           "metric": "entries/s of gcp_grad (zero rejection + gradient + fold)"}
    for name, bf16 in (("fp32", False), ("bf16", True)):
        F = gcp.Factors(A, bf16=bf16)
        tuned = autotune(h, F, gcp.LOSS_POISSON_LOG, spec, launches=10, stream=stream,
                         configs=with_grids([dict(c, early_draws=1) for c in candidates(rank)], p + q))
        G = F.like()
        t = _time_calls(torch, lambda: gcp.gcp_grad(h, F, gcp.LOSS_POISSON_LOG, G, S=spec, stream=stream), stream, 50)
        for x in G:
            x.zero_()
        gcp.gcp_grad(h, F, gcp.LOSS_POISSON_LOG, G, S=spec, stream=stream)
        stream.synchronize()
        got = [x[:, :rank].double().cpu().numpy() for x in G]
        cb = call_bytes[2 if bf16 else 4]
        out[name] = {"value": (p + q) / t, "us_per_call": t * 1e6, "grad_rel_err_vs_fp64_oracle": rel_err(got, ref),
                     "call_bytes": cb, "frac_of_measured_hbm": cb / t / 1e9 / peak,
                     "launch": gcp.gcp_get_launch(h, F, p + q), "tuning": tuned["best"]}
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


def form_batched(torch, gcp, stream, peak, tau=20, epochs=3):
    """64 independent dense problems (d in {3,4}, dims U[50,2000] with at most
    2e7 entries, ranks {4,8,16,32,64}, mixed losses, 1e4-1e5 draws/iteration):
    one batched launch per step under one CUDA graph, against the same 64
    problems run one after another (each its own graph-replayed epoch)."""
    from paper_1906_01687_gb300 import synth
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
    # algorithmic bytes per iteration over all problems: each draw reads its
    # dense value and d rows and adds d rows; each Adam step moves 32 B per entry
    it_bytes = sum(sh["s"] * (4 + row_bytes(len(sh["dims"]), sh["rank"], 4)) + adam_bytes(sh["dims"], sh["rank"])
                   for sh in shapes)
    torch.cuda.synchronize()
    batch = GcpAdamBatch(specs, tau=tau, alpha=1e-3, kappa=1_000_000, stream=stream, autotune=True)
    batch.capture()
    batch.run_epoch()
    stream.synchronize()
    t_batch = _time_calls(torch, batch.run_epoch, stream, epochs)
    # the Adam step's share of a batched iteration (what fusing it into the
    # gradient launch could save at most): a captured sequence of Adam steps alone
    from paper_1906_01687_gb300.autotune import side_stream
    g_adam = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g_adam, stream=side_stream(stream)):
        for _ in range(tau):
            batch.batch.adam_step(stream=torch.cuda.current_stream())
    t_adam = _time_calls(torch, g_adam.replay, stream, epochs) / tau
    del g_adam
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
        errs.append(rel_err(a, b))
    entries = tau * draws
    return {"workload": f"64 dense problems, d 3-4, dims 50-2000 (<= 2e7 entries), ranks 4-64, mixed losses, "
                        f"{draws} draws/iteration in total, tau {tau}",
            "metric": "sampled-gradient entries/s over one epoch (all problems)",
            "bytes_per_iteration": it_bytes,
            "batched": {"value": entries / t_batch, "ms_per_epoch": t_batch * 1e3,
                        "frac_of_measured_hbm": tau * it_bytes / t_batch / 1e9 / peak,
                        "launches_per_iteration": 1 if batch.fused else 2, "tuning": batch.tuned,
                        "adam_us_per_iteration": t_adam * 1e6,
                        "adam_share_of_iteration": t_adam * tau / t_batch},
            "sequential": {"value": entries / t_seq, "ms_per_epoch": t_seq * 1e3,
                           "frac_of_measured_hbm": tau * it_bytes / t_seq / 1e9 / peak,
                           "launches_per_iteration": 2 * len(specs)},
            "batched_over_sequential": t_seq / t_batch,
            "factor_rel_diff_vs_single_runs_after_2_epochs_max": max(errs)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the other workloads and forms")
    ap.add_argument("--no-sweep", action="store_true", help="skip the draws-per-iteration sweep")
    ap.add_argument("--tuning", default=None, help="JSON gcp_tuning fields to use instead of autotuning")
    ap.add_argument("--nnz", type=int, default=None,
                    help="nonzeros of the benchmark tensor (default 1e8); a smaller tensor of the same shape, "
                         "draws and rank is the small case for profiling")
    ap.add_argument("--form", default=None, choices=["dense100", "count", "batched"],
                    help="run one of the other workloads alone and print its JSON object (the command "
                         "profiled for that workload's kernel breakdown)")
    ap.add_argument("--bf16", action="store_true", help="with --profile: BF16-stored factor rows")
    ap.add_argument("--profile", type=int, default=0, metavar="ITERS",
                    help="only set up the benchmark's run and take ITERS eager GCP-Adam iterations, then exit "
                         "(the command profiled with ncu; prints one line of timing); with --form count, ITERS "
                         "gcp_grad calls on the count tensor instead; with --form dense100, ITERS iterations on "
                         "the dense 100^4 tensor")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.nnz is not None:
        global NNZ, WORKLOAD
        NNZ = int(args.nnz)
        WORKLOAD = WORKLOAD.replace("nnz1e8", f"nnz{NNZ:.0e}".replace("+0", ""))
    if args.impl == "reference":
        return reference_arm(args)
    if args.profile:
        return profile_arm(args)
    if args.form:
        return form_arm(args)
    return ours_arm(args)


def form_arm(args):
    """One of the other workloads alone (one JSON object)."""
    import torch
    from paper_1906_01687_gb300 import gcp
    stream = torch.cuda.Stream()
    peak, _ = peaks()
    fn = {"dense100": lambda: form_dense100(torch, gcp, stream, peak, args),
          "count": lambda: form_count(torch, gcp, stream, peak),
          "batched": lambda: form_batched(torch, gcp, stream, peak)}[args.form]
    print(json.dumps({"form": args.form, args.form: fn()}), flush=True)
    return 0


def profile_arm(args):
    """The benchmark's run set up as in ours_arm (no autotuning: the shape
    given by --tuning, else the automatic one), then --profile eager
    iterations: a short, bounded command for ncu.  With --form count, the
    count tensor's gcp_grad call instead (--profile calls); with --form
    dense100, eager GCP-Adam iterations on the dense 100^4 tensor."""
    import torch
    from paper_1906_01687_gb300 import gcp
    from paper_1906_01687_gb300.adam import GcpAdam
    stream = torch.cuda.Stream()
    if args.form == "count":
        return profile_count(args, torch, gcp, stream)
    if args.form == "dense100":
        return profile_dense100(args, torch, gcp, stream)
    if args.form:
        raise SystemExit("--profile takes no --form but count and dense100")
    idx, A0, _ = large_input()
    XT = gcp.DataTensor.coo(DIMS, idx, None)
    with torch.cuda.stream(stream):
        run = GcpAdam(XT, A0, gcp.LOSS_BERNOULLI_LOGIT, gcp.SAMPLER_SEMI_STRATIFIED, P_DRAWS, Q_DRAWS, EST_P, EST_Q,
                      seed=1687, est_seed=7, alpha=ALPHA, tau=TAU, kappa=1_000_000, stream=stream, bf16=args.bf16)
        if args.tuning:
            gcp.gcp_set_tuning(run.h, **json.loads(args.tuning))
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    gcp.gcp_profile(run.h, True, args.profile)
    with torch.cuda.stream(stream):
        a.record(stream)
        for _ in range(args.profile):
            run.iteration()
        b.record(stream)
    stream.synchronize()
    ms, n = gcp.gcp_profile_read(run.h, 0)
    gcp.gcp_profile(run.h, False)
    print(json.dumps({"profile": WORKLOAD + ("-bf16" if args.bf16 else ""), "iterations": args.profile,
                      "us_per_iteration": a.elapsed_time(b) * 1e3 / args.profile,
                      "grad_kernel_us": ms * 1e3 / max(n, 1),
                      "launch": gcp.gcp_get_launch(run.h, run.F, P_DRAWS + Q_DRAWS)}), flush=True)
    return 0


def profile_count(args, torch, gcp, stream):
    """--profile calls of gcp_grad on the count tensor (ordered zero pass,
    gradient, replica fold) in the shape --tuning gives, with the gradient
    kernel's own event time beside the call's."""
    dims, rank, p, q, idx, vals, h, A, spec = count_problem(gcp)
    F = gcp.Factors(A)
    G = F.like()
    if args.tuning:
        gcp.gcp_set_tuning(h, **json.loads(args.tuning))
    call = lambda: gcp.gcp_grad(h, F, gcp.LOSS_POISSON_LOG, G, S=spec, stream=stream)
    call()
    stream.synchronize()
    t_call = _time_calls(torch, call, stream, args.profile)
    gcp.gcp_profile(h, True, args.profile)
    for _ in range(args.profile):
        call()
    stream.synchronize()
    ms, n = gcp.gcp_profile_read(h, 0)
    gcp.gcp_profile(h, False)
    print(json.dumps({"profile": "coo-6186x24x77x32-nnz5330673-r10-poissonlog-stratified-1e5+1e5",
                      "calls": args.profile, "us_per_call": t_call * 1e6, "grad_kernel_us": ms * 1e3 / max(n, 1),
                      "launch": gcp.gcp_get_launch(h, F, p + q)}), flush=True)
    return 0


def profile_dense100(args, torch, gcp, stream):
    """--profile eager GCP-Adam iterations (gradient + Adam launches) on the
    dense 100^4 tensor, rank 10, Gaussian, uniform 1e5 draws, in the shape
    --tuning gives, with the gradient kernel's own event time."""
    from paper_1906_01687_gb300 import synth
    from paper_1906_01687_gb300.adam import GcpAdam
    dims, rank, s = (100, 100, 100, 100), 10, 100_000
    X32, _ = synth.dense_100_4()
    A0 = synth.initial_guess(dims, rank, seed=3, target_norm=float(np.linalg.norm(X32)))
    XT = gcp.DataTensor.dense(X32, device=stream.device)
    with torch.cuda.stream(stream):
        run = GcpAdam(XT, A0, gcp.LOSS_GAUSSIAN, gcp.SAMPLER_UNIFORM, 0, s, 0, 100_000, seed=1687, est_seed=7,
                      alpha=1e-3, tau=100, kappa=1_000_000, stream=stream)
        if args.tuning:
            gcp.gcp_set_tuning(run.h, **json.loads(args.tuning))
    iter_s = time_iterations(torch, gcp, run.h, run.F, run.loss, run.spec, stream, iters=50)
    mean_s, n, adam_s = time_grad_kernel(torch, gcp, run.h, run.iteration, stream, launches=args.profile)
    print(json.dumps({"profile": "dense-100x100x100x100-r10-gaussian-uniform-s1e5", "iterations": args.profile,
                      "iteration_us_in_graph": iter_s * 1e6, "grad_kernel_us": mean_s * 1e6,
                      "adam_kernel_us": adam_s * 1e6, "launch": gcp.gcp_get_launch(run.h, run.F, s)}), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
