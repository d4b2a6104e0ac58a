"""GCP-Adam for many independent problems at once (multi-start runs, uneven
dims, ranks and losses), through the batched C-ABI entry points.

Every problem follows Alg. 4 on its own: its own draws (Philox key
(seed, problem), stream word = its iteration counter), loss estimate, Adam
state, learning-rate decay and stopping.  Each step of the epoch is one
kernel launch for all problems; the whole epoch (tau iterations, loss
estimates, accept/revert) is captured once in a CUDA graph and replayed.
"""
from __future__ import annotations

import math
from typing import Optional, Sequence

import numpy as np
import torch

from . import gcp


class GcpAdamBatch:
    def __init__(self, specs: Sequence[dict], tau: int = 1000, kappa: int = 1, nu: float = 0.1,
                 alpha: float = 0.01, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8,
                 lower: float = -math.inf, bf16: bool = False, stream=None, autotune: bool = False):
        """specs: dicts with X (dense numpy array or DataTensor), A0 (factor
        list), loss (int), s (draws per iteration), est (loss-estimate draws),
        seed, est_seed, and optional problem (key word; default its index)."""
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.stream.wait_stream(torch.cuda.current_stream())
        self.tau = int(tau)
        device = self.stream.device
        self.problems = []
        self.handles = []
        with torch.cuda.stream(self.stream):
            for i, sp in enumerate(specs):
                X = sp["X"] if isinstance(sp["X"], gcp.DataTensor) else gcp.DataTensor.dense(sp["X"], device=device)
                h = gcp.Handle(X, stream=self.stream)
                self.handles.append(h)
                problem = int(sp.get("problem", i))
                F = gcp.Factors(sp["A0"], bf16=bf16, device=device)
                est = gcp.gcp_sample(h, gcp.Sampling(gcp.SAMPLER_UNIFORM, 0, int(sp["est"]), int(sp["est_seed"]),
                                                     gcp.STREAM_EST, problem), stream=self.stream)
                state = gcp.new_state(device)
                gcp.gcp_state_init(state, alpha, stream=self.stream)
                self.problems.append(dict(
                    X=X, F=F, loss=int(sp["loss"]), est=est, state=state,
                    S=gcp.Sampling(gcp.SAMPLER_UNIFORM, 0, int(sp["s"]), int(sp["seed"]), 0, problem),
                    G=F.like(), B=F.like(), C=F.like(), SA=F.like(), SB=F.like(), SC=F.like(),
                    adam=dict(beta1=beta1, beta2=beta2, eps=eps, lower=lower, eps_inside_sqrt=True),
                    epoch=dict(tau=tau, nu=nu, kappa=kappa)))
        self.batch = gcp.Batch(self.problems, stream=self.stream)
        self.batch.loss_est(stream=self.stream)
        self.batch.epoch_begin(stream=self.stream)
        self.graph = None
        self.tuned = None
        if autotune:
            self.tuned = self.autotune()

    # -- launches ---------------------------------------------------------------
    def iteration(self):
        self.batch.iteration(stream=self.stream)

    def enqueue_epoch(self):
        for _ in range(self.tau):
            self.batch.iteration(stream=self.stream)
        self.batch.loss_est(stream=self.stream)
        self.batch.epoch_end(stream=self.stream)

    def capture(self):
        self.stream.synchronize()
        g = torch.cuda.CUDAGraph()
        from .autotune import side_stream
        cap = side_stream(self.stream)
        with torch.cuda.graph(g, stream=cap):
            saved, self.stream = self.stream, torch.cuda.current_stream()
            try:
                self.enqueue_epoch()
            finally:
                self.stream = saved
        self.graph = g
        return g

    def run_epoch(self):
        if self.graph is not None:
            with torch.cuda.stream(self.stream):
                self.graph.replay()
        else:
            self.enqueue_epoch()

    def states(self):
        self.stream.synchronize()
        return [gcp.read_state(p["state"]) for p in self.problems]

    def fit(self, max_epochs: int = 100, use_graph: bool = True):
        if use_graph and self.graph is None:
            self.capture()
        for _ in range(max_epochs):
            self.run_epoch()
            if all(st["done"] for st in self.states()):
                break
        return self.states()

    def factors(self, i):
        self.stream.synchronize()
        return self.problems[i]["F"].numpy()

    @property
    def draws_per_iteration(self) -> int:
        return sum(p["S"].q for p in self.problems)

    # -- launch shape ---------------------------------------------------------------
    def autotune(self, launches: int = 10):
        """Times the batched gradient for block sizes and grid sizes on a
        throwaway copy of the batch (same draws and shapes) and keeps the
        fastest; returns it with its time."""
        import statistics
        shadow = []
        with torch.cuda.stream(self.stream):
            for p in self.problems:
                F = gcp.Factors([a[:, : p["F"].rank] for a in p["F"].A], bf16=p["F"].bf16, device=p["F"].A[0].device)
                st = gcp.new_state(F.A[0].device)
                gcp.gcp_state_init(st, 0.0, stream=self.stream)
                q = dict(p)
                q.update(F=F, state=st, G=F.like(), B=F.like(), C=F.like(), SA=F.like(), SB=F.like(), SC=F.like())
                shadow.append(q)
        tb = gcp.Batch(shadow, stream=self.stream)
        best, best_t = None, float("inf")
        sms = torch.cuda.get_device_properties(self.stream.device).multi_processor_count
        for block in (128, 256):
            for waves in (0, 1, 2, 4):
                grid = 0 if waves == 0 else sms * waves * (256 // block)
                tb.set_tuning(block, grid)
                tb.grad(stream=self.stream)
                self.stream.synchronize()
                evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                       for _ in range(launches)]
                with torch.cuda.stream(self.stream):
                    torch.cuda._sleep(50_000_000)
                    for a, b in evs:
                        a.record(self.stream)
                        tb.grad(stream=self.stream)
                        b.record(self.stream)
                self.stream.synchronize()
                t = statistics.median(a.elapsed_time(b) for a, b in evs) * 1e-3
                if t < best_t:
                    best, best_t = dict(block=block, grid_blocks=grid), t
        tb.close()
        self.batch.set_tuning(**best)
        return dict(best=best, seconds=best_t)
