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
                 lower: float = -math.inf, bf16: bool = False, stream=None, autotune: bool = False,
                 fused: bool = False):
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
        self.fused = bool(fused)  # one launch per iteration (gradient and Adam fused) instead of two
        self.tuned = None
        if autotune:
            self.tuned = self.autotune()

    # -- launches ---------------------------------------------------------------
    def iteration(self):
        if self.fused:
            self.batch.iteration_fused(stream=self.stream)
        else:
            self.batch.iteration(stream=self.stream)

    def enqueue_epoch(self):
        for _ in range(self.tau):
            self.iteration()
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
    SHAPES = [(cpl, target, maxr) for cpl in (1, 2, 4) for target, maxr in ((64, 32), (16, 32), (0, 1))]

    def autotune(self, iterations: int = 10, shapes=None):
        """Chooses the batched iteration's form and shape -- one persistent
        launch (gradient and Adam fused) or two launches, threads per block and
        blocks (grid waves), chunks per lane (the rows per warp step) and the
        replica width (the pre-reduction of heavily hit rows) -- by timing whole
        iterations on a throwaway copy of the batch (same draws and shapes),
        captured in a CUDA graph as an epoch is; keeps the fastest.  Returns it
        with its time per iteration and the per-problem shapes it gives."""
        from .autotune import side_stream
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
        cap = side_stream(self.stream)
        sms = torch.cuda.get_device_properties(self.stream.device).multi_processor_count

        def timed(step):
            with torch.cuda.stream(self.stream):
                step(self.stream)
            self.stream.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=cap):
                for _ in range(iterations):
                    step(cap)
            with torch.cuda.stream(self.stream):
                g.replay()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(self.stream)
                g.replay()
                g.replay()
                b.record(self.stream)
            self.stream.synchronize()
            del g
            return a.elapsed_time(b) * 1e-3 / (2 * iterations)

        best, best_t, tried, best_fused_t = None, float("inf"), 0, float("inf")
        for cpl, target, maxr in (shapes or self.SHAPES):
            tb.set_shape(cpl, target, maxr, stream=self.stream)
            # the one-launch iteration (its grid is one resident wave of 256-thread blocks)
            t = timed(lambda st: tb.iteration_fused(stream=st))
            tried += 1
            best_fused_t = min(best_fused_t, t)
            if t < best_t:
                best_t = t
                best = dict(fused=True, block=0, grid_blocks=0, chunks_per_lane=cpl, replica_target=target,
                            max_replicas=maxr)
            for block in (128, 256):
                for waves in (0, 1, 2, 4):
                    grid = 0 if waves == 0 else sms * waves * (256 // block)
                    tb.set_tuning(block, grid)
                    t = timed(lambda st: tb.iteration(stream=st))
                    tried += 1
                    if t < best_t:
                        best_t = t
                        best = dict(fused=False, block=block, grid_blocks=grid, chunks_per_lane=cpl,
                                    replica_target=target, max_replicas=maxr)
        tb.close()
        self.fused = best["fused"]
        self.set_shape(**{k: v for k, v in best.items() if k != "fused"})
        shapes = [self.batch.get_shape(i) for i in range(len(self.problems))]
        return dict(best=best, seconds_per_iteration=best_t, best_fused_seconds_per_iteration=best_fused_t,
                    tried=tried, shapes=shapes)

    def set_shape(self, block=0, grid_blocks=0, chunks_per_lane=0, replica_target=0, max_replicas=0):
        """Sets the batched gradient's launch and per-problem shape (before capture)."""
        self.batch.set_shape(chunks_per_lane, replica_target, max_replicas, stream=self.stream)
        self.batch.set_tuning(block, grid_blocks)
        self.graph = None
