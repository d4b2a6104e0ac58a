"""GCP-Adam (Alg. 4) driven through the C ABI, with device-resident state.

One epoch is: tau x (fused sampled gradient, Adam step with projection),
then the fixed-sample loss estimate and the accept-or-revert decision, all
enqueued on one stream.  The Philox stream word of each iteration's draws is
read by the gradient kernel from the device state (``iter``), so an epoch's
launches are identical every time and can be captured once in a CUDA graph
and replayed; the host reads the 64-byte state only to decide when to stop.

The gradient kernel of each iteration makes its first draws while the
previous iteration's Adam step is still running (the handle's early_draws
tuning, on by default here): the draws read only the data tensor, and the
kernel checks its predicted stream word against the device counter after
waiting, so the draws are the same as with the wait first.

Readings of Alg. 4 (shared with the oracle's driver): the bias correction of
step t uses t + 1; an equal estimate is accepted; a non-finite one fails; the
draws' stream word counts every iteration ever run and is never wound back.
"""
from __future__ import annotations

import math
from typing import Optional, Sequence

import torch

from . import gcp


class GcpAdam:
    def __init__(self, X: gcp.DataTensor, A0: Sequence, loss: int, sampler: int, p: int, q: int,
                 est_p: int, est_q: int, seed: int, est_seed: int, alpha: float = 0.01, beta1: float = 0.9,
                 beta2: float = 0.999, eps: float = 1e-8, tau: int = 1000, kappa: int = 1, nu: float = 0.1,
                 lower: float = -math.inf, bf16: bool = False, problem: int = 0, oversample: float = 1.1,
                 handle: Optional[gcp.Handle] = None, eps_inside_sqrt: bool = True, stream=None,
                 autotune: bool = False, early_draws: bool = True):
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.stream.wait_stream(torch.cuda.current_stream())  # X and A0 may come from the current stream
        self.h = handle if handle is not None else gcp.Handle(X, stream=self.stream)
        self.early_draws = bool(early_draws)
        if self.early_draws:  # every other field of the handle's launch shape automatic
            gcp.gcp_set_tuning(self.h, early_draws=1)
        self.loss = loss
        self.tau, self.kappa, self.nu = int(tau), int(kappa), float(nu)
        self.adam = dict(beta1=beta1, beta2=beta2, eps=eps, lower=lower, eps_inside_sqrt=eps_inside_sqrt)
        device = self.stream.device if hasattr(self.stream, "device") else "cuda"
        with torch.cuda.stream(self.stream):
            self.F = gcp.Factors(A0, bf16=bf16, device=device)
            self.G, self.B, self.C = self.F.like(), self.F.like(), self.F.like()
            self.SA, self.SB, self.SC = self.F.like(), self.F.like(), self.F.like()
            self.state = gcp.new_state(device)
        self.spec = gcp.Sampling(sampler, p, q, seed, 0, problem, oversample)
        est_spec = gcp.Sampling(sampler, est_p, est_q, est_seed, gcp.STREAM_EST, problem, oversample)
        gcp.gcp_reserve(self.h, self.spec, stream=self.stream)
        gcp.gcp_reserve(self.h, est_spec, stream=self.stream)
        self.est = gcp.gcp_sample(self.h, est_spec, stream=self.stream)
        gcp.gcp_state_init(self.state, alpha, stream=self.stream)
        gcp.gcp_loss_est(self.h, self.F, loss, self.est, self.state[0:1], stream=self.stream)
        gcp.gcp_epoch_begin(self.F, self.B, self.C, self.SA, self.SB, self.SC, self.state, stream=self.stream)
        self.graph = None
        self.history = []
        self.tuned = None
        if autotune:
            self.tuned = self.autotune()

    # -- one epoch of launches --------------------------------------------
    def iteration(self):
        """One sampled gradient + Adam step (draws from the device iteration counter)."""
        gcp.gcp_iteration(self.h, self.F, self.loss, self.spec, self.G, self.B, self.C, self.state,
                          stream_dev=self.state[3:4], stream=self.stream, **self.adam)

    def end_epoch(self):
        gcp.gcp_loss_est(self.h, self.F, self.loss, self.est, self.state[0:1], stream=self.stream)
        gcp.gcp_epoch_end(self.F, self.B, self.C, self.SA, self.SB, self.SC, self.state, self.tau, self.nu,
                          self.kappa, stream=self.stream)

    def enqueue_epoch(self):
        for _ in range(self.tau):
            self.iteration()
        self.end_epoch()

    def _warm(self):
        """Runs every kernel of an epoch once on throwaway copies, so that no
        kernel is first loaded inside a graph capture."""
        with torch.cuda.stream(self.stream):
            F = gcp.Factors([a[:, : self.F.rank] for a in self.F.A], bf16=self.F.bf16, device=self.F.A[0].device)
            G, B, C, SA, SB, SC = (F.like() for _ in range(6))
            st = gcp.new_state(self.F.A[0].device)
        gcp.gcp_state_init(st, 0.0, stream=self.stream)
        gcp.gcp_iteration(self.h, F, self.loss, self.spec, G, B, C, st, stream_dev=st[3:4], stream=self.stream,
                          **self.adam)
        gcp.gcp_loss_est(self.h, F, self.loss, self.est, st[0:1], stream=self.stream)
        gcp.gcp_epoch_end(F, B, C, SA, SB, SC, st, self.tau, self.nu, self.kappa, stream=self.stream)
        self.stream.synchronize()

    def autotune(self, launches: int = 20):
        """Chooses the gradient's launch shape by timing whole iterations
        (gradient + Adam with the replica fold) on throwaway copies, captured
        in a CUDA graph as an epoch is, so that the overlap between one
        iteration's kernels and the next is part of the measurement."""
        from .autotune import autotune as _autotune, candidates
        with torch.cuda.stream(self.stream):
            F = gcp.Factors([a[:, : self.F.rank] for a in self.F.A], bf16=self.F.bf16, device=self.F.A[0].device)
            G, B, C = F.like(), F.like(), F.like()
            st = gcp.new_state(self.F.A[0].device)
            gcp.gcp_state_init(st, 0.0, stream=self.stream)

        def call(spec, stream):
            gcp.gcp_iteration(self.h, F, self.loss, spec, G, B, C, st, stream_dev=st[3:4], stream=stream,
                              **self.adam)
        from .autotune import with_grids
        configs = with_grids([dict(c, early_draws=int(self.early_draws)) for c in candidates(F.rank)], self.spec.count())
        return _autotune(self.h, F, self.loss, self.spec, configs=configs, launches=launches, stream=self.stream,
                         call=call, graph=True)

    def capture(self, refresh: bool = False):
        """Captures one epoch's launches in a CUDA graph (replayed by run_epoch).
        With refresh the graph first takes up new contents of the data
        tensor's arrays (gcp_refresh: the caller rewrites them in place
        between replays, e.g. a new upload of the same-shaped tensor)."""
        self._warm()
        self.stream.synchronize()
        g = torch.cuda.CUDAGraph()
        from .autotune import side_stream
        cap = side_stream(self.stream)
        with torch.cuda.graph(g, stream=cap):
            saved, self.stream = self.stream, torch.cuda.current_stream()
            try:
                if refresh:
                    gcp.gcp_refresh(self.h, stream=self.stream)
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

    def status(self) -> dict:
        self.stream.synchronize()
        return gcp.read_state(self.state)

    def fit(self, max_epochs: int = 1000, use_graph: bool = True, log=None) -> dict:
        if use_graph and self.graph is None:
            self.capture()
        st = self.status()
        self.history.append(st["F"])
        for epoch in range(max_epochs):
            self.run_epoch()
            st = self.status()
            self.history.append(st["F"])
            if log is not None:
                log(dict(epoch=epoch + 1, **st))
            if st["done"]:
                break
        return st

    def factors(self):
        self.stream.synchronize()
        return self.F.numpy()

    # -- checkpoint / resume ----------------------------------------------------
    def state_dict(self) -> dict:
        """Everything a resumed run needs: factors (FP32 master), Adam moments,
        the epoch snapshot and the 64-byte optimizer state.  The draws are a
        function of (seed, problem, iteration), so a resumed run draws exactly
        what the uninterrupted run would have."""
        self.stream.synchronize()
        cpu = lambda xs: [x.detach().cpu().clone() for x in xs]
        return dict(A=cpu(self.F.A), B=cpu(self.B), C=cpu(self.C), SA=cpu(self.SA), SB=cpu(self.SB),
                    SC=cpu(self.SC), state=self.state.detach().cpu().clone(),
                    spec=dict(kind=self.spec.kind, p=self.spec.p, q=self.spec.q, seed=self.spec.seed,
                              problem=self.spec.problem))

    def load_state_dict(self, sd: dict):
        spec = sd["spec"]
        if (spec["kind"], spec["p"], spec["q"], spec["seed"], spec["problem"]) != (
                self.spec.kind, self.spec.p, self.spec.q, self.spec.seed, self.spec.problem):
            raise ValueError("checkpoint belongs to a different sampling spec")
        with torch.cuda.stream(self.stream):
            for name in ("B", "C", "SA", "SB", "SC"):
                for dst, src in zip(getattr(self, name), sd[name]):
                    dst.copy_(src, non_blocking=True)
            for dst, src in zip(self.F.A, sd["A"]):
                dst.copy_(src, non_blocking=True)
            self.state.copy_(sd["state"], non_blocking=True)
            if self.F.A_bf16 is not None:
                gcp.gcp_factors_to_bf16(self.F, stream=self.stream)
        self.stream.synchronize()
