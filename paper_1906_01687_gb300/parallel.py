"""Sample-parallel GCP-Adam: one problem's draws split across GPUs.

Every draw of an iteration is a pure function of its number (counter-based
Philox sampling, Algs. 1-3), so rank g of P takes the contiguous range
draw_range(g, P, n) of the iteration's n draws, computes the sampled
gradient of those draws alone (gcp_grad_range), and one all-reduce (sum) of
the flat gradient buffer gives every rank the gradient of all n draws: the
same sample set, and the same gradient up to the FP32 summation order, as one
GPU drawing all of them.  The Adam step (Alg. 4) then runs replicated on
every rank from identical inputs, and so do the fixed-sample loss estimate
and the epoch's accept-or-revert decision, so the ranks' factors stay
identical without further exchange.  This is the parallel use of sampling
that the paper's conclusions (Section 6) point to: each rank computes on a
subset of the entries.

The host-side pieces (draw_range, the flat gradient layout, the sum across
ranks) need no GPU; the optimizer class loads the CUDA library and fails
loudly without it.
"""
from __future__ import annotations

import math
from typing import List, Optional, Sequence, Tuple

import torch


def draw_range(rank: int, world: int, n: int) -> Tuple[int, int]:
    """(first, count) of rank's share of draws 0..n-1: contiguous ranges that
    partition [0, n), sizes differing by at most one."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError(f"bad split: rank {rank} of {world}, {n} draws")
    first = n * rank // world
    return first, n * (rank + 1) // world - first


def flat_buffers(rows: Sequence[int], ld: int, device="cuda", dtype=torch.float32) -> Tuple[torch.Tensor, List]:
    """One contiguous zeroed buffer holding every mode's n_k x ld matrix, and
    the per-mode views into it (each 16-byte aligned: ld is a multiple of 4),
    so that the whole gradient is summed across ranks by one collective."""
    if ld % 4:
        raise ValueError("ld must be a multiple of 4 (16-byte rows)")
    flat = torch.zeros(sum(rows) * ld, dtype=dtype, device=device)
    views, off = [], 0
    for n in rows:
        views.append(flat[off:off + n * ld].view(n, ld))
        off += n * ld
    return flat, views


def sum_across_ranks(flat: torch.Tensor, group=None) -> torch.Tensor:
    """The sum of every rank's flat gradient, in place on every rank (one
    all-reduce; a no-op on a single rank)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(flat, op=dist.ReduceOp.SUM, group=group)
    return flat


class SampleParallelGcpAdam:
    """GCP-Adam (Alg. 4) on one problem whose draws are split over the ranks
    of a process group (NCCL across GPUs; a single rank needs none).

    Every rank holds the whole data tensor and replicated factors, moments
    and optimizer state.  Per iteration: the partial sampled gradient of the
    rank's draw range, one all-reduce of the flat gradient, the Adam step.
    Per epoch: the loss estimate on the fixed list (every rank, the whole
    list) and the accept-or-revert kernel.
    """

    def __init__(self, X, A0: Sequence, loss: int, sampler: int, p: int, q: int, est_p: int, est_q: int,
                 seed: int, est_seed: int, alpha: float = 0.01, beta1: float = 0.9, beta2: float = 0.999,
                 eps: float = 1e-8, tau: int = 1000, kappa: int = 1, nu: float = 0.1, lower: float = -math.inf,
                 bf16: bool = False, problem: int = 0, oversample: float = 1.1, eps_inside_sqrt: bool = True,
                 group=None, stream=None, early_draws: bool = True):
        from . import gcp
        import torch.distributed as dist
        self.gcp = gcp
        self.group = group
        if dist.is_available() and dist.is_initialized():
            self.world, self.rank = dist.get_world_size(group), dist.get_rank(group)
        else:
            self.world, self.rank = 1, 0
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.stream.wait_stream(torch.cuda.current_stream())
        self.h = gcp.Handle(X, stream=self.stream)
        if early_draws:
            gcp.gcp_set_tuning(self.h, early_draws=1)
        self.loss = loss
        self.tau, self.kappa, self.nu = int(tau), int(kappa), float(nu)
        self.adam = dict(beta1=beta1, beta2=beta2, eps=eps, lower=lower, eps_inside_sqrt=eps_inside_sqrt)
        device = self.stream.device
        with torch.cuda.stream(self.stream):
            self.F = gcp.Factors(A0, bf16=bf16, device=device)
            self.G_flat, self.G = flat_buffers(self.F.dims, self.F.ld, device=device)
            self.B, self.C = self.F.like(), self.F.like()
            self.SA, self.SB, self.SC = self.F.like(), self.F.like(), self.F.like()
            self.state = gcp.new_state(device)
        self.spec = gcp.Sampling(sampler, p, q, seed, 0, problem, oversample)
        self.first, self.count = draw_range(self.rank, self.world, self.spec.count())
        est_spec = gcp.Sampling(sampler, est_p, est_q, est_seed, gcp.STREAM_EST, problem, oversample)
        gcp.gcp_reserve(self.h, self.spec, stream=self.stream)
        gcp.gcp_reserve(self.h, est_spec, stream=self.stream)
        self.est = gcp.gcp_sample(self.h, est_spec, stream=self.stream)
        gcp.gcp_state_init(self.state, alpha, stream=self.stream)
        gcp.gcp_loss_est(self.h, self.F, loss, self.est, self.state[0:1], stream=self.stream)
        gcp.gcp_epoch_begin(self.F, self.B, self.C, self.SA, self.SB, self.SC, self.state, stream=self.stream)
        self.history = []

    def partial_gradient(self):
        """This rank's share: the sampled gradient of its draw range (into G)."""
        self.gcp.gcp_grad_range(self.h, self.F, self.loss, self.G, self.spec, self.first, self.count,
                                stream_dev=self.state[3:4], stream=self.stream)

    def iteration(self):
        self.partial_gradient()
        with torch.cuda.stream(self.stream):
            sum_across_ranks(self.G_flat, self.group)
        self.gcp.gcp_adam_step(self.F, self.G, self.B, self.C, self.state, stream=self.stream, **self.adam)

    def end_epoch(self):
        gcp = self.gcp
        gcp.gcp_loss_est(self.h, self.F, self.loss, self.est, self.state[0:1], stream=self.stream)
        gcp.gcp_epoch_end(self.F, self.B, self.C, self.SA, self.SB, self.SC, self.state, self.tau, self.nu,
                          self.kappa, stream=self.stream)

    def run_epoch(self):
        for _ in range(self.tau):
            self.iteration()
        self.end_epoch()

    def status(self) -> dict:
        self.stream.synchronize()
        return self.gcp.read_state(self.state)

    def fit(self, max_epochs: int = 1000) -> dict:
        st = self.status()
        self.history.append(st["F"])
        for _ in range(max_epochs):
            self.run_epoch()
            st = self.status()
            self.history.append(st["F"])
            if st["done"]:
                break
        return st

    def factors(self):
        self.stream.synchronize()
        return self.F.numpy()
