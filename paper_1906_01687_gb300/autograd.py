"""torch.autograd.Function over the sampled GCP loss.

Forward: the loss estimate F-hat(A_1..A_d) on a fixed list of drawn entries
(Eqs. (5.1)-(5.2), FP64 result).  Backward: the sampled gradient of
Eq. (4.3) on the same list, which is exactly dF-hat/dA_k (the list's weights
and classes enter both the same way), scaled by the incoming gradient.
Both directions run in the library's CUDA kernels.
"""
from __future__ import annotations

import torch

from . import gcp


class GcpLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, handle: gcp.Handle, loss: int, samples: gcp.SampleList, *A: torch.Tensor):
        F = gcp.Factors([a.detach() for a in A], device=A[0].device)
        out = torch.zeros(1, dtype=torch.float64, device=A[0].device)
        gcp.gcp_loss_est(handle, F, loss, samples, out)
        ctx.handle, ctx.loss, ctx.samples, ctx.F = handle, loss, samples, F
        ctx.rank = A[0].shape[1]
        return out[0]

    @staticmethod
    def backward(ctx, grad_out):
        G = ctx.F.like()
        gcp.gcp_grad(ctx.handle, ctx.F, ctx.loss, G, samples=ctx.samples)
        scale = grad_out.to(torch.float32)
        grads = [g[:, : ctx.rank] * scale for g in G]
        return (None, None, None, *grads)


def gcp_loss(handle: gcp.Handle, loss: int, samples: gcp.SampleList, *A: torch.Tensor) -> torch.Tensor:
    """F-hat of the factor matrices A_k (n_k x r FP32 CUDA tensors) on a fixed list."""
    return GcpLoss.apply(handle, loss, samples, *A)
