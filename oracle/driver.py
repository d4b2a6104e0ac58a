"""GCP-Adam (Alg. 4) over the FP64 oracle's sampled gradient.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The loop follows Alg. 4 in its order: estimate F-hat on a fixed sample set;
per epoch save {A, B, C} and F-hat, run tau iterations of (sampled gradient,
Adam step with projection, t += 1), re-estimate F-hat, and on an increase
restore the saved state, wind t back by tau, multiply alpha by nu and count a
bad epoch; stop after more than kappa bad epochs (or max_epochs).

Readings: the bias correction of step t uses t + 1 (see ``adam_step``); an
estimate equal to the previous one is accepted; a non-finite estimate counts
as an increase.  The Philox stream of iteration t's draws is the running
count of iterations ever taken (never wound back), so a retried epoch draws
fresh samples.
"""
import math

import numpy as np

from . import adam_step, concat_factors, grad, loss_estimate, sample, split_factors

EST_STREAM = 0xFFFFFFFFFFFFFFFF  # the Philox stream word of the fixed estimate set


def gcp_adam(X, factors0, loss, kind, p, q, est_p, est_q, seed, est_seed,
             alpha=0.01, beta1=0.9, beta2=0.999, eps=1e-8, tau=1000, kappa=1, nu=0.1,
             lower=-math.inf, max_epochs=1000, problem=0, log=None, first_iter=0):
    """Runs Alg. 4 from factors0 and returns (factors, history of F-hat per
    epoch).  first_iter is the stream word of the first iteration's draws
    (0 for a run that starts fresh; tests use it to start a run where another
    run's draws stand)."""
    dims = X.dims
    rank = factors0[0].shape[1]
    A = concat_factors(factors0).copy()
    B = np.zeros_like(A)
    C = np.zeros_like(A)
    est = sample(X, kind, est_p, est_q, est_seed, EST_STREAM, problem=problem)
    F = loss_estimate(dims, split_factors(A, dims, rank), loss, est)
    history = [F]
    c = 0
    t = 0
    it = first_iter
    epochs = 0
    while c <= kappa and epochs < max_epochs:
        saved = (A.copy(), B.copy(), C.copy())
        F_old = F
        for _ in range(tau):
            S = sample(X, kind, p, q, seed, it, problem=problem)
            G = concat_factors(grad(dims, split_factors(A, dims, rank), loss, S))
            adam_step(A, B, C, G, alpha, beta1, beta2, eps, lower, t)
            t += 1
            it += 1
        F = loss_estimate(dims, split_factors(A, dims, rank), loss, est)
        epochs += 1
        if not (F <= F_old):
            A, B, C = saved
            F = F_old
            t -= tau
            alpha *= nu
            c += 1
        history.append(F)
        if log is not None:
            log(dict(epoch=epochs, F=F, alpha=alpha, t=t, bad=c))
    return split_factors(A, dims, rank), history
