"""Fitting a dense tensor with GCP-Adam (Alg. 4) from Python.

    python examples/fit_dense.py

Fits a planted rank-3 Gaussian problem (20 x 30 x 40) with uniform sampling
(1000 draws per iteration, a fixed 500-entry loss-estimate set) and prints
the estimated loss before and after.  Needs a GPU and the built library.
"""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), ".."))

from paper_1906_01687_gb300 import gcp, synth  # noqa: E402
from paper_1906_01687_gb300.adam import GcpAdam  # noqa: E402


def fit(max_epochs=50):
    """Returns (the optimizer state after the fit, the estimate history, the factors)."""
    X = synth.dense_small()[0]  # or any numpy/torch array; COO via DataTensor.coo
    A0 = synth.initial_guess(X.shape, 3, seed=1, target_norm=float(np.linalg.norm(X)))
    run = GcpAdam(gcp.DataTensor.dense(X), A0, gcp.LOSS_GAUSSIAN, gcp.SAMPLER_UNIFORM, p=0, q=1000,
                  est_p=0, est_q=500, seed=1, est_seed=2, tau=100)
    state = run.fit(max_epochs=max_epochs)  # epochs replayed from one CUDA graph
    return state, run.history, run.factors()


if __name__ == "__main__":
    state, history, A = fit()
    print(f"estimated loss {history[0]:.4g} -> {state['F']:.4g} after {len(history) - 1} epochs; "
          f"factor shapes {[a.shape for a in A]}")
