"""Pins of the oracle's Adam step (Alg. 4) and of the GCP-Adam loop.

- With eps outside the root, several steps equal torch.optim.Adam (the
  textbook method of Kingma and Ba, an independent implementation).
- With eps inside the root as Alg. 4 prints it, the first step from zero
  moments is the closed form A - alpha G / sqrt(G^2 + eps).
- The projection max(A, lower) holds after every step.
- GCP-Adam on a planted, well-conditioned Gaussian problem recovers the
  planted factors: cosine score >= 0.9 (App. E).
"""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle.driver import gcp_adam
from oracle.score import cosine_score
from paper_1906_01687_gb300 import synth


def test_matches_torch_adam_with_eps_outside_root():
    rng = np.random.default_rng(0)
    n = 37
    A = rng.standard_normal(n)
    B, C = np.zeros(n), np.zeros(n)
    p = torch.tensor(A.copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([p], lr=0.01, betas=(0.9, 0.999), eps=1e-8)
    for t in range(6):
        G = rng.standard_normal(n) * (t + 1)
        oracle.adam_step(A, B, C, G, 0.01, 0.9, 0.999, 1e-8, -math.inf, t, eps_inside_sqrt=False)
        opt.zero_grad()
        p.grad = torch.tensor(G)
        opt.step()
        np.testing.assert_allclose(A, p.detach().numpy(), rtol=1e-13, atol=1e-15)


def test_first_step_closed_form_eps_inside_root():
    rng = np.random.default_rng(1)
    n = 50
    A0 = rng.standard_normal(n)
    G = rng.standard_normal(n) * 1e-3
    G[0] = 0.0
    A, B, C = A0.copy(), np.zeros(n), np.zeros(n)
    oracle.adam_step(A, B, C, G, 0.01, 0.9, 0.999, 1e-8, -math.inf, 0)
    np.testing.assert_allclose(B, 0.1 * G, rtol=1e-14)
    np.testing.assert_allclose(C, 0.001 * G * G, rtol=1e-14)
    np.testing.assert_allclose(A, A0 - 0.01 * G / np.sqrt(G * G + 1e-8), rtol=1e-13, atol=1e-16)


def test_second_step_bias_correction():
    G1, G2 = np.array([0.5, -2.0]), np.array([1.5, 0.25])
    A, B, C = np.zeros(2), np.zeros(2), np.zeros(2)
    oracle.adam_step(A, B, C, G1, 0.1, 0.9, 0.999, 1e-8, -math.inf, 0)
    a1 = A.copy()
    oracle.adam_step(A, B, C, G2, 0.1, 0.9, 0.999, 1e-8, -math.inf, 1)
    b = 0.9 * 0.1 * G1 + 0.1 * G2
    c = 0.999 * 0.001 * G1 ** 2 + 0.001 * G2 ** 2
    bh, ch = b / (1 - 0.81), c / (1 - 0.999 ** 2)
    np.testing.assert_allclose(A, a1 - 0.1 * bh / np.sqrt(ch + 1e-8), rtol=1e-13)


def test_projection():
    A = np.array([0.001, 0.5, -0.2])
    B, C = np.zeros(3), np.zeros(3)
    oracle.adam_step(A, B, C, np.array([1.0, 1.0, 1.0]), 0.01, 0.9, 0.999, 1e-8, 0.0, 0)
    assert np.all(A >= 0.0)
    assert A[0] == 0.0 and A[2] == 0.0 and A[1] == pytest.approx(0.5 - 0.01, rel=1e-6)
    # a nonzero bound: entries below it land on it, not on zero
    A = np.array([0.3, 0.5, -0.2])
    B, C = np.zeros(3), np.zeros(3)
    oracle.adam_step(A, B, C, np.array([1.0, -1.0, 1.0]), 0.01, 0.9, 0.999, 1e-8, 0.295, 0)
    assert A[0] == 0.295 and A[2] == 0.295 and A[1] == pytest.approx(0.5 + 0.01, rel=1e-6)


def test_planted_recovery_gaussian():
    """A planted rank-3 model with noise at 10% of the model norm is recovered
    (App. E score >= 0.9) by GCP-Adam with uniform sampling."""
    dims, rank = (20, 30, 40), 3
    rng = np.random.default_rng(5)
    true = [rng.standard_normal((n, rank)) for n in dims]
    true = [a / np.linalg.norm(a, axis=0, keepdims=True) for a in true]
    lam = np.array([30.0, 25.0, 20.0])
    M = synth.dense_from_factors(true, lam)
    X = M + 0.1 * np.linalg.norm(M) / math.sqrt(M.size) * rng.standard_normal(M.shape)
    T = oracle.Tensor(dims, dense=X)
    A0 = synth.initial_guess(dims, rank, 6, target_norm=np.linalg.norm(X), dtype=np.float64)
    est, hist = gcp_adam(T, A0, oracle.GAUSSIAN, oracle.UNIFORM, 0, 1000, 0, 500, seed=7, est_seed=8,
                         alpha=0.01, tau=100, max_epochs=40)
    assert hist[-1] < hist[0]
    assert cosine_score(true, est) >= 0.9
