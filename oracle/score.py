"""Cosine similarity score between a true and an estimated CP model (App. E).

TEST INFRASTRUCTURE ONLY (see the package docstring).

score = (1/r) sum_j prod_k cos(a_k(:,j), ahat_k(:,pi(j))), maximised over the
permutation pi of the estimated components; the true solution counts as
recovered when the score is at least 0.9.  The sign of a column is free in a
CP model with an even number of sign flips, so each cosine enters with its
absolute value: flipping two columns' signs leaves the model unchanged.
"""
import itertools

import numpy as np


def _cos_matrix(a, b):
    an = a / np.linalg.norm(a, axis=0, keepdims=True)
    bn = b / np.linalg.norm(b, axis=0, keepdims=True)
    return an.T @ bn  # r x r, entry (j, l) = cos(a(:,j), b(:,l))


def cosine_score(true_factors, est_factors) -> float:
    r = true_factors[0].shape[1]
    prod = np.ones((r, r))
    for a, b in zip(true_factors, est_factors):
        prod *= np.abs(_cos_matrix(np.asarray(a, float), np.asarray(b, float)))
    if r <= 8:
        best = max(sum(prod[j, pi[j]] for j in range(r)) for pi in itertools.permutations(range(r)))
    else:
        from scipy.optimize import linear_sum_assignment
        rows, cols = linear_sum_assignment(-prod)
        best = prod[rows, cols].sum()
    return float(best / r)
