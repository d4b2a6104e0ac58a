"""Pins of App. E's cosine score (oracle/score.py) by cases whose value is
known exactly: the same model written differently scores 1, a component
orthogonal in one mode contributes 0, and the assignment solver used for
more than 8 components agrees with the exhaustive search."""
import itertools

import numpy as np
import pytest

from oracle.score import _cos_matrix, cosine_score


def factors(dims, r, seed):
    rng = np.random.default_rng(seed)
    return [rng.standard_normal((n, r)) for n in dims]


def test_same_model_written_differently_scores_one():
    true = factors((6, 7, 8), 4, 1)
    perm = [2, 0, 3, 1]
    scale = np.array([2.0, 0.5, 3.0, 1.5])
    signs = [np.array([1, -1, 1, -1]), np.array([1, -1, -1, 1]), np.array([1, 1, -1, -1])]  # even flips per column
    est = [a[:, perm] * s[perm] * (scale[perm] if k == 0 else 1.0) for k, (a, s) in enumerate(zip(true, signs))]
    assert cosine_score(true, est) == pytest.approx(1.0, abs=1e-12)


def test_component_orthogonal_in_one_mode_scores_zero():
    true = [np.eye(4)[:, :2], np.eye(5)[:, :2], np.eye(3)[:, :2]]
    est = [t.copy() for t in true]
    est[1][:, 1] = np.eye(5)[:, 4]  # component 2 orthogonal to both true components in mode 2
    assert cosine_score(true, est) == pytest.approx(0.5, abs=1e-12)


def test_partial_match_is_the_mean_of_cosine_products():
    true = [np.eye(3)[:, :2], np.eye(3)[:, :2]]
    c = np.cos(0.3)
    est = [np.array([[c, 0], [np.sin(0.3), 0], [0, 1]]), np.eye(3)[:, [0, 2]]]
    # component 1: cos 0.3 in mode 1 and 1 in mode 2; component 2 matches nothing of true component 2
    assert cosine_score(true, est) == pytest.approx((c * 1.0 + 0.0) / 2, abs=1e-12)


def test_assignment_solver_matches_exhaustive_search():
    r = 9
    true, est = factors((10, 11, 12), r, 2), factors((10, 11, 12), r, 3)
    prod = np.ones((r, r))
    for a, b in zip(true, est):
        prod *= np.abs(_cos_matrix(a, b))
    best = max(sum(prod[j, pi[j]] for j in range(r)) for pi in itertools.permutations(range(r)))
    assert cosine_score(true, est) == pytest.approx(best / r, rel=1e-12)
