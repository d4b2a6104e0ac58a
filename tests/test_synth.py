"""Checks of the seeded input generators (they feed both the CUDA path and the oracle)."""
import pytest
import numpy as np

from paper_1906_01687_gb300 import synth


def test_batched_problem_shapes():
    """The batched workload's shapes respect their stated bounds (and the
    generator terminates for 4-way shapes)."""
    probs = synth.batched_problems()
    assert len(probs) == 64
    for p in probs:
        assert len(p["dims"]) in (3, 4)
        assert all(50 <= n <= 2000 for n in p["dims"])
        assert np.prod(np.array(p["dims"], dtype=np.float64)) <= 2e7
        assert p["rank"] in (4, 8, 16, 32, 64) and 10_000 <= p["s"] <= 100_000


def test_planted_dense_matches_its_factors():
    X, factors, w = synth.planted_dense((4, 5, 6), 2, seed=3, noise_std=0.0)
    M = np.einsum("ir,jr,kr->ijk", *factors)
    np.testing.assert_allclose(X, M, rtol=1e-12)


def test_initial_guess_hits_target_norm():
    A = synth.initial_guess((7, 8, 9), 3, seed=1, target_norm=5.0, dtype=np.float64)
    M = np.einsum("ir,jr,kr->ijk", *A)
    assert abs(np.linalg.norm(M) - 5.0) < 1e-9


def test_count_tensor_small():
    idx, vals, _ = synth.count_tensor(dims=(50, 6, 7, 8), nnz=2000, rank=3, seed=2)
    keys = ((idx[0].astype(np.int64) * 6 + idx[1]) * 7 + idx[2]) * 8 + idx[3]
    assert len(np.unique(keys)) == 2000 and (vals >= 1).all()
    # the skewed first mode: its first tenth holds more than a tenth of the nonzeros
    assert (idx[0] < 5).mean() > 0.1


def test_app_c_and_d_generators():
    X, f = synth.gamma_problem(dims=(10, 8, 6), rank=2, seed=4)
    assert (X >= 0).all() and X.shape == (10, 8, 6)
    X, f = synth.binary_odds_problem(dims=(20, 15, 10, 5), rank=4, seed=5)
    assert set(np.unique(X)) <= {0.0, 1.0} and 0 < X.mean() < 0.5


def test_binary_odds_coo_draws_app_d_model():
    """The device generator of App. D's sparse binary tensor: indices valid,
    unique and row-major sorted; the number of ones matches the model's
    expected count sum_i m_i / (1 + m_i) within 5 binomial sigma."""
    torch = pytest.importorskip("torch")
    dims = (40, 30, 20, 10)
    idx, factors = synth.binary_odds_coo(dims, rank=5, seed=4, device="cpu", slab=7)
    assert all(i.dtype == torch.int32 for i in idx)
    for i, n in zip(idx, dims):
        assert int(i.min()) >= 0 and int(i.max()) < n
    lin = idx[0].long()
    for i, n in zip(idx[1:], dims[1:]):
        lin = lin * n + i.long()
    assert bool((lin[1:] > lin[:-1]).all())
    M = synth.dense_from_factors(factors)
    p = M / (1.0 + M)
    mean, sd = p.sum(), np.sqrt((p * (1 - p)).sum())
    assert abs(idx[0].numel() - mean) < 5 * sd
