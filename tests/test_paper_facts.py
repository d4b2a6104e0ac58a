"""Numbers printed in the paper (tests/golden/paper_facts.json), checked
against the oracle's defaults and the formulas they follow from."""
import inspect
import json
import math
import os

import pytest
from scipy import stats

import oracle
from oracle.driver import gcp_adam

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_facts.json")))


def test_oracle_adam_defaults():
    g = GOLDEN["adam_defaults"]
    sig = inspect.signature(gcp_adam).parameters
    for name in ("alpha", "beta1", "beta2", "eps", "tau", "nu", "kappa"):
        assert sig[name].default == g[name], name


def test_oracle_oversample_default():
    assert inspect.signature(oracle.sample).parameters["rho"].default == GOLDEN["oversample_default"]["rho"]


def rho_needed(s_zero, p_zero, quantile):
    """App. B: rho >= (s_zero + s_reject) p_zero / s_zero with s_reject the
    negative-binomial quantile of rejections before s_zero successes."""
    s_reject = stats.nbinom.ppf(quantile, s_zero, p_zero)
    return (s_zero + s_reject) * p_zero / s_zero


def test_app_b_default_rate_is_adequate():
    g = GOLDEN["oversample_default"]
    for s_zero in (1000, 10000, 100000):
        for p_zero in (0.99, 0.995, 0.999):
            assert rho_needed(s_zero, p_zero, g["quantile"]) <= g["rho"]
    # the two trends App. B states
    assert rho_needed(100, 0.9, g["quantile"]) > rho_needed(1000, 0.9, g["quantile"])
    assert rho_needed(1000, 0.7, g["quantile"]) > rho_needed(1000, 0.9, g["quantile"])


def test_sample_split():
    for s, p, q in GOLDEN["sample_split"]["cases"]:
        assert (s // 2, -(-s // 2)) == (p, q)


def test_gamma_problem_counts():
    g = GOLDEN["gamma_problem"]
    assert sum(g["dims"]) * g["rank"] == g["free_parameters"]
    assert math.prod(g["dims"]) // g["tau"] == g["one_pass_s"]


def test_storage_examples():
    g = GOLDEN["storage_binary_400"]
    d = len(g["dims"])
    assert (d + 1) * g["nnz"] * 8 / 1e9 == pytest.approx(g["sparse_gb"], abs=0.005)
    assert math.prod(g["dims"]) * 8 / 1e9 == pytest.approx(g["dense_gb"], rel=0.02)
    h = GOLDEN["dense_y_storage"]
    assert h["n"] ** h["d"] * 8 / 1e12 == h["tb"]
