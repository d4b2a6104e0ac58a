"""Pins of the oracle's fixed-sample loss estimate (Eqs. (5.1)-(5.2)).

- The full enumeration with weight 1 gives the objective F of Eq. (1.2)
  (covered for every class in test_oracle_grad's enumeration identities).
- E[F-hat] = F: the mean over many independent sample sets approaches F
  within a CLT bound, for the uniform, stratified and semi-stratified forms.
"""
import numpy as np
import pytest

import oracle
from test_oracle_grad import coo_of, numpy_f, einsum_model, problem


@pytest.mark.parametrize("kind", [oracle.UNIFORM, oracle.STRATIFIED, oracle.SEMI_STRATIFIED])
@pytest.mark.parametrize("loss", [oracle.GAUSSIAN, oracle.BERNOULLI_LOGIT, oracle.POISSON_LOG])
def test_estimate_unbiased(kind, loss):
    dims = (4, 3, 5)
    X, A = problem(dims, 2, loss, 30, density=0.3)
    F = numpy_f(loss, X, einsum_model(A)).sum()
    if kind == oracle.UNIFORM:
        T, p, q = oracle.Tensor(dims, dense=X), 0, 20
    else:
        coo, vals = coo_of(X)
        T, p, q = oracle.Tensor(dims, coo=coo, vals=vals), 10, 10
    N = 4000
    est = np.array([oracle.loss_estimate(dims, A, loss, oracle.sample(T, kind, p, q, 31, t)) for t in range(N)])
    se = est.std(ddof=1) / np.sqrt(N)
    assert abs(est.mean() - F) <= 5 * se


def test_estimate_set_is_fixed():
    """The estimate's sample set depends only on (seed, stream): repeated
    draws with the same pair are identical (Section 5.1: the same set serves
    every epoch and every run)."""
    dims = (5, 6, 7)
    X = np.random.default_rng(0).standard_normal(dims)
    T = oracle.Tensor(dims, dense=X)
    S1 = oracle.sample(T, oracle.UNIFORM, 0, 100, 99, 2**64 - 1)
    S2 = oracle.sample(T, oracle.UNIFORM, 0, 100, 99, 2**64 - 1)
    assert np.array_equal(S1.idx, S2.idx) and np.array_equal(S1.x, S2.x)
