"""Pins of the oracle's elementwise losses f(x, m) and derivatives g = df/dm.

Gaussian: f = (x - m)^2 (Section 1).  Bernoulli-logit and Poisson-log are the
log-link forms of the GCP paper this one builds on: the negative
log-likelihoods of Bernoulli(sigmoid(m)) and Poisson(e^m) up to terms free of
m.  They are checked here against scipy's distributions and special
functions, and g against central differences of f.
"""
import math

import numpy as np
import pytest
from scipy import special, stats

import oracle

LOSSES = [oracle.GAUSSIAN, oracle.BERNOULLI_LOGIT, oracle.POISSON_LOG]


def test_gaussian_values():
    assert oracle.loss_f(oracle.GAUSSIAN, 1.0, 3.0) == 4.0
    assert oracle.loss_g(oracle.GAUSSIAN, 1.0, 3.0) == 4.0
    assert oracle.loss_g(oracle.GAUSSIAN, 3.0, 1.0) == -4.0


@pytest.mark.parametrize("m", [-40.0, -5.0, -0.3, 0.0, 0.7, 3.0, 40.0])
@pytest.mark.parametrize("x", [0.0, 1.0])
def test_bernoulli_logit_is_negative_log_likelihood(x, m):
    # -log P(x | p = sigmoid(m)) from scipy's Bernoulli distribution
    nll = -stats.bernoulli.logpmf(int(x), special.expit(m)) if abs(m) < 30 else None
    f = oracle.loss_f(oracle.BERNOULLI_LOGIT, x, m)
    if nll is not None:
        assert f == pytest.approx(nll, rel=1e-12, abs=1e-14)
    # log(1 + e^m) - x m via logaddexp, valid at every m
    assert f == pytest.approx(np.logaddexp(0.0, m) - x * m, rel=1e-13, abs=1e-15)
    assert oracle.loss_g(oracle.BERNOULLI_LOGIT, x, m) == pytest.approx(special.expit(m) - x, rel=1e-13, abs=1e-300)


@pytest.mark.parametrize("m", [-3.0, -0.5, 0.0, 1.2, 4.0])
@pytest.mark.parametrize("x", [0, 1, 2, 7])
def test_poisson_log_is_negative_log_likelihood(x, m):
    # f differs from -log P(x | lambda = e^m) by log(x!), which is free of m
    nll = -stats.poisson.logpmf(x, math.exp(m)) - special.gammaln(x + 1)
    assert oracle.loss_f(oracle.POISSON_LOG, float(x), m) == pytest.approx(nll, rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("loss", LOSSES)
@pytest.mark.parametrize("x", [0.0, 1.0, 2.5])
@pytest.mark.parametrize("m", [-2.0, -0.1, 0.0, 0.4, 1.7])
def test_g_is_derivative_of_f(loss, x, m):
    h = 1e-5
    fd = (oracle.loss_f(loss, x, m + h) - oracle.loss_f(loss, x, m - h)) / (2 * h)
    assert oracle.loss_g(loss, x, m) == pytest.approx(fd, rel=1e-8, abs=1e-9)


def test_special_points():
    assert oracle.loss_f(oracle.BERNOULLI_LOGIT, 0.0, 0.0) == pytest.approx(math.log(2.0))
    assert oracle.loss_g(oracle.BERNOULLI_LOGIT, 1.0, 0.0) == pytest.approx(-0.5)
    assert oracle.loss_f(oracle.POISSON_LOG, 5.0, 0.0) == pytest.approx(1.0)
    assert oracle.loss_g(oracle.POISSON_LOG, 5.0, 0.0) == pytest.approx(-4.0)
    # Bernoulli-logit stays finite far from 0
    assert math.isfinite(oracle.loss_f(oracle.BERNOULLI_LOGIT, 1.0, -800.0))
    assert oracle.loss_f(oracle.BERNOULLI_LOGIT, 1.0, 800.0) == pytest.approx(0.0, abs=1e-300)


@pytest.mark.parametrize("loss", LOSSES)
def test_entry_forms(loss):
    """Class-dependent y and F terms of Algs. 1-3: only the semi-stratified
    nonzero subtracts the x = 0 term."""
    x, m, w = 2.0, 0.3, 7.5
    g, g0 = oracle.loss_g(loss, x, m), oracle.loss_g(loss, 0.0, m)
    f, f0 = oracle.loss_f(loss, x, m), oracle.loss_f(loss, 0.0, m)
    for cls in (oracle.CLS_UNIFORM, oracle.CLS_STRAT_NZ, oracle.CLS_STRAT_ZERO, oracle.CLS_SEMI_ZERO):
        assert oracle.entry_y(loss, cls, x, m, w) == pytest.approx(w * g)
        assert oracle.entry_f(loss, cls, x, m, w) == pytest.approx(w * f)
    assert oracle.entry_y(loss, oracle.CLS_SEMI_NZ, x, m, w) == pytest.approx(w * (g - g0))
    assert oracle.entry_f(loss, oracle.CLS_SEMI_NZ, x, m, w) == pytest.approx(w * (f - f0))
