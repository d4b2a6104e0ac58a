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


# ---------------------------------------------------------------------------
# the paper's own odds / identity-link losses (Section 1, Sections 5.2-5.4)
# ---------------------------------------------------------------------------
POSITIVE_LOSSES = [oracle.BERNOULLI_ODDS, oracle.POISSON_IDENTITY, oracle.GAMMA, oracle.BETA_HALF]


@pytest.mark.parametrize("m", [0.05, 0.7, 1.0, 3.0])
@pytest.mark.parametrize("x", [0.0, 1.0])
def test_bernoulli_odds_is_negative_log_likelihood(x, m):
    # m is the odds of a one: P(x = 1) = m / (1 + m)
    nll = -stats.bernoulli.logpmf(int(x), m / (1.0 + m))
    assert oracle.loss_f(oracle.BERNOULLI_ODDS, x, m) == pytest.approx(nll, rel=1e-8)


@pytest.mark.parametrize("m", [0.3, 1.0, 4.5])
@pytest.mark.parametrize("x", [0, 1, 5])
def test_poisson_identity_is_negative_log_likelihood(x, m):
    nll = -stats.poisson.logpmf(x, m) - special.gammaln(x + 1)
    assert oracle.loss_f(oracle.POISSON_IDENTITY, float(x), m) == pytest.approx(nll, rel=1e-8, abs=1e-9)


@pytest.mark.parametrize("m", [0.3, 1.0, 4.5])
@pytest.mark.parametrize("x", [0.2, 1.0, 7.0])
def test_gamma_is_exponential_negative_log_likelihood(x, m):
    # gamma with shape k = 1 (App. C) and mean m is the exponential distribution
    nll = -stats.expon.logpdf(x, scale=m)
    assert oracle.loss_f(oracle.GAMMA, x, m) == pytest.approx(nll, rel=1e-8)


def test_beta_half_closed_form():
    for x, m in [(0.0, 4.0), (1.0, 1.0), (9.0, 0.25)]:
        assert oracle.loss_f(oracle.BETA_HALF, x, m) == pytest.approx(2 * math.sqrt(m) + 2 * x / math.sqrt(m), rel=1e-8)
    # minimised at m = x
    fs = [oracle.loss_f(oracle.BETA_HALF, 2.0, m) for m in (1.5, 2.0, 2.5)]
    assert fs[1] < fs[0] and fs[1] < fs[2]


@pytest.mark.parametrize("loss", POSITIVE_LOSSES)
@pytest.mark.parametrize("x", [0.0, 1.0, 2.5])
@pytest.mark.parametrize("m", [0.2, 0.9, 3.0])
def test_positive_loss_g_is_derivative(loss, x, m):
    h = 1e-6
    fd = (oracle.loss_f(loss, x, m + h) - oracle.loss_f(loss, x, m - h)) / (2 * h)
    assert oracle.loss_g(loss, x, m) == pytest.approx(fd, rel=1e-6, abs=1e-8)


@pytest.mark.parametrize("loss", POSITIVE_LOSSES)
def test_positive_losses_finite_at_zero_model(loss):
    assert math.isfinite(oracle.loss_f(loss, 1.0, 0.0)) and math.isfinite(oracle.loss_g(loss, 1.0, 0.0))
