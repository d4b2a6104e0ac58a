"""Pins of the oracle's sampled gradient (Eqs. (4.1)-(4.3), Algs. 1-3).

- Closed form: the full Gaussian gradient is 2 (M - X)_(k) Z_k, the textbook
  MTTKRP, computed here with numpy.einsum.
- Enumeration identity: one draw of every index of Omega with weight 1 gives
  exactly the full gradient G_k = Y_(k) Z_k, for each sampler's classes.
- Finite differences: the sampled gradient is the derivative of the
  fixed-sample loss estimate on the same draws.
- Unbiasedness: the mean of many sampled gradients approaches the full
  gradient within a CLT bound (E[Y~] = Y, Sections 4.1-4.3).
"""
import itertools

import numpy as np
import pytest
from scipy import special

import oracle
from oracle import Samples

LOSSES = [oracle.GAUSSIAN, oracle.BERNOULLI_LOGIT, oracle.POISSON_LOG]
LETTERS = "ijklmnop"


def einsum_model(factors):
    d = len(factors)
    spec = ",".join(f"{LETTERS[k]}z" for k in range(d)) + "->" + LETTERS[:d]
    return np.einsum(spec, *factors)


def einsum_mttkrp(Y, factors, k):
    """Y_(k) Z_k written as an einsum over all modes but k."""
    d = len(factors)
    ops = [Y] + [factors[l] for l in range(d) if l != k]
    spec = LETTERS[:d] + "," + ",".join(f"{LETTERS[l]}z" for l in range(d) if l != k)
    return np.einsum(spec + f"->{LETTERS[k]}z", *ops)


def numpy_g(loss, X, M):
    if loss == oracle.GAUSSIAN:
        return 2.0 * (M - X)
    if loss == oracle.BERNOULLI_LOGIT:
        return special.expit(M) - X
    return np.exp(M) - X


def numpy_f(loss, X, M):
    if loss == oracle.GAUSSIAN:
        return (X - M) ** 2
    if loss == oracle.BERNOULLI_LOGIT:
        return np.logaddexp(0.0, M) - X * M
    return np.exp(M) - X * M


def problem(dims, rank, loss, seed, density=None):
    rng = np.random.default_rng(seed)
    A = [0.7 * rng.standard_normal((n, rank)) for n in dims]
    M = einsum_model(A)
    if loss == oracle.GAUSSIAN:
        X = M + 0.3 * rng.standard_normal(M.shape)
    elif loss == oracle.BERNOULLI_LOGIT:
        X = (rng.random(M.shape) < 0.3).astype(float)
    else:
        X = rng.poisson(1.5, M.shape).astype(float)
    if density is not None:
        X = X * (rng.random(M.shape) < density)
    return X, A


def all_indices(dims):
    return np.array(list(itertools.product(*[range(n) for n in dims])), dtype=np.int64)


def test_gaussian_full_gradient_is_textbook_mttkrp():
    dims, rank = (3, 4, 5), 3
    X, A = problem(dims, rank, oracle.GAUSSIAN, 1)
    G, F = oracle.full_grad(dims, A, oracle.GAUSSIAN, X)
    M = einsum_model(A)
    for k in range(3):
        np.testing.assert_allclose(G[k], einsum_mttkrp(2.0 * (M - X), A, k), rtol=1e-12, atol=1e-12)
    assert F == pytest.approx(np.sum((X - M) ** 2), rel=1e-12)


@pytest.mark.parametrize("loss", LOSSES)
@pytest.mark.parametrize("dims", [(4, 5), (3, 4, 5), (1, 4, 3), (2, 3, 2, 3), (2, 2, 3, 2, 2), (2, 3, 2, 2, 1, 2, 2, 3)])
def test_full_gradient_matches_einsum(loss, dims):
    X, A = problem(dims, 2, loss, 2)
    G, F = oracle.full_grad(dims, A, loss, X)
    M = einsum_model(A)
    Y = numpy_g(loss, X, M)
    for k in range(len(dims)):
        np.testing.assert_allclose(G[k], einsum_mttkrp(Y, A, k), rtol=1e-11, atol=1e-11)
    assert F == pytest.approx(numpy_f(loss, X, M).sum(), rel=1e-12)


def test_weighted_full_gradient():
    """Weighted GCP (Eq. (4.5)): y_i = v_i g(x_i, m_i); zero weight removes an entry."""
    dims = (3, 4, 5)
    X, A = problem(dims, 2, oracle.BERNOULLI_LOGIT, 3)
    v = np.random.default_rng(0).random(dims) * (np.random.default_rng(1).random(dims) < 0.7)
    G, F = oracle.full_grad(dims, A, oracle.BERNOULLI_LOGIT, X, weights=v)
    M = einsum_model(A)
    Y = v * numpy_g(oracle.BERNOULLI_LOGIT, X, M)
    for k in range(3):
        np.testing.assert_allclose(G[k], einsum_mttkrp(Y, A, k), rtol=1e-11, atol=1e-12)
    assert F == pytest.approx((v * numpy_f(oracle.BERNOULLI_LOGIT, X, M)).sum(), rel=1e-12)


@pytest.mark.parametrize("loss", LOSSES)
def test_enumeration_identity_uniform(loss):
    dims = (3, 4, 5)
    X, A = problem(dims, 3, loss, 4)
    idx = all_indices(dims)
    S = Samples(idx, X.reshape(-1), np.ones(len(idx)), np.full(len(idx), oracle.CLS_UNIFORM))
    Gs = oracle.grad(dims, A, loss, S)
    G, F = oracle.full_grad(dims, A, loss, X)
    for k in range(3):
        np.testing.assert_allclose(Gs[k], G[k], rtol=1e-12, atol=1e-12)
    assert oracle.loss_estimate(dims, A, loss, S) == pytest.approx(F, rel=1e-12)


@pytest.mark.parametrize("loss", LOSSES)
def test_enumeration_identity_stratified(loss):
    """All nonzeros (weight 1, class nonzero) plus all zeros (weight 1, class
    zero) give the full gradient: the two strata partition Omega."""
    dims = (3, 4, 5)
    X, A = problem(dims, 2, loss, 5, density=0.3)
    idx = all_indices(dims)
    x = X.reshape(-1)
    nz = x != 0
    cls = np.where(nz, oracle.CLS_STRAT_NZ, oracle.CLS_STRAT_ZERO)
    S = Samples(idx, x, np.ones(len(idx)), cls)
    Gs = oracle.grad(dims, A, loss, S)
    G, F = oracle.full_grad(dims, A, loss, X)
    for k in range(3):
        np.testing.assert_allclose(Gs[k], G[k], rtol=1e-12, atol=1e-12)
    assert oracle.loss_estimate(dims, A, loss, S) == pytest.approx(F, rel=1e-12)


@pytest.mark.parametrize("loss", LOSSES)
def test_enumeration_identity_semi_stratified(loss):
    """All nonzeros with the correction g(x,m) - g(0,m) plus every index of
    Omega as a "zero" with g(0,m) give the full gradient (Section 4.3)."""
    dims = (3, 4, 5)
    X, A = problem(dims, 2, loss, 6, density=0.3)
    idx = all_indices(dims)
    x = X.reshape(-1)
    nz = np.nonzero(x)[0]
    S = Samples(np.concatenate([idx[nz], idx]), np.concatenate([x[nz], np.zeros(len(idx))]),
                np.ones(len(nz) + len(idx)),
                np.concatenate([np.full(len(nz), oracle.CLS_SEMI_NZ), np.full(len(idx), oracle.CLS_SEMI_ZERO)]))
    Gs = oracle.grad(dims, A, loss, S)
    G, F = oracle.full_grad(dims, A, loss, X)
    for k in range(3):
        np.testing.assert_allclose(Gs[k], G[k], rtol=1e-11, atol=1e-11)
    assert oracle.loss_estimate(dims, A, loss, S) == pytest.approx(F, rel=1e-11)


def random_sample_list(dims, X, n, seed):
    rng = np.random.default_rng(seed)
    idx = np.stack([rng.integers(0, nk, n) for nk in dims], axis=1)
    cls = rng.integers(0, 5, n).astype(np.int8)
    x = X[tuple(idx.T)]
    x = np.where((cls == oracle.CLS_STRAT_ZERO) | (cls == oracle.CLS_SEMI_ZERO), 0.0, x)
    w = rng.uniform(0.5, 3.0, n)
    return Samples(idx, x, w, cls)


@pytest.mark.parametrize("loss", LOSSES)
@pytest.mark.parametrize("dims", [(3, 4, 2, 3), (2, 3, 2, 2, 2, 3, 2, 2)], ids=["d4", "d8"])
def test_gradient_is_derivative_of_estimate(loss, dims):
    X, A = problem(dims, 3, loss, 7)
    S = random_sample_list(dims, X, 40, 8)
    G = oracle.grad(dims, A, loss, S)
    h = 1e-6
    for k in range(len(dims)):
        for i in range(dims[k]):
            for j in range(3):
                Ap = [a.copy() for a in A]
                Am = [a.copy() for a in A]
                Ap[k][i, j] += h
                Am[k][i, j] -= h
                fd = (oracle.loss_estimate(dims, Ap, loss, S) - oracle.loss_estimate(dims, Am, loss, S)) / (2 * h)
                assert G[k][i, j] == pytest.approx(fd, rel=2e-6, abs=2e-7)


def mc_check(dims, A, loss, X, kind, p, q, N, seed_base, X_obj):
    G_full, _ = oracle.full_grad(dims, A, loss, X)
    samples = []
    for t in range(N):
        S = oracle.sample(X_obj, kind, p, q, seed_base, t)
        samples.append(np.concatenate([g.reshape(-1) for g in oracle.grad(dims, A, loss, S)]))
    samples = np.array(samples)
    mean = samples.mean(axis=0)
    se = samples.std(axis=0, ddof=1) / np.sqrt(N)
    full = np.concatenate([g.reshape(-1) for g in G_full])
    assert np.all(np.abs(mean - full) <= 5 * se + 1e-12), np.max(np.abs(mean - full) / (se + 1e-300))
    # a biased estimator (e.g. a dropped weight) would be off by far more than 5 SE somewhere
    return samples


def coo_of(X):
    nzi = np.argwhere(X != 0)
    return nzi, X[tuple(nzi.T)]


@pytest.mark.parametrize("loss", [oracle.GAUSSIAN, oracle.BERNOULLI_LOGIT])
def test_uniform_sampler_unbiased(loss):
    dims = (3, 4, 5)
    X, A = problem(dims, 2, loss, 9)
    mc_check(dims, A, loss, X, oracle.UNIFORM, 0, 30, 3000, 11, oracle.Tensor(dims, dense=X))


@pytest.mark.parametrize("kind", [oracle.STRATIFIED, oracle.SEMI_STRATIFIED])
@pytest.mark.parametrize("loss", [oracle.BERNOULLI_LOGIT, oracle.POISSON_LOG])
def test_stratified_samplers_unbiased(kind, loss):
    dims = (3, 4, 5)
    X, A = problem(dims, 2, loss, 10, density=0.25)
    coo, vals = coo_of(X)
    T = oracle.Tensor(dims, coo=coo, vals=vals)
    mc_check(dims, A, loss, X, kind, 10, 10, 3000, 12, T)


def test_stratified_variance_below_uniform():
    """On a very sparse binary tensor, near a model whose zeros have small
    derivatives, the stratified and semi-stratified gradients have lower
    empirical variance than uniform sampling at equal s (the ordering of
    Table 1, not its values)."""
    dims = (10, 8, 6)
    rng = np.random.default_rng(3)
    A = [1.44 * (1.0 + 0.1 * rng.standard_normal((n, 2))) for n in dims]
    A[0] = -A[0]  # m near -3: sigmoid(m) ~ 0.05 at the zeros
    X = (rng.random(dims) < 0.02).astype(float)
    loss = oracle.BERNOULLI_LOGIT
    coo, vals = coo_of(X)
    Td = oracle.Tensor(dims, dense=X)
    Ts = oracle.Tensor(dims, coo=coo, vals=vals)
    N = 600

    def var(kind, T, p, q):
        gs = []
        for t in range(N):
            S = oracle.sample(T, kind, p, q, 21, t)
            gs.append(np.concatenate([g.reshape(-1) for g in oracle.grad(dims, A, loss, S)]))
        gs = np.array(gs)
        return np.mean(np.sum((gs - gs.mean(axis=0)) ** 2, axis=1))

    v_uni = var(oracle.UNIFORM, Td, 0, 40)
    v_strat = var(oracle.STRATIFIED, Ts, 20, 20)
    v_semi = var(oracle.SEMI_STRATIFIED, Ts, 20, 20)
    assert v_strat < v_uni and v_semi < v_uni, (v_uni, v_strat, v_semi)


def test_abs_scales_bound_the_sums():
    """grad_abs and loss_abs (tolerance scales) dominate |G| and |F-hat| and
    equal them when every term is nonnegative."""
    dims = (3, 4, 5)
    X, A = problem(dims, 2, oracle.GAUSSIAN, 40)
    S = random_sample_list(dims, X, 60, 41)
    G = oracle.grad(dims, A, oracle.GAUSSIAN, S)
    Gabs = oracle.grad_abs(dims, A, oracle.GAUSSIAN, S)
    for g, ga in zip(G, Gabs):
        assert np.all(np.abs(g) <= ga + 1e-12)
    assert oracle.loss_abs(dims, A, oracle.GAUSSIAN, S) >= abs(oracle.loss_estimate(dims, A, oracle.GAUSSIAN, S))
    Splain = Samples(S.idx, S.x, S.w, np.full(S.n, oracle.CLS_UNIFORM))
    assert oracle.loss_abs(dims, A, oracle.GAUSSIAN, Splain) == pytest.approx(
        oracle.loss_estimate(dims, A, oracle.GAUSSIAN, Splain), rel=1e-12)  # Gaussian terms are >= 0
    Apos = [np.abs(a) for a in A]
    Spos = Samples(S.idx, S.x, S.w, np.full(S.n, oracle.CLS_UNIFORM))
    Xbig = X + 100.0
    Spos.x = Xbig[tuple(S.idx.T)]
    G = oracle.grad(dims, Apos, oracle.GAUSSIAN, Spos)  # m < x everywhere: every term is negative
    Gabs = oracle.grad_abs(dims, Apos, oracle.GAUSSIAN, Spos)
    for g, ga in zip(G, Gabs):
        np.testing.assert_allclose(-g, ga, rtol=1e-12)
    # Poisson-log terms e^m - x m change sign: the scale is the sum of the
    # single-entry magnitudes, strictly above |F-hat|
    Xp = np.random.default_rng(42).poisson(3.0, dims).astype(float)
    Sp = Samples(S.idx, Xp[tuple(S.idx.T)], S.w, np.full(S.n, oracle.CLS_UNIFORM))
    terms = [oracle.loss_estimate(dims, A, oracle.POISSON_LOG,
                                  Samples(Sp.idx[e:e + 1], Sp.x[e:e + 1], Sp.w[e:e + 1], Sp.cls[e:e + 1]))
             for e in range(Sp.n)]
    assert min(terms) < 0 < max(terms)
    assert oracle.loss_abs(dims, A, oracle.POISSON_LOG, Sp) == pytest.approx(np.abs(terms).sum(), rel=1e-12)


def numpy_g_positive(loss, X, M):
    Mp = M + oracle.M_EPS
    if loss == oracle.BERNOULLI_ODDS:
        return 1.0 / (Mp + 1.0) - X / Mp
    if loss == oracle.POISSON_IDENTITY:
        return 1.0 - X / Mp
    if loss == oracle.GAMMA:
        return -X / Mp ** 2 + 1.0 / Mp
    return Mp ** -0.5 - X * Mp ** -1.5


@pytest.mark.parametrize("loss", [oracle.BERNOULLI_ODDS, oracle.POISSON_IDENTITY, oracle.GAMMA, oracle.BETA_HALF])
def test_positive_losses_full_gradient_and_derivative(loss):
    """Odds/identity-link losses on a nonnegative model: the full gradient is
    the einsum MTTKRP of Y, and the sampled gradient is dF-hat/dA."""
    dims = (3, 4, 5)
    rng = np.random.default_rng(50 + loss)
    A = [rng.uniform(0.2, 1.0, (n, 2)) for n in dims]
    M = einsum_model(A)
    X = rng.poisson(1.0, dims).astype(float) if loss != oracle.GAMMA else rng.exponential(M)
    if loss == oracle.BERNOULLI_ODDS:
        X = (X > 0).astype(float)
    G, _ = oracle.full_grad(dims, A, loss, X)
    Y = numpy_g_positive(loss, X, M)
    for k in range(3):
        np.testing.assert_allclose(G[k], einsum_mttkrp(Y, A, k), rtol=1e-11, atol=1e-11)
    S = random_sample_list(dims, X, 30, 60)
    Gs = oracle.grad(dims, A, loss, S)
    h = 1e-6
    for k in range(3):
        for i in range(dims[k]):
            for j in range(2):
                Ap = [a.copy() for a in A]
                Am = [a.copy() for a in A]
                Ap[k][i, j] += h
                Am[k][i, j] -= h
                fd = (oracle.loss_estimate(dims, Ap, loss, S) - oracle.loss_estimate(dims, Am, loss, S)) / (2 * h)
                assert Gs[k][i, j] == pytest.approx(fd, rel=2e-5, abs=2e-6)


def test_weighted_uniform_sampling_unbiased():
    """With entry weights v the uniform sampler's gradient is unbiased for the
    weighted full gradient of Eq. (4.5)."""
    dims = (3, 4, 5)
    X, A = problem(dims, 2, oracle.BERNOULLI_LOGIT, 70)
    v = np.random.default_rng(71).random(dims) * (np.random.default_rng(72).random(dims) < 0.7)
    G_full, _ = oracle.full_grad(dims, A, oracle.BERNOULLI_LOGIT, X, weights=v)
    T = oracle.Tensor(dims, dense=X, weights=v)
    N = 3000
    gs = np.array([np.concatenate([g.reshape(-1) for g in
                                   oracle.grad(dims, A, oracle.BERNOULLI_LOGIT, oracle.sample(T, oracle.UNIFORM, 0, 30, 5, t))])
                   for t in range(N)])
    full = np.concatenate([g.reshape(-1) for g in G_full])
    se = gs.std(axis=0, ddof=1) / np.sqrt(N)
    assert np.all(np.abs(gs.mean(axis=0) - full) <= 5 * se + 1e-12)


def test_uniform_over_sparse_enumeration_identity():
    """Every index once (weight 1) through the sparse value lookup gives the
    full gradient of the dense equivalent."""
    dims = (3, 4, 5)
    X, A = problem(dims, 2, oracle.POISSON_LOG, 73, density=0.3)
    coo, vals = coo_of(X)
    T = oracle.Tensor(dims, coo=coo, vals=vals)
    keys, svals = T.sorted_pairs()
    lib = oracle._load()
    idx = all_indices(dims)
    x = np.array([lib.orc_sparse_value(T.nnz, oracle._p(keys), oracle._p(svals), oracle.linear_key(dims, ix))
                  for ix in idx])
    np.testing.assert_array_equal(x, X.reshape(-1))
    S = Samples(idx, x, np.ones(len(idx)), np.full(len(idx), oracle.CLS_UNIFORM))
    Gs = oracle.grad(dims, A, oracle.POISSON_LOG, S)
    G, _ = oracle.full_grad(dims, A, oracle.POISSON_LOG, X)
    for k in range(3):
        np.testing.assert_allclose(Gs[k], G[k], rtol=1e-12, atol=1e-12)


def test_observed_sampling_unbiased():
    """Drawing only the entries of nonzero weight (Section 4.4, missing data
    as weight 0) keeps the gradient unbiased for the weighted full gradient,
    with 40% of the entries missing."""
    dims = (3, 4, 5)
    X, A = problem(dims, 2, oracle.POISSON_LOG, 73)
    rng = np.random.default_rng(74)
    v = (0.5 + rng.random(dims)) * (rng.random(dims) >= 0.4)
    G_full, _ = oracle.full_grad(dims, A, oracle.POISSON_LOG, X, weights=v)
    T = oracle.Tensor(dims, dense=X, weights=v)
    N = 3000
    gs = np.array([np.concatenate([g.reshape(-1) for g in
                                   oracle.grad(dims, A, oracle.POISSON_LOG, oracle.sample(T, oracle.OBSERVED, 0, 30, 5, t))])
                   for t in range(N)])
    full = np.concatenate([g.reshape(-1) for g in G_full])
    se = gs.std(axis=0, ddof=1) / np.sqrt(N)
    assert np.all(np.abs(gs.mean(axis=0) - full) <= 5 * se + 1e-12)
