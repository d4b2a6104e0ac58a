"""Pins of the oracle's samplers (Algs. 1-3) against a pure-Python twin.

The twin builds every draw from numpy's Philox (an independent
implementation of the generator), Python integers for randi, and a Python
set for nonzero membership, following the sampling conventions: nonzero
draws first, then zeros; stratified zeros are the first q accepted
candidates in candidate order.
"""
import math

import numpy as np
import pytest

import oracle
from test_oracle_rng import numpy_philox_block


def twin_index(dims, seed, stream, tag, j, problem=0):
    return [(numpy_philox_block([j, stream, tag, k // 4], [seed, problem])[k % 4] * n) >> 64
            for k, n in enumerate(dims)]


def twin_key(dims, ix):
    key = 0
    for n, i in zip(dims, ix):
        key = key * n + i
    return key


def twin_sample(dims, dense, coo, vals, kind, p, q, seed, stream, rho=1.1, problem=0):
    omega = math.prod(dims)
    out = []  # (idx, x, w, cls)
    if kind == oracle.UNIFORM:
        for j in range(q):
            ix = twin_index(dims, seed, stream, oracle.TAG_UNIFORM, j, problem)
            out.append((ix, dense[tuple(ix)], omega / q, oracle.CLS_UNIFORM))
        return out
    eta = len(coo)
    for j in range(p):
        w0 = numpy_philox_block([j, stream, oracle.TAG_NONZERO, 0], [seed, problem])[0]
        xi = (w0 * eta) >> 64
        out.append((list(coo[xi]), 1.0 if vals is None else vals[xi], eta / p,
                    oracle.CLS_STRAT_NZ if kind == oracle.STRATIFIED else oracle.CLS_SEMI_NZ))
    if kind == oracle.SEMI_STRATIFIED:
        for j in range(q):
            ix = twin_index(dims, seed, stream, oracle.TAG_SEMI_ZERO, j, problem)
            out.append((ix, 0.0, omega / q, oracle.CLS_SEMI_ZERO))
        return out
    nzset = {twin_key(dims, c) for c in coo}
    zeta = omega - eta
    c = 0
    while len(out) < p + q:
        ix = twin_index(dims, seed, stream, oracle.TAG_ZERO_CANDIDATE, c, problem)
        c += 1
        if twin_key(dims, ix) in nzset:
            continue
        out.append((ix, 0.0, zeta / q, oracle.CLS_STRAT_ZERO))
    return out


def compare(S, twin):
    assert S.n == len(twin)
    for e, (ix, x, w, cls) in enumerate(twin):
        assert S.idx[e].tolist() == [int(v) for v in ix]
        assert S.x[e] == x
        assert S.w[e] == pytest.approx(w, rel=1e-15)
        assert S.cls[e] == cls


def sparse_problem(dims, density, seed, binary=False):
    rng = np.random.default_rng(seed)
    X = (rng.random(dims) < density) * (1.0 if binary else rng.integers(1, 5, dims))
    coo = np.argwhere(X != 0)
    vals = None if binary else X[tuple(coo.T)]
    return X, coo, vals


def test_uniform_matches_twin():
    dims = (5, 6, 7)
    X = np.random.default_rng(0).standard_normal(dims)
    S = oracle.sample(oracle.Tensor(dims, dense=X), oracle.UNIFORM, 0, 200, 17, 3)
    compare(S, twin_sample(dims, X, None, None, oracle.UNIFORM, 0, 200, 17, 3))


@pytest.mark.parametrize("binary", [False, True])
def test_stratified_matches_twin(binary):
    dims = (6, 5, 4, 3)
    X, coo, vals = sparse_problem(dims, 0.3, 1, binary)
    T = oracle.Tensor(dims, coo=coo, vals=vals)
    S = oracle.sample(T, oracle.STRATIFIED, 50, 80, 23, 9)
    compare(S, twin_sample(dims, X, coo, vals, oracle.STRATIFIED, 50, 80, 23, 9))
    # accepted zeros are zeros; nonzero draws are nonzeros
    for e in range(S.n):
        is_nz = X[tuple(S.idx[e])] != 0
        assert is_nz == (S.cls[e] == oracle.CLS_STRAT_NZ)


@pytest.mark.parametrize("binary", [False, True])
def test_semi_stratified_matches_twin(binary):
    dims = (6, 5, 4, 3, 2)
    X, coo, vals = sparse_problem(dims, 0.2, 2, binary)
    T = oracle.Tensor(dims, coo=coo, vals=vals)
    S = oracle.sample(T, oracle.SEMI_STRATIFIED, 40, 60, 29, 4)
    compare(S, twin_sample(dims, X, coo, vals, oracle.SEMI_STRATIFIED, 40, 60, 29, 4))


def test_stratified_candidates_counted():
    dims = (8, 8, 8)
    X, coo, vals = sparse_problem(dims, 0.5, 3)
    T = oracle.Tensor(dims, coo=coo, vals=vals)
    S = oracle.sample(T, oracle.STRATIFIED, 10, 100, 5, 0)
    nzset = {twin_key(dims, c) for c in coo}
    rejected = sum(twin_key(dims, twin_index(dims, 5, 0, oracle.TAG_ZERO_CANDIDATE, c)) in nzset
                   for c in range(S.candidates_used))
    assert S.candidates_used - rejected == 100
    # the last candidate examined was accepted
    last = twin_index(dims, 5, 0, oracle.TAG_ZERO_CANDIDATE, S.candidates_used - 1)
    assert twin_key(dims, last) not in nzset


def test_stratified_shortfall_is_reported():
    """With a single zero entry and rho tiny, 64 batches cannot supply q zeros."""
    dims = (4, 4, 4)
    coo = np.array([c for c in np.ndindex(*dims) if c != (1, 2, 3)])
    T = oracle.Tensor(dims, coo=coo, vals=np.ones(len(coo)))
    with pytest.raises(RuntimeError, match="short"):
        oracle.sample(T, oracle.STRATIFIED, 1, 50, 1, 0, rho=0.01)


def test_nonzero_draw_counts_are_binomial():
    dims = (10, 10, 10)
    X, coo, vals = sparse_problem(dims, 0.05, 4)
    T = oracle.Tensor(dims, coo=coo, vals=vals)
    p = 20000
    S = oracle.sample(T, oracle.SEMI_STRATIFIED, p, 0, 8, 0)
    keys = [twin_key(dims, ix) for ix in S.idx[:p].tolist()]
    eta = len(coo)
    counts = np.array([keys.count(twin_key(dims, c)) for c in coo])
    sd = math.sqrt(p * (1 / eta) * (1 - 1 / eta))
    assert np.all(np.abs(counts - p / eta) < 5 * sd)


def test_sorted_keys_membership():
    dims = (7, 9, 11)
    X, coo, vals = sparse_problem(dims, 0.1, 5)
    T = oracle.Tensor(dims, coo=coo, vals=vals)
    keys = T.sorted_keys()
    assert np.all(np.diff(keys.astype(np.float64)) > 0)
    flat = X.reshape(-1)
    lib = oracle._load()
    for key in range(flat.size):
        assert bool(lib.orc_is_nonzero(T.nnz, oracle._p(keys), key)) == (flat[key] != 0)


def test_uniform_over_sparse_tensor_matches_twin():
    """Alg. 1 on a sparse tensor: the value of a drawn index is its nonzero's
    value, or 0 (a Python dict lookup in the twin)."""
    dims = (6, 5, 4, 3)
    X, coo, vals = sparse_problem(dims, 0.3, 7)
    T = oracle.Tensor(dims, coo=coo, vals=vals)
    S = oracle.sample(T, oracle.UNIFORM, 0, 500, 3, 2)
    compare(S, twin_sample(dims, X, None, None, oracle.UNIFORM, 0, 500, 3, 2))


def test_uniform_with_entry_weights_matches_twin():
    """Weighted GCP (Eq. (4.5)) under Alg. 1: the draw's weight is (omega/s) v_i."""
    dims = (5, 6, 7)
    rng = np.random.default_rng(8)
    X = rng.standard_normal(dims)
    v = rng.random(dims) * (rng.random(dims) < 0.8)
    S = oracle.sample(oracle.Tensor(dims, dense=X, weights=v), oracle.UNIFORM, 0, 300, 4, 1)
    twin = twin_sample(dims, X, None, None, oracle.UNIFORM, 0, 300, 4, 1)
    twin = [(ix, x, w * v[tuple(ix)], c) for ix, x, w, c in twin]
    compare(S, twin)


def twin_observed(dims, X, v, q, seed, stream, rho=1.1, problem=0):
    """Uniform draws over the entries of nonzero weight (Section 4.4): candidates
    from their own stream, the first q with v != 0 kept in candidate order."""
    observed = int(np.count_nonzero(v))
    out, c = [], 0
    cap = 64 * math.ceil(rho * q * math.prod(dims) / observed)
    while len(out) < q:
        assert c < cap
        ix = twin_index(dims, seed, stream, oracle.TAG_OBSERVED, c, problem)
        c += 1
        if v[tuple(ix)] == 0:
            continue
        out.append((ix, X[tuple(ix)], observed / q * v[tuple(ix)], oracle.CLS_UNIFORM))
    return out


@pytest.mark.parametrize("missing", [0.0, 0.3, 0.9])
def test_observed_sampler_matches_twin(missing):
    dims = (6, 7, 8)
    rng = np.random.default_rng(10)
    X = rng.standard_normal(dims)
    v = rng.random(dims) * (rng.random(dims) >= missing)
    if missing == 0.0:
        v = np.ones(dims)
    S = oracle.sample(oracle.Tensor(dims, dense=X, weights=v), oracle.OBSERVED, 0, 400, 11, 6)
    compare(S, twin_observed(dims, X, v, 400, 11, 6))
    assert all(v[tuple(ix)] != 0 for ix in S.idx.tolist())  # missing entries are never drawn


def test_observed_sampler_shortfall_and_arguments():
    dims = (4, 4, 4)
    X = np.ones(dims)
    v = np.zeros(dims)
    v[1, 2, 3] = 1.0
    with pytest.raises(RuntimeError, match="short"):
        oracle.sample(oracle.Tensor(dims, dense=X, weights=v), oracle.OBSERVED, 0, 50, 1, 0, rho=0.01)
    with pytest.raises(ValueError):  # no weights: nothing defines the observed set
        oracle.sample(oracle.Tensor(dims, dense=X), oracle.OBSERVED, 0, 5, 1, 0)
    with pytest.raises(ValueError):  # every entry missing
        oracle.sample(oracle.Tensor(dims, dense=X, weights=np.zeros(dims)), oracle.OBSERVED, 0, 5, 1, 0)


def test_random_configurations_match_twin():
    """Forty seeded random configurations: 2 to 8 modes (modes 4-7 come from
    the second Philox block), extent-1 modes, densities from sparse to
    mostly full, random 64-bit seeds, streams (including the estimate stream
    2^64 - 1) and problem words, every sampler kind, p or q of 0."""
    rng = np.random.default_rng(2024)
    kinds = [oracle.UNIFORM, oracle.STRATIFIED, oracle.SEMI_STRATIFIED, oracle.OBSERVED]
    for case in range(40):
        d = int(rng.integers(2, 9))
        dims = tuple(int(n) for n in rng.integers(1, 7, d))
        while math.prod(dims) < 24:
            dims = tuple(n + 1 for n in dims)
        kind = kinds[case % 4]
        seed, problem = (int(v) * 2 + 1 for v in rng.integers(0, 2**63, 2, dtype=np.int64))  # full 64-bit words
        stream = 2**64 - 1 if case % 7 == 0 else int(rng.integers(0, 2**62))
        p = 0 if kind in (oracle.UNIFORM, oracle.OBSERVED) or case % 5 == 0 else int(rng.integers(1, 40))
        q = 0 if case % 5 == 1 else int(rng.integers(1, 60))
        if kind in (oracle.UNIFORM, oracle.OBSERVED):
            X = rng.standard_normal(dims)
            if kind == oracle.OBSERVED:
                v = rng.random(dims) * (rng.random(dims) >= rng.uniform(0.0, 0.8))
                v.reshape(-1)[0] = 1.0  # at least one observed entry
                S = oracle.sample(oracle.Tensor(dims, dense=X, weights=v), kind, 0, q, seed, stream, problem=problem)
                twin = twin_observed(dims, X, v, q, seed, stream, problem=problem)
            else:
                S = oracle.sample(oracle.Tensor(dims, dense=X), kind, 0, q, seed, stream, problem=problem)
                twin = twin_sample(dims, X, None, None, kind, 0, q, seed, stream, problem=problem)
        else:
            X, coo, vals = sparse_problem(dims, float(rng.uniform(0.05, 0.6)), case, binary=bool(case % 2))
            if len(coo) == 0 or len(coo) == math.prod(dims):
                continue
            T = oracle.Tensor(dims, coo=coo, vals=vals)
            S = oracle.sample(T, kind, p, q, seed, stream, problem=problem)
            twin = twin_sample(dims, X, coo, vals, kind, p, q, seed, stream, problem=problem)
        compare(S, twin)


@pytest.mark.parametrize("kind", [oracle.STRATIFIED, oracle.OBSERVED])
def test_rejection_stops_after_exactly_64_batches(kind):
    """One acceptable entry in 10^4 and q = 1: the first acceptance comes at
    candidate c*.  Batches of b candidates find it iff 64 b > c* (the cap is
    64 batches), so a b with 64 b <= c* < 65 b falls short and b + 1 does not
    once 64 (b + 1) > c*."""
    dims = (10, 10, 100)
    omega = math.prod(dims)
    lone = (3, 7, 42)
    for seed in range(1, 200):
        if kind == oracle.STRATIFIED:
            coo = np.array([c for c in np.ndindex(*dims) if c != lone])
            T = oracle.Tensor(dims, coo=coo, vals=np.ones(len(coo)))
            p = 1
        else:
            v = np.zeros(dims)
            v[lone] = 1.0
            T = oracle.Tensor(dims, dense=np.ones(dims), weights=v)
            p = 0
        c_star = oracle.sample(T, kind, p, 1, seed, 0, rho=1.0).candidates_used - 1
        b = -(-(c_star + 1) // 65)  # ceil((c* + 1) / 65): 65 b > c*
        if 64 * b <= c_star:
            break
    else:
        pytest.fail("no seed puts the first acceptance at the cap boundary")
    rho = lambda batch: (batch - 0.5) / omega  # ceil(rho q omega / 1) = batch
    with pytest.raises(RuntimeError, match="short"):
        oracle.sample(T, kind, p, 1, seed, 0, rho=rho(b))
    ok_b = -(-(c_star + 1) // 64)
    S = oracle.sample(T, kind, p, 1, seed, 0, rho=rho(ok_b))
    assert S.candidates_used == c_star + 1 and tuple(S.idx[-1]) == lone


def test_first_batch_success_rate_is_binomial():
    """App. B's oversampling argument: a batch of b candidates, each a zero
    with probability zeta / omega, holds at least q zeros with probability
    P(Binomial(b, zeta / omega) >= q).  Over many seeds the share of runs
    that stop within the first batch matches it (scipy's binomial tail)."""
    from scipy import stats
    dims = (20, 20, 20)
    omega = math.prod(dims)
    rng = np.random.default_rng(77)
    keys = rng.choice(omega, omega // 2, replace=False)
    coo = np.stack(np.unravel_index(keys, dims), axis=1)
    T = oracle.Tensor(dims, coo=coo, vals=np.ones(len(coo)))
    q, rho = 200, 1.0
    batch = math.ceil(rho * q * omega / (omega - len(coo)))
    p_one = stats.binom.sf(q - 1, batch, (omega - len(coo)) / omega)
    runs = 600
    within = sum(oracle.sample(T, oracle.STRATIFIED, 0, q, seed, 0, rho=rho).candidates_used <= batch
                 for seed in range(runs))
    sd = math.sqrt(p_one * (1 - p_one) / runs)
    assert abs(within / runs - p_one) < 5 * sd, (within / runs, p_one)
