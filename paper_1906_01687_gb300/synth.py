"""Seeded synthetic inputs shaped like the paper's workloads.

This module makes data only: planted low-rank tensors (dense or COO), initial
guesses, and the shapes of the five standard workloads.  It holds none of the
sampled-gradient arithmetic, imports nothing else from this package, and is
the one module that both the CUDA path's callers and the FP64 oracle's
callers use, so that the two see identical inputs.

All arrays are numpy (host).  Dense tensors are row-major (last mode fastest).
COO tensors are returned as SoA int32 index arrays ``idx[k]`` (length nnz)
plus values (or None for an all-ones binary tensor), with unique indices.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


# ---------------------------------------------------------------------------
# the five standard workloads
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Workload:
    name: str
    dims: tuple
    rank: int
    loss: str            # "gaussian" | "bernoulli_logit" | "poisson_log"
    sampler: str         # "uniform" | "stratified" | "semi_stratified"
    p: int               # nonzero draws per iteration (0 for uniform)
    q: int               # zero / uniform draws per iteration
    est_p: int           # loss-estimate sample set
    est_q: int
    sparse: bool
    nnz: int = 0
    lr: float = 1e-3
    tau: int = 100       # iterations per epoch


# Dense 20x30x40, planted rank 3, Gaussian, uniform s = 1000, 500 estimate samples.
DENSE_SMALL = Workload("dense-20x30x40-r3-gaussian-uniform", (20, 30, 40), 3, "gaussian",
                       "uniform", 0, 1000, 0, 500, False, lr=1e-3, tau=100)
# Dense 100^4 (1e8 entries), planted rank 10, Gaussian, uniform s = 1e5.
DENSE_100_4 = Workload("dense-100x100x100x100-r10-gaussian-uniform", (100, 100, 100, 100), 10,
                       "gaussian", "uniform", 0, 100_000, 0, 100_000, False, lr=1e-3, tau=100)
# Sparse count tensor with the Chicago crime shape, ~5.33M nonzeros, Poisson-log, stratified.
COUNT_CHICAGO_SHAPE = Workload("coo-6186x24x77x32-r10-poissonlog-stratified", (6186, 24, 77, 32), 10,
                               "poisson_log", "stratified", 100_000, 100_000, 100_000, 100_000,
                               True, nnz=5_330_673, lr=1e-3, tau=100)
# Sparse binary 1e5 x 1e5 x 1e4, 1e8 nonzeros, Bernoulli-logit, semi-stratified.
BINARY_LARGE = Workload("coo-1e5x1e5x1e4-r32-bernoullilogit-semistratified", (100_000, 100_000, 10_000),
                        32, "bernoulli_logit", "semi_stratified", 1_000_000, 1_000_000,
                        100_000, 100_000, True, nnz=100_000_000, lr=1e-3, tau=100)

WORKLOADS = {w.name: w for w in (DENSE_SMALL, DENSE_100_4, COUNT_CHICAGO_SHAPE, BINARY_LARGE)}


# ---------------------------------------------------------------------------
# planted models
# ---------------------------------------------------------------------------

def _khatri_rao_rows(factors):
    """Row-major Khatri-Rao product of factors[0..] (rows of the last factor fastest)."""
    out = factors[0]
    for a in factors[1:]:
        out = (out[:, None, :] * a[None, :, :]).reshape(-1, a.shape[1])
    return out


def dense_from_factors(factors, weights=None) -> np.ndarray:
    """Dense row-major tensor sum_j w_j a_1j o ... o a_dj (data synthesis)."""
    dims = tuple(a.shape[0] for a in factors)
    rank = factors[0].shape[1]
    w = np.ones(rank) if weights is None else np.asarray(weights, dtype=np.float64)
    first = factors[0] * w[None, :]
    rest = _khatri_rao_rows(list(factors[1:])) if len(factors) > 1 else np.ones((1, rank))
    return (first @ rest.T).reshape(dims)


def planted_dense(dims, rank, seed, noise_std, normalize_columns=False, weights=None,
                  dtype=np.float64):
    """Planted rank-r dense tensor X = M_true + noise_std * N(0,1).

    Factor entries are iid N(0,1); with normalize_columns each column has unit
    2-norm.  Returns (X, true_factors, weights).
    """
    rng = np.random.default_rng(seed)
    factors = [rng.standard_normal((n, rank)) for n in dims]
    if normalize_columns:
        factors = [a / np.linalg.norm(a, axis=0, keepdims=True) for a in factors]
    w = np.ones(rank) if weights is None else np.asarray(weights, dtype=np.float64)
    M = dense_from_factors(factors, w)
    X = M + noise_std * rng.standard_normal(M.shape)
    return X.astype(dtype), factors, w


def dense_small(seed=1907):
    """20x30x40 FP64 tensor: planted rank 3 (N(0,1) factors, unit columns, weights 1) + 0.1 N(0,1)."""
    return planted_dense((20, 30, 40), 3, seed, 0.1, normalize_columns=True, dtype=np.float64)


def dense_100_4(seed=1908):
    """100^4 FP32 tensor: planted rank 10 (N(0,1) factors) + N(0, 0.01) noise (std 0.1)."""
    rng = np.random.default_rng(seed)
    dims, rank = (100, 100, 100, 100), 10
    factors = [rng.standard_normal((n, rank)).astype(np.float32) for n in dims]
    kr = _khatri_rao_rows([a.astype(np.float32) for a in factors[1:]])  # 1e6 x 10
    M = (factors[0] @ kr.T).reshape(dims)
    M += np.float32(0.1) * rng.standard_normal(M.shape, dtype=np.float32)
    return M, factors


# ---------------------------------------------------------------------------
# sparse tensors
# ---------------------------------------------------------------------------

def _row_major_keys(idx, dims):
    key = np.zeros(idx[0].shape[0], dtype=np.uint64)
    for k, n in enumerate(dims):
        key = key * np.uint64(n) + idx[k].astype(np.uint64)
    return key


def _keys_to_idx(keys, dims):
    idx = [None] * len(dims)
    rem = keys.copy()
    for k in range(len(dims) - 1, -1, -1):
        idx[k] = (rem % np.uint64(dims[k])).astype(np.int32)
        rem //= np.uint64(dims[k])
    return idx


def count_tensor(dims=(6186, 24, 77, 32), nnz=5_330_673, rank=10, seed=1909, zipf_a=1.0):
    """Sparse count tensor shaped like the Chicago crime tensor (Section 5.6).

    Nonzero positions: mode-1 index drawn with P(i) proportional to 1/(i+1)^zipf_a
    (a skewed day axis), other modes uniform, duplicates removed until nnz
    unique positions remain.  Values: 1 + Poisson(lambda_i), lambda_i the
    planted nonnegative rank-r model (gamma(1,1) factors) at the position,
    rescaled to mean 1.  Returns (idx[d] int32, vals float32, factors).
    """
    rng = np.random.default_rng(seed)
    d = len(dims)
    omega = int(np.prod(np.array(dims, dtype=np.float64)))
    assert nnz < omega
    p1 = 1.0 / np.power(np.arange(1, dims[0] + 1, dtype=np.float64), zipf_a)
    p1 /= p1.sum()
    cdf1 = np.cumsum(p1)
    keys = np.zeros(0, dtype=np.uint64)
    while keys.shape[0] < nnz:
        need = int((nnz - keys.shape[0]) * 1.3) + 1024
        u = rng.random(need)
        i0 = np.minimum(np.searchsorted(cdf1, u, side="right"), dims[0] - 1).astype(np.int64)
        cand = [i0] + [rng.integers(0, n, need) for n in dims[1:]]
        ck = _row_major_keys(cand, dims)
        keys = np.unique(np.concatenate([keys, ck]))
    # keep a random subset of exactly nnz unique positions
    keep = np.sort(rng.choice(keys.shape[0], nnz, replace=False))
    keys = keys[keep]
    idx = _keys_to_idx(keys, dims)
    factors = [rng.gamma(1.0, 1.0, (n, rank)) for n in dims]
    lam = np.ones(nnz)
    for j in range(rank):
        col = np.ones(nnz)
        for k in range(d):
            col *= factors[k][idx[k], j]
        lam = lam + col if j else col
    lam *= 1.0 / lam.mean()
    vals = (1.0 + rng.poisson(lam)).astype(np.float32)
    return idx, vals, factors


def binary_tensor(dims=(100_000, 100_000, 10_000), nnz=100_000_000, rank=32, seed=1910,
                  device="cpu", chunk=1 << 22):
    """Sparse binary tensor drawn from a planted rank-r logistic model.

    Candidate positions are uniform over the index space; a candidate is kept
    with probability sigmoid(m_i) of the planted model (factor entries
    N(0, s^2) with s set so that m_i has unit variance), duplicates are
    removed, and the first nnz unique positions in draw order are kept.
    Uses torch (on ``device``) for speed at 1e8 nonzeros; the result is
    returned as host numpy arrays.  Returns (idx[d] int32, None, factors).
    """
    import torch

    d = len(dims)
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    s = (1.0 / rank) ** (1.0 / (2 * d))  # var(m) = r * s^(2d) = 1
    factors = [torch.randn((n, rank), generator=g, device=device) * s for n in dims]
    kept = []
    total = 0
    while total < nnz * 1.02 + 1024:
        cand = [torch.randint(0, n, (chunk,), generator=g, device=device) for n in dims]
        prod = factors[0][cand[0]]
        for k in range(1, d):
            prod = prod * factors[k][cand[k]]
        m = prod.sum(dim=1)
        u = torch.rand((chunk,), generator=g, device=device)
        acc = u < torch.sigmoid(m)
        key = torch.zeros(chunk, dtype=torch.int64, device=device)
        for k in range(d):
            key = key * dims[k] + cand[k]
        kept.append(key[acc])
        total += int(acc.sum())
    keys = torch.cat(kept)
    uniq, inv = torch.unique(keys, sorted=True, return_inverse=True)
    # first occurrence of each unique key, in draw order
    first = torch.full((uniq.shape[0],), keys.shape[0], dtype=torch.int64, device=device)
    first.scatter_reduce_(0, inv, torch.arange(keys.shape[0], device=device), reduce="amin")
    order = torch.argsort(first)[:nnz]
    sel = torch.sort(uniq[order]).values
    keys_np = sel.cpu().numpy().astype(np.uint64)
    idx = _keys_to_idx(keys_np, dims)
    return idx, None, [f.cpu().numpy() for f in factors]


# ---------------------------------------------------------------------------
# initial guesses
# ---------------------------------------------------------------------------

def initial_guess(dims, rank, seed, target_norm=None, positive=False, dtype=np.float32):
    """Random initial factor matrices (Alg. 4, first loop).

    Entries iid N(0,1) (or uniform(0,1) when positive).  With target_norm the
    factors are scaled equally so that the model's Frobenius norm, computed in
    closed form from the Gram matrices, equals target_norm.
    """
    rng = np.random.default_rng(seed)
    if positive:
        A = [rng.random((n, rank)) for n in dims]
    else:
        A = [rng.standard_normal((n, rank)) for n in dims]
    if target_norm is not None:
        gram = np.ones((rank, rank))
        for a in A:
            gram *= a.T @ a
        norm_m = math.sqrt(max(gram.sum(), 1e-300))
        scale = (target_norm / norm_m) ** (1.0 / len(dims))
        A = [a * scale for a in A]
    return [a.astype(dtype) for a in A]


# ---------------------------------------------------------------------------
# batched problems (many independent decompositions)
# ---------------------------------------------------------------------------

def batched_problems(count=64, seed=1911, dim_lo=50, dim_hi=2000, max_entries=20_000_000,
                     ranks=(4, 8, 16, 32, 64), losses=("gaussian", "bernoulli_logit", "poisson_log"),
                     s_lo=10_000, s_hi=100_000):
    """Shapes of independent dense problems: d in {3,4}; each dim uniform in
    [dim_lo, cap] where cap = min(dim_hi, the largest value that still lets the
    remaining dims reach dim_lo within max_entries), dims then shuffled (plain
    rejection of whole shapes almost never accepts a 4-way shape); rank from
    ``ranks``; loss mixed; draws per iteration log-uniform in [s_lo, s_hi]."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(count):
        d = int(rng.integers(3, 5))
        dims, prod = [], 1
        for k in range(d):
            remaining = d - k - 1
            cap = int(min(dim_hi, max_entries // (prod * dim_lo ** remaining)))
            n = int(rng.integers(dim_lo, max(dim_lo, cap) + 1))
            dims.append(n)
            prod *= n
        dims = tuple(int(v) for v in rng.permutation(dims))
        rank = int(ranks[rng.integers(0, len(ranks))])
        loss = losses[b % len(losses)]
        s = int(round(math.exp(rng.uniform(math.log(s_lo), math.log(s_hi)))))
        out.append(dict(dims=dims, rank=rank, loss=loss, s=s))
    return out


def planted_for_loss(dims, rank, loss, seed, dtype=np.float32):
    """Planted dense data for one batched problem.

    gaussian: N(0,1) factors scaled to unit-variance entries, plus 0.1 N(0,1);
    bernoulli_logit: x ~ Bernoulli(sigmoid(m)); poisson_log: x ~ Poisson(exp(m)),
    with m of unit variance.
    """
    rng = np.random.default_rng(seed)
    d = len(dims)
    s = (1.0 / rank) ** (1.0 / (2 * d))
    factors = [rng.standard_normal((n, rank)) * s for n in dims]
    M = dense_from_factors(factors)
    if loss == "gaussian":
        X = M + 0.1 * rng.standard_normal(M.shape)
    elif loss == "bernoulli_logit":
        X = (rng.random(M.shape) < 1.0 / (1.0 + np.exp(-M))).astype(np.float64)
    elif loss == "poisson_log":
        X = rng.poisson(np.exp(np.minimum(M, 10.0))).astype(np.float64)
    else:
        raise ValueError(loss)
    return X.astype(dtype), factors


# ---------------------------------------------------------------------------
# the paper's test-problem recipes for its odds / identity-link losses
# ---------------------------------------------------------------------------

def gamma_problem(dims=(200, 150, 100, 50), rank=5, seed=1912):
    """App. C: factor entries uniform(0,1); x_i ~ gamma with shape 1 and mean
    m_i (an exponential draw).  Returns (X float32, factors)."""
    rng = np.random.default_rng(seed)
    factors = [rng.random((n, rank)) for n in dims]
    M = dense_from_factors(factors)
    X = rng.exponential(M)
    return X.astype(np.float32), factors


def app_d_factors(rng, dims, rank, delta=0.15, p_high=0.9, p_low=0.0025):
    """App. D's planted odds model: components 1..r-1 sparse (density delta,
    nonzero entries |N(root_d(p_high / (1 - p_high)), 0.5^2)|), component r
    dense with entries root_d(p_low / (1 - p_low))."""
    d = len(dims)
    hi = (p_high / (1 - p_high)) ** (1.0 / d)
    lo = (p_low / (1 - p_low)) ** (1.0 / d)
    factors = []
    for n in dims:
        a = np.zeros((n, rank))
        mask = rng.random((n, rank - 1)) < delta
        a[:, : rank - 1] = np.where(mask, np.abs(rng.normal(hi, 0.5, (n, rank - 1))), 0.0)
        a[:, rank - 1] = lo
        factors.append(a)
    return factors


def binary_odds_problem(dims=(200, 150, 100, 50), rank=5, delta=0.15, p_high=0.9, p_low=0.0025, seed=1913):
    """App. D: x_i ~ Bernoulli(m_i / (1 + m_i)) with m the odds of the planted
    model of app_d_factors.  Dense generation on the host (moderate sizes).
    Returns (X float32, factors)."""
    rng = np.random.default_rng(seed)
    factors = app_d_factors(rng, dims, rank, delta, p_high, p_low)
    M = dense_from_factors(factors)
    X = (rng.random(M.shape) < M / (1.0 + M)).astype(np.float32)
    return X, factors


def binary_odds_coo(dims=(400, 300, 200, 100), rank=5, delta=0.15, p_high=0.9, p_low=0.0025, seed=1913,
                    device="cuda", slab=8):
    """App. D at the size of the paper's sampler comparison (Section 5.2:
    400 x 300 x 200 x 100, rank 5, about 0.38% nonzeros), generated on the
    device a few mode-1 slices at a time (torch's seeded generator draws the
    Bernoulli variables).  Returns (COO indices as one int32 tensor per mode,
    sorted row-major, and the factors)."""
    import torch
    rng = np.random.default_rng(seed)
    factors = app_d_factors(rng, dims, rank, delta, p_high, p_low)
    A = [torch.as_tensor(a, device=device, dtype=torch.float64) for a in factors]
    rest = A[1]
    for a in A[2:]:  # Khatri-Rao-like outer product of modes 2..d, kept per component
        rest = (rest.unsqueeze(-2) * a.reshape((1,) * (rest.dim() - 1) + a.shape)).reshape(-1, rank)
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    parts = []
    for i0 in range(0, dims[0], slab):
        i1 = min(dims[0], i0 + slab)
        M = A[0][i0:i1] @ rest.T  # (slab, prod(dims[1:])) odds
        u = torch.rand(M.shape, generator=gen, device=device, dtype=torch.float64)
        nz = torch.nonzero(u < M / (1.0 + M))
        nz[:, 0] += i0
        parts.append(nz)
    nz = torch.cat(parts)
    idx = [nz[:, 0].to(torch.int32)]
    rem = nz[:, 1]
    tail = []
    for n in reversed(dims[1:]):
        tail.append((rem % n).to(torch.int32))
        rem = rem // n
    idx += list(reversed(tail))
    return idx, factors
