"""FP64 CPU oracle for the sampled GCP gradient (arXiv:1906.01687).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` are the only
callers.  The product library never imports this package, and this package
imports nothing from the product.

The arithmetic lives in ``gcp_oracle.c`` (plain C, FP64).  This module builds
it with gcc on first use, loads it with ctypes and converts numpy arrays.
Each wrapper names the passage of the paper its C function follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gcp_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libgcp_oracle.so")
_lock = threading.Lock()
_lib = None

# classes, losses and samplers: the same numbering the C file defines
UNIFORM, STRATIFIED, SEMI_STRATIFIED, OBSERVED = 0, 1, 2, 3
GAUSSIAN, BERNOULLI_LOGIT, POISSON_LOG = 0, 1, 2
BERNOULLI_ODDS, POISSON_IDENTITY, GAMMA, BETA_HALF = 3, 4, 5, 6
M_EPS = 1e-10  # odds/identity-link losses are evaluated at m + M_EPS
CLS_UNIFORM, CLS_STRAT_NZ, CLS_STRAT_ZERO, CLS_SEMI_NZ, CLS_SEMI_ZERO = 0, 1, 2, 3, 4
TAG_UNIFORM, TAG_NONZERO, TAG_ZERO_CANDIDATE, TAG_SEMI_ZERO, TAG_OBSERVED = 0, 1, 2, 3, 4
OK, ERR_ARG, ERR_SHORTFALL = 0, 1, 4


def build(force: bool = False) -> str:
    """Compile gcp_oracle.c into _build/libgcp_oracle.so (gcc -O2, no fast-math)."""
    with _lock:
        os.makedirs(os.path.dirname(_LIB), exist_ok=True)
        stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
        if force or stale:
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(
                ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
                 "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    P = ctypes.POINTER
    u64, i64, i32, f64 = ctypes.c_uint64, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    vp = ctypes.c_void_p
    lib.orc_philox4x64.argtypes = [vp, vp, vp]
    lib.orc_randi.argtypes = [u64, u64]
    lib.orc_randi.restype = u64
    lib.orc_draw_multi_index.argtypes = [i32, vp, u64, u64, u64, ctypes.c_uint32, u64, vp]
    lib.orc_draw_nonzero.argtypes = [i64, u64, u64, u64, u64]
    lib.orc_draw_nonzero.restype = i64
    lib.orc_linear_key.argtypes = [i32, vp, vp]
    lib.orc_linear_key.restype = u64
    lib.orc_loss_f.argtypes = [i32, f64, f64]
    lib.orc_loss_f.restype = f64
    lib.orc_loss_g.argtypes = [i32, f64, f64]
    lib.orc_loss_g.restype = f64
    lib.orc_model_value.argtypes = [i32, vp, i32, vp, vp]
    lib.orc_model_value.restype = f64
    lib.orc_sorted_keys.argtypes = [i32, vp, i64, vp, vp]
    lib.orc_is_nonzero.argtypes = [i64, vp, u64]
    lib.orc_is_nonzero.restype = i32
    lib.orc_sample_count.argtypes = [i32, i64, i64]
    lib.orc_sample_count.restype = i64
    lib.orc_sample.argtypes = [i32, vp, i32, vp, vp, i64, vp, vp, vp, vp, i32, i64, i64,
                               u64, u64, u64, f64, vp, vp, vp, vp, P(i64)]
    lib.orc_sorted_pairs.argtypes = [i32, vp, i64, vp, vp, vp, vp]
    lib.orc_sparse_value.argtypes = [i64, vp, vp, u64]
    lib.orc_sparse_value.restype = f64
    lib.orc_sample.restype = i32
    lib.orc_entry_y.argtypes = [i32, i32, f64, f64, f64]
    lib.orc_entry_y.restype = f64
    lib.orc_entry_f.argtypes = [i32, i32, f64, f64, f64]
    lib.orc_entry_f.restype = f64
    lib.orc_grad_from_samples.argtypes = [i32, vp, i32, vp, i32, i64, vp, vp, vp, vp, vp]
    lib.orc_grad_from_samples.restype = i32
    lib.orc_loss_from_samples.argtypes = [i32, vp, i32, vp, i32, i64, vp, vp, vp, vp]
    lib.orc_loss_from_samples.restype = f64
    lib.orc_loss_abs_from_samples.argtypes = [i32, vp, i32, vp, i32, i64, vp, vp, vp, vp]
    lib.orc_loss_abs_from_samples.restype = f64
    lib.orc_grad_abs_from_samples.argtypes = [i32, vp, i32, vp, i32, i64, vp, vp, vp, vp, vp]
    lib.orc_grad_abs_from_samples.restype = i32
    lib.orc_full_grad.argtypes = [i32, vp, i32, vp, i32, vp, vp, vp, P(f64)]
    lib.orc_full_grad.restype = i32
    lib.orc_adam_step.argtypes = [i64, vp, vp, vp, vp, f64, f64, f64, f64, f64, i64, i32]
    _lib = lib
    return lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------------------
# random numbers (Section 4.1; Philox4x64-10 of Salmon et al.)
# --------------------------------------------------------------------------

def philox4x64(counter, key) -> np.ndarray:
    """One Philox4x64-10 block: 4 uint64 words for counter (4 words), key (2 words)."""
    lib = _load()
    c = np.ascontiguousarray(counter, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib.orc_philox4x64(_p(c), _p(k), _p(out))
    return out


def randi(word: int, n: int) -> int:
    """0-based randi(n) of Section 4.1: floor(word * n / 2^64)."""
    return int(_load().orc_randi(int(word), int(n)))


def draw_multi_index(dims, seed, problem, stream, tag, j) -> np.ndarray:
    dims = _i64(dims)
    out = np.zeros(len(dims), dtype=np.int64)
    _load().orc_draw_multi_index(len(dims), _p(dims), seed, problem, stream, tag, j, _p(out))
    return out


def draw_nonzero(nnz, seed, problem, stream, j) -> int:
    return int(_load().orc_draw_nonzero(nnz, seed, problem, stream, j))


def linear_key(dims, idx) -> int:
    dims, idx = _i64(dims), _i64(idx)
    return int(_load().orc_linear_key(len(dims), _p(dims), _p(idx)))


# --------------------------------------------------------------------------
# losses (Section 1; log-link forms of the cited GCP paper)
# --------------------------------------------------------------------------

def loss_f(loss: int, x: float, m: float) -> float:
    return float(_load().orc_loss_f(loss, x, m))


def loss_g(loss: int, x: float, m: float) -> float:
    return float(_load().orc_loss_g(loss, x, m))


def entry_y(loss, cls, x, m, w) -> float:
    return float(_load().orc_entry_y(loss, cls, x, m, w))


def entry_f(loss, cls, x, m, w) -> float:
    return float(_load().orc_entry_f(loss, cls, x, m, w))


# --------------------------------------------------------------------------
# tensors and factors
# --------------------------------------------------------------------------

class Tensor:
    """A dense or COO tensor as the oracle sees it (FP64 values, int64 indices).

    dense: ``vals`` holds prod(dims) entries in row-major order.
    sparse: ``coo`` is nnz x d (int64), ``vals`` nnz values or None (all ones).
    """

    def __init__(self, dims, dense=None, coo=None, vals=None, weights=None):
        self.dims = _i64(dims)
        self.weights = None if weights is None else _f64(np.asarray(weights).reshape(-1))
        self.d = len(self.dims)
        self.sparse = coo is not None
        if self.sparse:
            coo = np.asarray(coo)
            if coo.ndim != 2 or coo.shape[1] != self.d:  # one orientation only: nnz == d would be ambiguous
                raise ValueError(f"coo must be nnz x d (one row per nonzero), got shape {coo.shape}")
            self.coo = _i64(coo)
            self.nnz = self.coo.shape[0]
            self.vals = None if vals is None else _f64(vals)
            self.dense = None
            self._keys = None
        else:
            self.dense = _f64(np.asarray(dense).reshape(-1))
            self.coo, self.vals, self.nnz, self._keys = None, None, 0, None

    def sorted_pairs(self):
        """(keys, values) of the nonzeros sorted by key: the value lookup of uniform sampling."""
        if getattr(self, "_pairs", None) is None:
            keys = np.zeros(self.nnz, dtype=np.uint64)
            vals = np.zeros(self.nnz)
            _load().orc_sorted_pairs(self.d, _p(self.dims), self.nnz, _p(self.coo), _p(self.vals), _p(keys), _p(vals))
            self._pairs = (keys, vals)
        return self._pairs

    def sorted_keys(self) -> np.ndarray:
        """Sorted row-major linear keys of the nonzeros (Section 4.2's lookup list)."""
        if self._keys is None:
            keys = np.zeros(self.nnz, dtype=np.uint64)
            _load().orc_sorted_keys(self.d, _p(self.dims), self.nnz, _p(self.coo), _p(keys))
            self._keys = keys
        return self._keys


def concat_factors(factors) -> np.ndarray:
    """Concatenate n_k x r factor matrices (row-major) into one FP64 vector."""
    return np.concatenate([_f64(a).reshape(-1) for a in factors])


def split_factors(flat, dims, rank):
    out, off = [], 0
    for n in dims:
        out.append(flat[off:off + n * rank].reshape(n, rank))
        off += n * rank
    return out


def model_value(dims, factors, idx) -> float:
    dims = _i64(dims)
    rank = factors[0].shape[1]
    A = concat_factors(factors)
    idx = _i64(idx)
    return float(_load().orc_model_value(len(dims), _p(dims), rank, _p(A), _p(idx)))


# --------------------------------------------------------------------------
# sampling (Algs. 1-3) and the drawn-entry list
# --------------------------------------------------------------------------

class Samples:
    """An explicit list of drawn entries: idx (n x d), x, w, cls."""

    def __init__(self, idx, x, w, cls, candidates_used=0):
        self.idx = _i64(idx)
        self.x = _f64(x)
        self.w = _f64(w)
        self.cls = np.ascontiguousarray(cls, dtype=np.int8)
        self.n = self.x.shape[0]
        self.candidates_used = candidates_used


def sample(X: Tensor, kind: int, p: int, q: int, seed: int, stream: int,
           problem: int = 0, rho: float = 1.1) -> Samples:
    """Draw the sample list of Alg. 1 (kind 0), Alg. 2 (kind 1), Alg. 3 (kind 2),
    or uniform draws over the entries of nonzero weight (kind 3, Section 4.4;
    a dense tensor with weights).

    Raises RuntimeError on a shortfall (fewer than q accepted after 64 batches
    of candidates).
    """
    lib = _load()
    n = int(lib.orc_sample_count(kind, p, q))
    idx = np.zeros((n, X.d), dtype=np.int64)
    x = np.zeros(n)
    w = np.zeros(n)
    cls = np.zeros(n, dtype=np.int8)
    used = ctypes.c_int64(0)
    keys = X.sorted_keys() if (X.sparse and kind == STRATIFIED) else None
    svals = None
    if X.sparse and kind == UNIFORM:
        keys, svals = X.sorted_pairs()
    st = lib.orc_sample(X.d, _p(X.dims), int(X.sparse), _p(X.dense), _p(X.weights), X.nnz, _p(X.coo), _p(X.vals),
                        _p(keys), _p(svals), kind, p, q, seed, problem, stream, rho,
                        _p(idx), _p(x), _p(w), _p(cls), ctypes.byref(used))
    if st == ERR_SHORTFALL:
        raise RuntimeError(f"rejection sampling fell short after {used.value} candidates")
    if st != OK:
        raise ValueError(f"oracle sample: invalid arguments (status {st})")
    return Samples(idx, x, w, cls, used.value)


# --------------------------------------------------------------------------
# gradient, loss estimate, full gradient, Adam
# --------------------------------------------------------------------------

def grad(dims, factors, loss: int, S: Samples):
    """Sampled gradient {G_k} of Eq. (4.3) for the drawn entries S (FP64)."""
    lib = _load()
    dims = _i64(dims)
    rank = factors[0].shape[1]
    A = concat_factors(factors)
    G = np.zeros_like(A)
    st = lib.orc_grad_from_samples(len(dims), _p(dims), rank, _p(A), loss, S.n,
                                   _p(S.idx), _p(S.x), _p(S.w), _p(S.cls), _p(G))
    if st != OK:
        raise ValueError("oracle grad: invalid arguments")
    return split_factors(G, dims, rank)


def loss_estimate(dims, factors, loss: int, S: Samples) -> float:
    """Fixed-sample estimate F-hat of Eqs. (5.1)-(5.2) (FP64)."""
    lib = _load()
    dims = _i64(dims)
    rank = factors[0].shape[1]
    A = concat_factors(factors)
    return float(lib.orc_loss_from_samples(len(dims), _p(dims), rank, _p(A), loss, S.n,
                                           _p(S.idx), _p(S.x), _p(S.w), _p(S.cls)))


def loss_abs(dims, factors, loss: int, S: Samples) -> float:
    """Sum of |term| of F-hat over S: the error scale of any summation order."""
    lib = _load()
    dims = _i64(dims)
    rank = factors[0].shape[1]
    A = concat_factors(factors)
    return float(lib.orc_loss_abs_from_samples(len(dims), _p(dims), rank, _p(A), loss, S.n,
                                               _p(S.idx), _p(S.x), _p(S.w), _p(S.cls)))


def grad_abs(dims, factors, loss: int, S: Samples):
    """Per-entry sum of |contribution| to the sampled gradient over S."""
    lib = _load()
    dims = _i64(dims)
    rank = factors[0].shape[1]
    A = concat_factors(factors)
    G = np.zeros_like(A)
    st = lib.orc_grad_abs_from_samples(len(dims), _p(dims), rank, _p(A), loss, S.n,
                                       _p(S.idx), _p(S.x), _p(S.w), _p(S.cls), _p(G))
    if st != OK:
        raise ValueError("oracle grad_abs: invalid arguments")
    return split_factors(G, dims, rank)


def full_grad(dims, factors, loss: int, X_dense, weights=None):
    """Full gradient G_k = Y_(k) Z_k (Eq. (4.2)) and F (Eq. (1.2)) of a dense tensor."""
    lib = _load()
    dims = _i64(dims)
    rank = factors[0].shape[1]
    A = concat_factors(factors)
    G = np.zeros_like(A)
    Xd = _f64(np.asarray(X_dense).reshape(-1))
    v = None if weights is None else _f64(np.asarray(weights).reshape(-1))
    F = ctypes.c_double(0.0)
    st = lib.orc_full_grad(len(dims), _p(dims), rank, _p(A), loss, _p(Xd), _p(v), _p(G), ctypes.byref(F))
    if st != OK:
        raise ValueError("oracle full_grad: invalid arguments")
    return split_factors(G, dims, rank), F.value


def adam_step(A, B, C, G, alpha, beta1=0.9, beta2=0.999, eps=1e-8, lower=-np.inf,
              t=0, eps_inside_sqrt=True):
    """One Adam step with projection (Alg. 4) on flat FP64 arrays, in place.

    t counts the steps already taken; the bias correction uses t + 1.
    """
    lib = _load()
    for a in (A, B, C):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    G = _f64(G)
    lib.orc_adam_step(A.size, _p(A), _p(B), _p(C), _p(G), alpha, beta1, beta2, eps, lower,
                      int(t), int(bool(eps_inside_sqrt)))
