"""Helpers of the GPU parity tests: move seeded inputs to both sides, compare
the CUDA path's results with the FP64 oracle's."""
import math

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")

GRAD_RTOL = 1e-5        # norm-wise, FP32 path vs FP64 oracle (per mode and over the whole gradient)
GRAD_ELEM_RTOL = 1e-4   # element-wise against the sum of |contributions| of that element
BF16_RTOL = 1e-2        # BF16-stored factors vs the oracle at the FP32 factors
LOSS_RTOL = 2e-6        # F-hat against the sum of |terms|


def gcp():
    from paper_1906_01687_gb300 import gcp as g
    return g


def rng_factors(dims, rank, seed, scale=1.0, positive=False):
    r = np.random.default_rng(seed)
    if positive:
        return [(scale * r.random((n, rank))).astype(np.float32) for n in dims]
    return [(scale * r.standard_normal((n, rank))).astype(np.float32) for n in dims]


def f64(mats):
    """FP64 copies of FP32 factor matrices: the oracle sees the same values."""
    return [np.asarray(a, dtype=np.float32).astype(np.float64) for a in mats]


def sparse_random(dims, nnz, seed, binary=False):
    """Unique random positions (SoA int32) and values 1 + Poisson(2) (or None)."""
    r = np.random.default_rng(seed)
    omega = math.prod(dims)
    keys = np.unique(r.integers(0, omega, int(nnz * 1.3) + 16))
    keys = r.permutation(keys)[:nnz]
    idx = []
    rem = keys.copy()
    for n in reversed(dims):
        idx.append((rem % n).astype(np.int32))
        rem //= n
    idx = idx[::-1]
    vals = None if binary else (1 + r.poisson(2.0, len(keys))).astype(np.float32)
    return idx, vals


def oracle_sparse(dims, idx, vals):
    return oracle.Tensor(dims, coo=np.stack([np.asarray(i, np.int64) for i in idx], axis=1),
                         vals=None if vals is None else np.asarray(vals, np.float64))


def list_to_oracle(L):
    """A device SampleList as an oracle.Samples (same values, FP64)."""
    idx = np.stack([i.cpu().numpy().astype(np.int64) for i in L.idx], axis=1)
    return oracle.Samples(idx, L.x.double().cpu().numpy(), L.w.double().cpu().numpy(), L.cls.cpu().numpy())


def assert_lists_equal(L, S):
    """Bit-exact sample lists: indices and classes equal, x and w equal the
    oracle's values rounded once to FP32."""
    assert L.n == S.n
    got_idx = np.stack([i.cpu().numpy().astype(np.int64) for i in L.idx], axis=1) if L.n else np.zeros((0, S.idx.shape[1]))
    np.testing.assert_array_equal(got_idx, S.idx)
    np.testing.assert_array_equal(L.cls.cpu().numpy(), S.cls)
    np.testing.assert_array_equal(L.x.cpu().numpy(), S.x.astype(np.float32))
    np.testing.assert_array_equal(L.w.cpu().numpy(), S.w.astype(np.float32))


def grad_to_numpy(G, rank):
    return [g[:, :rank].double().cpu().numpy() for g in G]


def assert_pads_zero(G, rank):
    for g in G:
        if g.shape[1] > rank:
            assert torch.count_nonzero(g[:, rank:]).item() == 0


def assert_grad_close(G_gpu, G_orc, Gabs=None, rtol=GRAD_RTOL, elem_rtol=GRAD_ELEM_RTOL):
    """Norm-wise relative error <= rtol per mode and overall; with Gabs,
    element-wise |diff| <= elem_rtol * Gabs + tiny."""
    num = den = 0.0
    for k, (a, b) in enumerate(zip(G_gpu, G_orc)):
        dn = np.linalg.norm(a - b)
        bn = np.linalg.norm(b)
        num += dn * dn
        den += bn * bn
        assert dn <= rtol * bn + 1e-30, f"mode {k}: rel err {dn / max(bn, 1e-300):.3e}"
        if Gabs is not None:
            scale = Gabs[k]
            bound = elem_rtol * scale + 1e-12 * (scale.max() if scale.size else 0.0)
            bad = np.abs(a - b) > bound
            assert not bad.any(), f"mode {k}: {bad.sum()} elements beyond elementwise bound"
    assert math.sqrt(num) <= rtol * math.sqrt(den) + 1e-30


def rel_norm(G_gpu, G_orc):
    num = sum(np.linalg.norm(a - b) ** 2 for a, b in zip(G_gpu, G_orc))
    den = sum(np.linalg.norm(b) ** 2 for b in G_orc)
    return math.sqrt(num / den) if den > 0 else math.sqrt(num)
