"""Stratified zeros made inside the gradient launch (gcp_tuning.zero_pass = 0,
the default for the group walk of 3 or 4 modes) against the FP64 oracle and
against the separate ordered pass that lists them first (zero_pass = 1).

Alg. 2 keeps the first q accepted candidates in candidate order; the launch
finds them with tiles of one block each (decoupled look-back, bounded waits)
and walks them without writing a list, so the kept set -- and the gradient,
up to the FP32 summation order -- must be the oracle's.  Covered: block sizes
from one warp to 256 threads (many tiles, a ragged last tile), every layout
the walk has, BF16 rows, the continuation past the first batch, a shortfall,
draw ranges that cut through the zeros, the observed-entry sampler (Section
4.4) and back-to-back launches (the tile words and counters reset).
"""
import numpy as np
import pytest

import oracle
from gpu_util import (BF16_RTOL, assert_grad_close, f64, gcp, grad_to_numpy, oracle_sparse, rel_norm, rng_factors,
                      sparse_random)

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1906_01687_gb300 import build
    build.build()


def grad(h, F, loss, S, **tuning):
    g = gcp()
    g.gcp_set_tuning(h, **tuning)
    G = F.like()
    g.gcp_grad(h, F, loss, G, S=S)
    torch.cuda.synchronize()
    status = g.gcp_get_device_status(h)
    g.gcp_set_tuning(h, reset=True)
    return G, status


@pytest.mark.parametrize("dims,nnz,rank", [((40, 30, 20), 1200, 8), ((30, 20, 10, 8), 2400, 10),
                                           ((300, 40, 25), 5000, 32), ((70000, 70000, 2), 3000, 5)])
@pytest.mark.parametrize("block", [32, 128, 256])
def test_zero_tiles_match_the_oracle_and_the_separate_pass(dims, nnz, rank, block):
    g = gcp()
    idx, vals = sparse_random(dims, nnz, 21, binary=False)
    h = g.Handle(g.DataTensor.coo(dims, idx, vals))
    XO = oracle_sparse(dims, idx, vals)
    A = rng_factors(dims, rank, 22, scale=(0.5 / rank) ** (1 / len(dims)))
    F = g.Factors(A)
    p, q = 1500, 2300
    S = g.Sampling(g.SAMPLER_STRATIFIED, p, q, seed=31, stream=4)
    assert g.gcp_get_launch(h, F, p + q)["zero_tiles"] == 1
    SO = oracle.sample(XO, oracle.STRATIFIED, p, q, 31, 4)
    ref = oracle.grad(dims, f64(A), oracle.POISSON_LOG, SO)
    gabs = oracle.grad_abs(dims, f64(A), oracle.POISSON_LOG, SO)
    G0, st0 = grad(h, F, g.LOSS_POISSON_LOG, S, block=block)
    G1, st1 = grad(h, F, g.LOSS_POISSON_LOG, S, block=block, zero_pass=1)
    assert st0 == 0 and st1 == 0
    assert_grad_close(grad_to_numpy(G0, rank), ref, gabs)
    assert_grad_close(grad_to_numpy(G0, rank), grad_to_numpy(G1, rank), rtol=1e-6)


def test_every_walk_shape_with_zero_tiles():
    """Each compiled (lanes, chunks) pair and accumulation option of the group
    walk, with the zeros made in the launch, gives the oracle's gradient."""
    g = gcp()
    dims = (35, 28, 22)
    idx, vals = sparse_random(dims, 2500, 23)
    h = g.Handle(g.DataTensor.coo(dims, idx, vals))
    XO = oracle_sparse(dims, idx, vals)
    S = g.Sampling(g.SAMPLER_STRATIFIED, 2100, 2900, seed=7, stream=2)
    SO = oracle.sample(XO, oracle.STRATIFIED, 2100, 2900, 7, 2)
    for rank, shapes in [(3, [(1, 1), (1, 2), (4, 1), (32, 1)]), (10, [(1, 3), (1, 4), (4, 1), (2, 2), (16, 1)]),
                         (32, [(8, 1), (4, 2), (32, 2)])]:
        A = rng_factors(dims, rank, 24, scale=0.4)
        F = g.Factors(A)
        ref = oracle.grad(dims, f64(A), oracle.GAUSSIAN, SO)
        for lanes, chunks in shapes:
            for acc in (dict(), dict(max_replicas=0), dict(max_replicas=8, replica_target=1), dict(group_draws=1),
                        dict(max_replicas=0, smem_bytes=65536, smem_min_hits=0), dict(grid_blocks=3)):
                G, st = grad(h, F, g.LOSS_GAUSSIAN, S, lanes=lanes, chunks=chunks, **acc)
                assert st == 0
                assert_grad_close(grad_to_numpy(G, rank), ref)


def test_zero_tiles_bf16_rows():
    g = gcp()
    dims = (30, 20, 10, 8)
    idx, vals = sparse_random(dims, 2400, 25, binary=True)
    h = g.Handle(g.DataTensor.coo(dims, idx, None))
    XO = oracle_sparse(dims, idx, None)
    A = rng_factors(dims, 12, 26, scale=0.6)
    F = g.Factors(A, bf16=True)
    S = g.Sampling(g.SAMPLER_STRATIFIED, 1800, 2200, seed=9, stream=5)
    SO = oracle.sample(XO, oracle.STRATIFIED, 1800, 2200, 9, 5)
    A_bf = [a.float()[:, :12].double().cpu().numpy() for a in F.A_bf16]
    G, st = grad(h, F, g.LOSS_BERNOULLI_LOGIT, S)
    assert st == 0
    got = grad_to_numpy(G, 12)
    assert_grad_close(got, oracle.grad(dims, A_bf, oracle.BERNOULLI_LOGIT, SO))
    assert rel_norm(got, oracle.grad(dims, f64(A), oracle.BERNOULLI_LOGIT, SO)) <= BF16_RTOL


@pytest.mark.parametrize("block", [32, 256])
def test_zero_tiles_continue_past_the_first_batch(block):
    """60% of the entries are nonzeros and rho = 0.5: the tiles accept fewer
    than q and the last tile's block continues in candidate order; the kept
    zeros are the oracle's."""
    g = gcp()
    dims = (16, 16, 16)
    idx, vals = sparse_random(dims, int(0.6 * 4096), 3)
    h = g.Handle(g.DataTensor.coo(dims, idx, vals))
    XO = oracle_sparse(dims, idx, vals)
    A = rng_factors(dims, 6, 27, scale=0.5)
    F = g.Factors(A)
    S = g.Sampling(g.SAMPLER_STRATIFIED, 100, 3000, seed=5, stream=1, oversample=0.5)
    SO = oracle.sample(XO, oracle.STRATIFIED, 100, 3000, 5, 1, rho=0.5)
    assert SO.candidates_used > 0.5 * 3000 * 4096 / (4096 - len(vals))  # the oracle went past the first batch
    G, st = grad(h, F, g.LOSS_POISSON_LOG, S, block=block)
    assert st == 0
    assert_grad_close(grad_to_numpy(G, 6), oracle.grad(dims, f64(A), oracle.POISSON_LOG, SO),
                      oracle.grad_abs(dims, f64(A), oracle.POISSON_LOG, SO))


def test_zero_tiles_report_a_shortfall():
    """One zero entry and a tiny rho: the launch reports the shortfall and
    its gradient equals the separate pass's (the same kept zeros)."""
    g = gcp()
    dims = (4, 4, 4)
    all_idx = [c for c in np.ndindex(*dims) if c != (1, 2, 3)]
    idx = [np.array([c[k] for c in all_idx], np.int32) for k in range(3)]
    h = g.Handle(g.DataTensor.coo(dims, idx, None))
    F = g.Factors(rng_factors(dims, 4, 28, scale=0.5))
    S = g.Sampling(g.SAMPLER_STRATIFIED, 1, 50, seed=1, stream=0, oversample=0.01)
    G0, st0 = grad(h, F, g.LOSS_BERNOULLI_LOGIT, S)
    G1, st1 = grad(h, F, g.LOSS_BERNOULLI_LOGIT, S, zero_pass=1)
    assert st0 == g.ERR_SAMPLE_SHORTFALL and st1 == g.ERR_SAMPLE_SHORTFALL
    assert_grad_close(grad_to_numpy(G0, 4), grad_to_numpy(G1, 4), rtol=1e-6)


def test_zero_tiles_in_draw_ranges():
    """Ranges that start, end or lie inside the zeros: each equals the
    oracle on the same slice of its list."""
    g = gcp()
    dims = (60, 50, 40)
    idx, vals = sparse_random(dims, 4000, 29)
    h = g.Handle(g.DataTensor.coo(dims, idx, vals))
    XO = oracle_sparse(dims, idx, vals)
    A = rng_factors(dims, 7, 30, scale=0.3)
    F = g.Factors(A)
    p, q = 3001, 4003
    S = g.Sampling(g.SAMPLER_STRATIFIED, p, q, seed=77, stream=6)
    SO = oracle.sample(XO, oracle.STRATIFIED, p, q, 77, 6)
    for first, count in ((p - 700, 1500), (p, q), (p + 1, 1), (p + 999, 2000), (p + q - 37, 37), (0, p + q)):
        G = F.like()
        g.gcp_grad_range(h, F, g.LOSS_POISSON_LOG, G, S, first, count)
        torch.cuda.synchronize()
        assert g.gcp_get_device_status(h) == 0
        sl = slice(first, first + count)
        part = oracle.Samples(SO.idx[sl], SO.x[sl], SO.w[sl], SO.cls[sl])
        assert_grad_close(grad_to_numpy(G, 7), oracle.grad(dims, f64(A), oracle.POISSON_LOG, part),
                          oracle.grad_abs(dims, f64(A), oracle.POISSON_LOG, part))


def test_observed_entries_made_in_the_launch():
    """Section 4.4's sampler over a dense tensor with missing entries: the
    observed entries picked inside the launch are the oracle's."""
    g = gcp()
    dims = (22, 17, 13)
    r = np.random.default_rng(31)
    X = r.standard_normal(dims).astype(np.float32)
    v = (r.random(dims) >= 0.3).astype(np.float32)
    h = g.Handle(g.DataTensor.dense(X, weights=v))
    XO = oracle.Tensor(dims, dense=X.astype(np.float64), weights=v.astype(np.float64))
    A = rng_factors(dims, 5, 32, scale=0.5)
    F = g.Factors(A)
    S = g.Sampling(g.SAMPLER_OBSERVED, 0, 3001, seed=8, stream=3)
    SO = oracle.sample(XO, oracle.OBSERVED, 0, 3001, 8, 3)
    ref = oracle.grad(dims, f64(A), oracle.GAUSSIAN, SO)
    G0, st0 = grad(h, F, g.LOSS_GAUSSIAN, S)
    G1, st1 = grad(h, F, g.LOSS_GAUSSIAN, S, zero_pass=1)
    assert st0 == 0 and st1 == 0
    assert_grad_close(grad_to_numpy(G0, 5), ref, oracle.grad_abs(dims, f64(A), oracle.GAUSSIAN, SO))
    assert_grad_close(grad_to_numpy(G0, 5), grad_to_numpy(G1, 5), rtol=1e-6)


def test_back_to_back_launches_reset_the_tiles():
    """Launches queued one after another (different iterations, one stream,
    no host sync between them): each is the oracle's gradient for its own
    stream, so every launch found its tile words and counters cleared."""
    g = gcp()
    dims = (40, 30, 20)
    idx, vals = sparse_random(dims, 1500, 33)
    h = g.Handle(g.DataTensor.coo(dims, idx, vals))
    XO = oracle_sparse(dims, idx, vals)
    A = rng_factors(dims, 9, 34, scale=0.5)
    F = g.Factors(A)
    outs = []
    for it in range(6):
        G = F.like()
        g.gcp_grad(h, F, g.LOSS_POISSON_LOG, G, S=g.Sampling(g.SAMPLER_STRATIFIED, 900, 1300, seed=3, stream=it))
        outs.append(G)
    torch.cuda.synchronize()
    assert g.gcp_get_device_status(h) == 0
    for it, G in enumerate(outs):
        SO = oracle.sample(XO, oracle.STRATIFIED, 900, 1300, 3, it)
        assert_grad_close(grad_to_numpy(G, 9), oracle.grad(dims, f64(A), oracle.POISSON_LOG, SO),
                          oracle.grad_abs(dims, f64(A), oracle.POISSON_LOG, SO))


def test_five_modes_keep_the_separate_pass():
    """Layout 3 exists for 3 and 4 modes; 5 modes list the zeros first."""
    g = gcp()
    dims = (9, 8, 7, 6, 5)
    idx, vals = sparse_random(dims, 700, 35)
    h = g.Handle(g.DataTensor.coo(dims, idx, vals))
    F = g.Factors(rng_factors(dims, 4, 36, scale=0.5))
    assert g.gcp_get_launch(h, F, 2000)["zero_tiles"] == 0
    h3 = g.Handle(g.DataTensor.coo((40, 30, 20), *sparse_random((40, 30, 20), 1000, 37)))
    F3 = g.Factors(rng_factors((40, 30, 20), 4, 38))
    assert g.gcp_get_launch(h3, F3, 2000)["zero_tiles"] == 1
    g.gcp_set_tuning(h3, zero_pass=1)
    assert g.gcp_get_launch(h3, F3, 2000)["zero_tiles"] == 0
    g.gcp_set_tuning(h3, prefetch=2)
    assert g.gcp_get_launch(h3, F3, 2000)["zero_tiles"] == 0
