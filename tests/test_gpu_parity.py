"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Sample lists must match bit for bit; gradients within 1e-5 norm-wise
relative error (FP32) plus an element-wise bound against each element's sum
of |contributions|; loss estimates within 2e-6 of the sum of |terms|.
Sizes span several warps and CTAs with ragged tails.
"""
import math

import numpy as np
import pytest

import oracle
from gpu_util import (GRAD_RTOL, LOSS_RTOL, assert_grad_close, assert_lists_equal, assert_pads_zero, f64, gcp,
                      grad_to_numpy, list_to_oracle, oracle_sparse, rng_factors, sparse_random)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
LOSS_IDS = {0: "gaussian", 1: "logit", 2: "poisson"}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1906_01687_gb300 import build
    build.build()


def dense_case(dims, seed):
    X = np.random.default_rng(seed).standard_normal(dims).astype(np.float32)
    g = gcp()
    return X, g.DataTensor.dense(X), oracle.Tensor(dims, dense=X.astype(np.float64))


def run_grad(h, F, loss, S=None, samples=None):
    g = gcp()
    G = F.like()
    g.gcp_grad(h, F, loss, G, S=S, samples=samples)
    torch.cuda.synchronize()
    assert g.gcp_get_device_status(h) == 0
    return G


# ---------------------------------------------------------------------------
# sample lists: bit-exact
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dims", [(20, 30, 40), (12, 10, 9, 11), (7, 6, 5, 4, 3), (50, 60), (1, 17, 5)])
@pytest.mark.parametrize("stream", [0, 7, 2**64 - 1])
def test_uniform_sample_list_bit_exact(dims, stream):
    g = gcp()
    X, XT, XO = dense_case(dims, 1)
    h = g.Handle(XT)
    S = g.Sampling(g.SAMPLER_UNIFORM, 0, 3001, seed=1687, stream=stream)
    L = g.gcp_sample(h, S)
    torch.cuda.synchronize()
    assert_lists_equal(L, oracle.sample(XO, oracle.UNIFORM, 0, 3001, 1687, stream))


@pytest.mark.parametrize("kind", ["stratified", "semi_stratified"])
@pytest.mark.parametrize("dims,nnz,binary", [((40, 30, 20), 1200, False), ((30, 20, 10, 8), 2400, True),
                                             ((9, 8, 7, 6, 5), 700, False), ((200, 3), 30, False),
                                             ((70000, 70000, 2), 3000, False)])
def test_sparse_sample_list_bit_exact(kind, dims, nnz, binary):
    """Sample lists equal the oracle's bit for bit, also on a tensor whose
    linear keys exceed 32 bits (the last one, 9.8e9 entries)."""
    g = gcp()
    idx, vals = sparse_random(dims, nnz, 2, binary)
    h = g.Handle(g.DataTensor.coo(dims, idx, vals))
    XO = oracle_sparse(dims, idx, vals)
    for stream, (p, q) in [(3, (1500, 1700)), (4, (0, 999)), (5, (1001, 0)), (6, (1, 1))]:
        S = g.Sampling(g.SAMPLERS[kind], p, q, seed=99, stream=stream)
        L = g.gcp_sample(h, S)
        torch.cuda.synchronize()
        assert g.gcp_get_device_status(h) == 0
        assert_lists_equal(L, oracle.sample(XO, g.SAMPLERS[kind], p, q, 99, stream))


def test_stratified_continuation_past_first_batch():
    """A dense-ish tensor (60% nonzero) with a small oversample rate: the
    parallel pass falls short and the in-order continuation must produce the
    oracle's list exactly."""
    g = gcp()
    dims = (16, 16, 16)
    idx, vals = sparse_random(dims, int(0.6 * 4096), 3)
    h = g.Handle(g.DataTensor.coo(dims, idx, vals))
    XO = oracle_sparse(dims, idx, vals)
    S = g.Sampling(g.SAMPLER_STRATIFIED, 100, 3000, seed=5, stream=1, oversample=0.5)
    L = g.gcp_sample(h, S)
    torch.cuda.synchronize()
    assert g.gcp_get_device_status(h) == 0
    assert_lists_equal(L, oracle.sample(XO, oracle.STRATIFIED, 100, 3000, 5, 1, rho=0.5))


def test_stratified_shortfall_reported():
    """One zero entry only and a tiny rho: both sides report a shortfall."""
    g = gcp()
    dims = (4, 4, 4)
    all_idx = [c for c in np.ndindex(*dims) if c != (1, 2, 3)]
    idx = [np.array([c[k] for c in all_idx], np.int32) for k in range(3)]
    h = g.Handle(g.DataTensor.coo(dims, idx, None))
    S = g.Sampling(g.SAMPLER_STRATIFIED, 1, 50, seed=1, stream=0, oversample=0.01)
    L = g.gcp_sample(h, S)
    torch.cuda.synchronize()
    assert g.gcp_get_device_status(h) == g.ERR_SAMPLE_SHORTFALL
    XO = oracle_sparse(dims, idx, None)
    with pytest.raises(RuntimeError):
        oracle.sample(XO, oracle.STRATIFIED, 1, 50, 1, 0, rho=0.01)
    # the single zero can be drawn at most once per candidate; unfilled slots carry weight zero
    w = L.w.cpu().numpy()[1:]
    assert (w == 0).sum() >= 1 and np.all((w == 0) | (w == np.float32(1 / 50)))


# ---------------------------------------------------------------------------
# gradient: fused sampling and listed draws
# ---------------------------------------------------------------------------

DENSE_CASES = [((20, 30, 40), 3), ((12, 10, 9, 11), 10), ((7, 6, 5, 4, 3), 5), ((50, 60), 16),
               ((30, 20, 10), 32), ((30, 20, 10), 64), ((20, 20, 20), 100), ((16, 9, 7), 200), ((1, 17, 5), 8)]


@pytest.mark.parametrize("dims,rank", DENSE_CASES)
@pytest.mark.parametrize("loss", [0, 1, 2], ids=LOSS_IDS.get)
def test_dense_uniform_gradient(dims, rank, loss):
    g = gcp()
    X, XT, XO = dense_case(dims, 4)
    if loss == 1:
        X = (X > 0.5).astype(np.float32)
        XT, XO = g.DataTensor.dense(X), oracle.Tensor(dims, dense=X.astype(np.float64))
    elif loss == 2:
        X = np.floor(np.abs(X) * 2).astype(np.float32)
        XT, XO = g.DataTensor.dense(X), oracle.Tensor(dims, dense=X.astype(np.float64))
    h = g.Handle(XT)
    A = rng_factors(dims, rank, 5, scale=(0.5 / rank) ** (1 / len(dims)))
    F = g.Factors(A)
    S = g.Sampling(g.SAMPLER_UNIFORM, 0, 3001, seed=11, stream=2)
    G = run_grad(h, F, loss, S=S)
    assert_pads_zero(G, rank)
    SO = oracle.sample(XO, oracle.UNIFORM, 0, 3001, 11, 2)
    assert_grad_close(grad_to_numpy(G, rank), oracle.grad(dims, f64(A), loss, SO),
                      oracle.grad_abs(dims, f64(A), loss, SO))


@pytest.mark.parametrize("kind", ["stratified", "semi_stratified"])
@pytest.mark.parametrize("loss", [0, 1, 2], ids=LOSS_IDS.get)
@pytest.mark.parametrize("dims,nnz,rank", [((40, 30, 20), 1200, 8), ((30, 20, 10, 8), 2400, 10),
                                           ((9, 8, 7, 6, 5), 700, 4), ((300, 40, 25), 5000, 32)])
def test_sparse_gradient(kind, loss, dims, nnz, rank):
    g = gcp()
    idx, vals = sparse_random(dims, nnz, 6, binary=(loss == 1))
    h = g.Handle(g.DataTensor.coo(dims, idx, vals))
    XO = oracle_sparse(dims, idx, vals)
    A = rng_factors(dims, rank, 7, scale=(0.5 / rank) ** (1 / len(dims)))
    F = g.Factors(A)
    S = g.Sampling(g.SAMPLERS[kind], 1500, 1700, seed=13, stream=3)
    G = run_grad(h, F, loss, S=S)
    SO = oracle.sample(XO, g.SAMPLERS[kind], 1500, 1700, 13, 3)
    assert_grad_close(grad_to_numpy(G, rank), oracle.grad(dims, f64(A), loss, SO),
                      oracle.grad_abs(dims, f64(A), loss, SO))


def test_listed_draws_equal_fused_draws():
    """gcp_grad over a materialised list equals gcp_grad with in-kernel sampling."""
    g = gcp()
    dims = (40, 30, 20)
    idx, vals = sparse_random(dims, 1500, 8)
    h = g.Handle(g.DataTensor.coo(dims, idx, vals))
    A = rng_factors(dims, 12, 9, scale=0.6)
    F = g.Factors(A)
    for kind in (g.SAMPLER_STRATIFIED, g.SAMPLER_SEMI_STRATIFIED):
        S = g.Sampling(kind, 2000, 2500, seed=17, stream=8)
        G1 = run_grad(h, F, g.LOSS_POISSON_LOG, S=S)
        G2 = run_grad(h, F, g.LOSS_POISSON_LOG, samples=g.gcp_sample(h, S))
        assert_grad_close(grad_to_numpy(G1, 12), grad_to_numpy(G2, 12), rtol=1e-6)


@pytest.mark.parametrize("loss", [0, 1, 2], ids=LOSS_IDS.get)
def test_enumeration_identity_on_gpu(loss):
    """Every index of Omega once, weight 1: the GPU's sampled gradient is the
    full gradient G_k = Y_(k) Z_k of the oracle."""
    g = gcp()
    dims = (6, 7, 8)
    X = np.random.default_rng(10).standard_normal(dims).astype(np.float32)
    if loss != 0:
        X = (X > 0).astype(np.float32)
    h = g.Handle(g.DataTensor.dense(X))
    A = rng_factors(dims, 5, 11, scale=0.7)
    allix = np.array(list(np.ndindex(*dims)), dtype=np.int32)
    n = len(allix)
    L = g.SampleList([torch.tensor(allix[:, k], device="cuda") for k in range(3)],
                     torch.tensor(X.reshape(-1), device="cuda"), torch.ones(n, device="cuda"),
                     torch.zeros(n, dtype=torch.int8, device="cuda"))
    G = run_grad(h, g.Factors(A), loss, samples=L)
    Gf, _ = oracle.full_grad(dims, f64(A), loss, X.astype(np.float64))
    assert_grad_close(grad_to_numpy(G, 5), Gf)


def test_every_launch_shape_agrees():
    """Each compiled (lanes, chunks) shape and the shared-memory path give the
    same gradient (only the summation order differs)."""
    g = gcp()
    dims = (25, 30, 35)
    X, XT, XO = dense_case(dims, 12)
    h = g.Handle(XT)
    for rank, shapes in [(3, [(1, 1), (1, 2), (4, 1), (8, 1), (32, 1)]),
                         (10, [(1, 3), (1, 4), (4, 1), (2, 2), (4, 2), (8, 1), (16, 1), (32, 1)]),
                         (32, [(8, 1), (4, 2), (8, 2), (16, 1), (32, 1), (32, 2)])]:
        A = rng_factors(dims, rank, 13, scale=0.5)
        F = g.Factors(A)
        S = g.Sampling(g.SAMPLER_UNIFORM, 0, 5003, seed=3, stream=1)
        SO = oracle.sample(XO, oracle.UNIFORM, 0, 5003, 3, 1)
        ref = oracle.grad(dims, f64(A), 0, SO)
        for (lanes, chunks) in shapes:
            for acc in (dict(max_replicas=0), dict(), dict(max_replicas=8, replica_target=1),
                        dict(max_replicas=0, smem_bytes=65536, smem_min_hits=0), dict(group_draws=1),
                        dict(group_draws=1, max_replicas=0), dict(prefetch=1), dict(prefetch=1, max_replicas=0),
                        dict(prefetch=2), dict(prefetch=2, max_replicas=0)):
                for grid in (0, 3):
                    g.gcp_set_tuning(h, lanes=lanes, chunks=chunks, grid_blocks=grid, **acc)
                    G = run_grad(h, F, 0, S=S)
                    assert_grad_close(grad_to_numpy(G, rank), ref)
        g.gcp_set_tuning(h, reset=True)


def test_empty_draws_leave_gradient_untouched():
    g = gcp()
    dims = (5, 6, 7)
    X, XT, XO = dense_case(dims, 14)
    h = g.Handle(XT)
    F = g.Factors(rng_factors(dims, 4, 15))
    G = run_grad(h, F, 0, S=g.Sampling(g.SAMPLER_UNIFORM, 0, 0, seed=1))
    assert all(torch.count_nonzero(x).item() == 0 for x in G)


def test_invalid_arguments_rejected():
    g = gcp()
    dims = (5, 6, 7)
    X, XT, XO = dense_case(dims, 16)
    h = g.Handle(XT)
    F = g.Factors(rng_factors(dims, 4, 17))
    G = F.like()
    with pytest.raises(g.GcpError) as e:  # stratified needs a sparse tensor
        g.gcp_grad(h, F, 0, G, S=g.Sampling(g.SAMPLER_STRATIFIED, 5, 5, seed=1))
    assert e.value.status == g.ERR_INVALID_ARG
    with pytest.raises(g.GcpError):  # both a spec and a list
        g.gcp_grad(h, F, 0, G, S=g.Sampling(0, 0, 5, seed=1), samples=g.SampleList.empty(3, 5))
    with pytest.raises(g.GcpError):  # unaligned G
        g.gcp_grad(h, F, 0, [G[0].view(-1)[1:], G[1], G[2]], S=g.Sampling(0, 0, 5, seed=1))
    with pytest.raises(g.GcpError):  # unknown loss
        g.gcp_grad(h, F, 7, G, S=g.Sampling(0, 0, 5, seed=1))


# ---------------------------------------------------------------------------
# loss estimate
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kind", ["uniform", "stratified", "semi_stratified"])
@pytest.mark.parametrize("loss", [0, 1, 2], ids=LOSS_IDS.get)
def test_loss_estimate(kind, loss):
    g = gcp()
    if kind == "uniform":
        dims = (20, 30, 40)
        X, XT, XO = dense_case(dims, 18)
        h = g.Handle(XT)
        S = g.Sampling(g.SAMPLER_UNIFORM, 0, 20001, seed=19, stream=g.STREAM_EST)
        p, q = 0, 20001
    else:
        dims = (40, 30, 20, 6)
        idx, vals = sparse_random(dims, 9000, 20, binary=(loss == 1))
        h = g.Handle(g.DataTensor.coo(dims, idx, vals))
        XO = oracle_sparse(dims, idx, vals)
        S = g.Sampling(g.SAMPLERS[kind], 10001, 10002, seed=19, stream=g.STREAM_EST)
        p, q = 10001, 10002
    A = rng_factors(dims, 10, 21, scale=(0.5 / 10) ** (1 / len(dims)))
    F = g.Factors(A)
    L = g.gcp_sample(h, S)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    g.gcp_loss_est(h, F, loss, L, out)
    torch.cuda.synchronize()
    SO = oracle.sample(XO, g.SAMPLERS[kind], p, q, 19, g.STREAM_EST)
    ref = oracle.loss_estimate(dims, f64(A), loss, SO)
    scale = oracle.loss_abs(dims, f64(A), loss, SO)
    assert abs(out.item() - ref) <= LOSS_RTOL * scale
    # deterministic: the same list gives the same bits
    out2 = torch.zeros(1, dtype=torch.float64, device="cuda")
    g.gcp_loss_est(h, F, loss, L, out2)
    torch.cuda.synchronize()
    assert out2.item() == out.item()


def test_autotuner_keeps_results():
    """The autotuner picks a shape; the tuned gradient still matches the oracle."""
    from paper_1906_01687_gb300.autotune import autotune
    g = gcp()
    dims = (40, 50, 60)
    X, XT, XO = dense_case(dims, 22)
    h = g.Handle(XT)
    A = rng_factors(dims, 10, 23, scale=0.6)
    F = g.Factors(A)
    S = g.Sampling(g.SAMPLER_UNIFORM, 0, 20000, seed=2, stream=4)
    res = autotune(h, F, 0, S, launches=3)
    assert res["tried"] > 4 and res["seconds"] > 0
    G = run_grad(h, F, 0, S=S)
    SO = oracle.sample(XO, oracle.UNIFORM, 0, 20000, 2, 4)
    assert_grad_close(grad_to_numpy(G, 10), oracle.grad(dims, f64(A), 0, SO))


# ---------------------------------------------------------------------------
# the paper's odds / identity-link losses, on nonnegative models
# ---------------------------------------------------------------------------
POSITIVE = [3, 4, 5, 6]
POS_IDS = {3: "bernoulli_odds", 4: "poisson_identity", 5: "gamma", 6: "beta_half"}


@pytest.mark.parametrize("loss", POSITIVE, ids=POS_IDS.get)
@pytest.mark.parametrize("kind", ["uniform", "stratified", "semi_stratified"])
def test_positive_losses_gradient_and_estimate(loss, kind):
    g = gcp()
    rs = np.random.default_rng(30 + loss)
    rank = 6
    if kind == "uniform":
        dims = (20, 30, 40)
        X = rs.exponential(1.0, dims).astype(np.float32) if loss in (5, 6) else rs.poisson(1.0, dims).astype(np.float32)
        if loss == 3:
            X = (X > 0).astype(np.float32)
        h = g.Handle(g.DataTensor.dense(X))
        XO = oracle.Tensor(dims, dense=X.astype(np.float64))
        p, q = 0, 4001
    else:
        dims = (40, 30, 20, 6)
        idx, vals = sparse_random(dims, 6000, 31, binary=(loss == 3))
        h = g.Handle(g.DataTensor.coo(dims, idx, vals))
        XO = oracle_sparse(dims, idx, vals)
        p, q = 2001, 2002
    A = [(rs.uniform(0.2, 1.0, (n, rank)) * (1.0 / rank) ** (1 / len(dims))).astype(np.float32) for n in dims]
    F = g.Factors(A)
    S = g.Sampling(g.SAMPLERS[kind], p, q, seed=5, stream=2)
    G = run_grad(h, F, loss, S=S)
    SO = oracle.sample(XO, g.SAMPLERS[kind], p, q, 5, 2)
    assert_grad_close(grad_to_numpy(G, rank), oracle.grad(dims, f64(A), loss, SO),
                      oracle.grad_abs(dims, f64(A), loss, SO))
    L = g.gcp_sample(h, g.Sampling(g.SAMPLERS[kind], p, q, seed=6, stream=g.STREAM_EST))
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    g.gcp_loss_est(h, F, loss, L, out)
    torch.cuda.synchronize()
    SE = oracle.sample(XO, g.SAMPLERS[kind], p, q, 6, 2**64 - 1)
    assert abs(out.item() - oracle.loss_estimate(dims, f64(A), loss, SE)) <= \
        LOSS_RTOL * oracle.loss_abs(dims, f64(A), loss, SE)


# ---------------------------------------------------------------------------
# uniform sampling of a sparse tensor; entry weights (weighted GCP, Eq. (4.5))
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("loss", [0, 2], ids=LOSS_IDS.get)
def test_uniform_over_sparse_tensor(loss):
    g = gcp()
    dims = (40, 30, 20, 6)
    idx, vals = sparse_random(dims, 30000, 41)
    h = g.Handle(g.DataTensor.coo(dims, idx, vals))
    XO = oracle_sparse(dims, idx, vals)
    S = g.Sampling(g.SAMPLER_UNIFORM, 0, 20001, seed=8, stream=3)
    L = g.gcp_sample(h, S)
    torch.cuda.synchronize()
    SO = oracle.sample(XO, oracle.UNIFORM, 0, 20001, 8, 3)
    assert_lists_equal(L, SO)
    assert (SO.x != 0).sum() > 100  # the draws do hit nonzeros
    A = rng_factors(dims, 8, 42, scale=0.5)
    G = run_grad(h, g.Factors(A), loss, S=S)
    assert_grad_close(grad_to_numpy(G, 8), oracle.grad(dims, f64(A), loss, SO), oracle.grad_abs(dims, f64(A), loss, SO))


def test_entry_weights_dense():
    g = gcp()
    dims = (20, 30, 40)
    rs = np.random.default_rng(43)
    X = rs.standard_normal(dims).astype(np.float32)
    v = (rs.random(dims) * (rs.random(dims) < 0.7)).astype(np.float32)
    h = g.Handle(g.DataTensor.dense(X, weights=v))
    XO = oracle.Tensor(dims, dense=X.astype(np.float64), weights=v.astype(np.float64))
    S = g.Sampling(g.SAMPLER_UNIFORM, 0, 10001, seed=9, stream=4)
    L = g.gcp_sample(h, S)
    torch.cuda.synchronize()
    SO = oracle.sample(XO, oracle.UNIFORM, 0, 10001, 9, 4)
    np.testing.assert_array_equal(np.stack([i.cpu().numpy() for i in L.idx], axis=1), SO.idx)
    np.testing.assert_allclose(L.w.cpu().numpy(), SO.w, rtol=2e-7)  # (omega/s) v in FP32 vs FP64
    A = rng_factors(dims, 5, 44, scale=0.5)
    G = run_grad(h, g.Factors(A), g.LOSS_BERNOULLI_LOGIT, S=S)
    assert_grad_close(grad_to_numpy(G, 5), oracle.grad(dims, f64(A), oracle.BERNOULLI_LOGIT, SO))


# ---------------------------------------------------------------------------
# the full (non-stochastic) gradient and objective (Eqs. (1.2), (4.2), (4.5))
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("loss", [0, 1, 2, 5], ids={0: "gaussian", 1: "logit", 2: "poisson", 5: "gamma"}.get)
@pytest.mark.parametrize("weighted", [False, True])
def test_full_gradient_and_objective(loss, weighted):
    g = gcp()
    dims = (17, 23, 31)
    rs = np.random.default_rng(60 + loss)
    if loss == 5:
        A = [(rs.uniform(0.2, 1.0, (n, 6)) * 0.5).astype(np.float32) for n in dims]
        X = rs.exponential(1.0, dims).astype(np.float32)
    else:
        A = rng_factors(dims, 6, 61, scale=0.5)
        X = rs.standard_normal(dims).astype(np.float32)
        if loss == 1:
            X = (X > 0).astype(np.float32)
        elif loss == 2:
            X = np.floor(np.abs(X) * 2).astype(np.float32)
    v = (rs.random(dims) * (rs.random(dims) < 0.8)).astype(np.float32) if weighted else None
    h = g.Handle(g.DataTensor.dense(X, weights=v))
    F = g.Factors(A)
    G = F.like()
    g.gcp_full_grad(h, F, loss, G)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    g.gcp_full_loss(h, F, loss, out)
    torch.cuda.synchronize()
    Gref, Fref = oracle.full_grad(dims, f64(A), loss, X.astype(np.float64),
                                  weights=None if v is None else v.astype(np.float64))
    assert_grad_close(grad_to_numpy(G, 6), Gref)
    assert out.item() == pytest.approx(Fref, rel=2e-6)


# ---------------------------------------------------------------------------
# uniform draws over the entries of nonzero weight (Section 4.4)
# ---------------------------------------------------------------------------

def weighted_dense(dims, seed, missing):
    r = np.random.default_rng(seed)
    X = r.standard_normal(dims).astype(np.float32)
    v = ((0.5 + r.random(dims)) * (r.random(dims) >= missing)).astype(np.float32)
    return X, v


@pytest.mark.parametrize("dims,missing", [((20, 30, 40), 0.3), ((12, 10, 9, 11), 0.9), ((7, 6, 5, 4, 3), 0.5),
                                          ((50, 60), 0.0)])
def test_observed_sample_list_bit_exact(dims, missing):
    g = gcp()
    X, v = weighted_dense(dims, 31, missing)
    h = g.Handle(g.DataTensor.dense(X, weights=v))
    XO = oracle.Tensor(dims, dense=X.astype(np.float64), weights=v.astype(np.float64))
    for stream, q in [(3, 3001), (4, 1), (5, 20000)]:
        S = g.Sampling(g.SAMPLER_OBSERVED, 0, q, seed=77, stream=stream)
        L = g.gcp_sample(h, S)
        torch.cuda.synchronize()
        assert g.gcp_get_device_status(h) == 0
        SO = oracle.sample(XO, oracle.OBSERVED, 0, q, 77, stream)
        assert_lists_equal(L, SO)
        assert np.all(v[tuple(L.idx[k].cpu().numpy() for k in range(len(dims)))] != 0)


@pytest.mark.parametrize("loss", [0, 1, 2], ids=LOSS_IDS.get)
def test_observed_gradient(loss):
    g = gcp()
    dims, rank = (30, 25, 20), 8
    X, v = weighted_dense(dims, 32, 0.4)
    if loss == 1:
        X = (X > 0.5).astype(np.float32)
    elif loss == 2:
        X = np.floor(np.abs(X) * 2).astype(np.float32)
    h = g.Handle(g.DataTensor.dense(X, weights=v))
    XO = oracle.Tensor(dims, dense=X.astype(np.float64), weights=v.astype(np.float64))
    A = rng_factors(dims, rank, 33, scale=(0.5 / rank) ** (1 / 3))
    F = g.Factors(A)
    for stream in (0, 9):
        S = g.Sampling(g.SAMPLER_OBSERVED, 0, 5003, seed=19, stream=stream)
        G = run_grad(h, F, loss, S=S)
        SO = oracle.sample(XO, oracle.OBSERVED, 0, 5003, 19, stream)
        assert_grad_close(grad_to_numpy(G, rank), oracle.grad(dims, f64(A), loss, SO),
                          oracle.grad_abs(dims, f64(A), loss, SO))


def test_observed_sampler_rejections():
    """Arguments: observed sampling needs a dense tensor with weights and p = 0;
    a tensor with every entry missing is rejected; an almost empty observed
    set with a tiny oversampling rate reports the shortfall."""
    g = gcp()
    dims = (8, 8, 8)
    X = np.ones(dims, np.float32)
    with pytest.raises(g.GcpError):
        g.gcp_sample(g.Handle(g.DataTensor.dense(X)), g.Sampling(g.SAMPLER_OBSERVED, 0, 10, seed=1))
    v = np.zeros(dims, np.float32)
    h = g.Handle(g.DataTensor.dense(X, weights=v))
    with pytest.raises(g.GcpError):
        g.gcp_sample(h, g.Sampling(g.SAMPLER_OBSERVED, 0, 10, seed=1))
    v[1, 2, 3] = 1.0
    h = g.Handle(g.DataTensor.dense(X, weights=v))
    with pytest.raises(g.GcpError):
        g.gcp_sample(h, g.Sampling(g.SAMPLER_OBSERVED, 3, 10, seed=1))
    L = g.gcp_sample(h, g.Sampling(g.SAMPLER_OBSERVED, 0, 50, seed=1, oversample=0.01))
    torch.cuda.synchronize()
    assert g.gcp_get_device_status(h) == g.ERR_SAMPLE_SHORTFALL
    w = L.w.cpu().numpy()
    assert np.count_nonzero(w) >= 1 and np.all((w == 0) | (w == np.float32(1 / 50)))
