"""Early descriptors (gcp_tuning.early_draws): the gradient kernel draws its
first batch per warp before waiting on the preceding kernel.  The draws must
be exactly those of the spec: checked against the FP64 oracle for every
eligible source, through a device stream word whose prediction is right and
wrong, and over a run of GCP-Adam iterations against the waiting kernel."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_grad_close, f64, gcp, grad_to_numpy, oracle_sparse, rng_factors, sparse_random

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")


def grad(h, F, loss, S, stream_dev=None):
    g = gcp()
    G = F.like()
    g.gcp_grad(h, F, loss, G, S=S, stream_dev=stream_dev)
    torch.cuda.synchronize()
    assert g.gcp_get_device_status(h) == 0
    return G


@pytest.mark.parametrize("dims,rank", [((20, 30, 40), 10), ((12, 10, 9, 11), 10), ((7, 6, 5, 4, 3), 5),
                                       ((100, 100, 100, 100), 10)])
def test_dense_uniform_early_matches_oracle(dims, rank):
    g = gcp()
    X = np.random.default_rng(1).standard_normal(dims).astype(np.float32)
    h = g.Handle(g.DataTensor.dense(X))
    XO = oracle.Tensor(dims, dense=X.astype(np.float64))
    A = rng_factors(dims, rank, 2, scale=(0.5 / rank) ** (1 / len(dims)))
    F = g.Factors(A)
    S = g.Sampling(g.SAMPLER_UNIFORM, 0, 4099, seed=5, stream=9)
    SO = oracle.sample(XO, oracle.UNIFORM, 0, 4099, 5, 9)
    ref, ref_abs = oracle.grad(dims, f64(A), 0, SO), oracle.grad_abs(dims, f64(A), 0, SO)
    for extra in (dict(), dict(group_draws=1), dict(prefetch=1), dict(grid_blocks=3), dict(prefetch=2),
                  dict(prefetch=2, grid_blocks=3)):
        g.gcp_set_tuning(h, early_draws=1, **extra)
        assert g.gcp_get_launch(h, F, 4099)["early_draws"] == 1
        assert_grad_close(grad_to_numpy(grad(h, F, 0, S), rank), ref, ref_abs)


@pytest.mark.parametrize("kind", ["stratified", "semi_stratified", "uniform"])
def test_sparse_sources_early_match_oracle(kind):
    """Semi-stratified and uniform-over-sparse draws are made early (the
    latter once its nonzero table exists); stratified draws read the zero
    list of the same call and always wait."""
    g = gcp()
    dims, rank = (40, 30, 20, 9), 8
    idx, vals = sparse_random(dims, 3000, 3)
    h = g.Handle(g.DataTensor.coo(dims, idx, vals))
    XO = oracle_sparse(dims, idx, vals)
    A = rng_factors(dims, rank, 4, scale=(0.5 / rank) ** 0.25)
    F = g.Factors(A)
    p, q = (0, 5000) if kind == "uniform" else (2000, 2500)
    for layout in (0, 1, 2):  # the group walk, the prefetch layout and the staged walk
        g.gcp_set_tuning(h, early_draws=1, prefetch=layout)
        for stream in (1, 2):  # the first uniform call builds the table and waits; the second draws early
            S = g.Sampling(g.SAMPLERS[kind], p, q, seed=7, stream=stream)
            SO = oracle.sample(XO, g.SAMPLERS[kind], p, q, 7, stream)
            assert_grad_close(grad_to_numpy(grad(h, F, 2, S), rank), oracle.grad(dims, f64(A), 2, SO),
                              oracle.grad_abs(dims, f64(A), 2, SO))


def test_device_stream_word_prediction_hits_and_misses():
    """With stream_dev the kernel predicts the previous launch's stream + 1 and
    redraws when the word says otherwise: repeated, decreasing and far jumps
    all give the oracle's draws for the word's value."""
    g = gcp()
    dims, rank = (30, 25, 20, 15), 10
    X = np.random.default_rng(6).standard_normal(dims).astype(np.float32)
    h = g.Handle(g.DataTensor.dense(X))
    XO = oracle.Tensor(dims, dense=X.astype(np.float64))
    A = rng_factors(dims, rank, 7, scale=(0.5 / rank) ** 0.25)
    F = g.Factors(A)
    word = torch.zeros(1, dtype=torch.int64, device="cuda")
    for early, layout in ((0, 0), (1, 0), (1, 1), (1, 2)):
        g.gcp_set_tuning(h, early_draws=early, prefetch=layout)
        for v in (5, 6, 7, 7, 100, 3, 2**40, 2**40 + 1):
            word.fill_(v)
            S = g.Sampling(g.SAMPLER_UNIFORM, 0, 3000, seed=8, stream=12345)  # the host stream is ignored
            SO = oracle.sample(XO, oracle.UNIFORM, 0, 3000, 8, v)
            assert_grad_close(grad_to_numpy(grad(h, F, 0, S, stream_dev=word), rank),
                              oracle.grad(dims, f64(A), 0, SO), oracle.grad_abs(dims, f64(A), 0, SO))


@pytest.mark.parametrize("sampler", ["uniform", "semi_stratified", "stratified"])
def test_iterations_with_early_draws_follow_waiting_run(sampler):
    """Thirty GCP-Adam iterations drawing from the device iteration counter:
    early and waiting kernels take the same draws (with stratified sampling
    only the warps whose first batch is all nonzero draws start early), so
    the factors agree to FP32 summation-order noise and the counters match."""
    g = gcp()
    dims, rank = (40, 35, 30), 6
    if sampler == "uniform":
        X = np.random.default_rng(9).standard_normal(dims).astype(np.float32)
        T = g.DataTensor.dense(X)
        S = g.Sampling(g.SAMPLER_UNIFORM, 0, 20000, seed=3)
    else:
        idx, vals = sparse_random(dims, 4000, 9)
        T = g.DataTensor.coo(dims, idx, vals)
        S = g.Sampling(g.SAMPLERS[sampler], 6000, 6000, seed=3)
    A0 = rng_factors(dims, rank, 10, scale=0.5)
    out = {}
    for early, layout in ((0, 0), (1, 0), (1, 1), (1, 2)):
        h = g.Handle(T)
        g.gcp_set_tuning(h, early_draws=early, prefetch=layout)
        F = g.Factors(A0)
        G, B, C = F.like(), F.like(), F.like()
        st = g.new_state()
        g.gcp_state_init(st, 1e-3)
        for _ in range(30):
            g.gcp_iteration(h, F, 0, S, G, B, C, st, stream_dev=st[3:4])
        torch.cuda.synchronize()
        assert g.gcp_get_device_status(h) == 0
        out[(early, layout)] = (np.concatenate([a[:, :rank].double().cpu().numpy().ravel() for a in F.A]),
                                g.read_state(st))
    a0, s0 = out[(0, 0)]
    for key in ((1, 0), (1, 1), (1, 2)):
        a1, s1 = out[key]
        assert s0["iter"] == s1["iter"] == 30 and s0["t"] == s1["t"] == 30
        assert np.linalg.norm(a1 - a0) <= 1e-5 * np.linalg.norm(a0), key

