"""Draw ranges (gcp_grad_range), the sample-parallel GCP-Adam of
paper_1906_01687_gb300/parallel.py, and gcp_refresh, on one GPU.

Ranges are checked against the FP64 oracle on the same draws: the partial
gradients of a partition of the draw counter sum to the whole gradient.  The
ranks of a sample-parallel run are emulated one after another on the one GPU
(each rank's kernels run to completion before the next rank's start; nothing
waits on another rank), with the all-reduce replaced by a sum on the device.
"""
import numpy as np
import pytest

import oracle
from gpu_util import (GRAD_RTOL, assert_grad_close, assert_lists_equal, assert_pads_zero, f64, gcp, grad_to_numpy,
                      oracle_sparse, rel_norm, rng_factors, sparse_random)

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1906_01687_gb300 import build
    build.build()


def _cases():
    """(name, handle, oracle tensor, dims, rank, loss ids, spec args)"""
    g = gcp()
    out = []
    dims = (30, 25, 20, 9)
    X = np.random.default_rng(2).standard_normal(dims).astype(np.float32)
    out.append(("uniform-dense", g.Handle(g.DataTensor.dense(X)), oracle.Tensor(dims, dense=X.astype(np.float64)),
                dims, 10, (g.LOSS_GAUSSIAN, oracle.GAUSSIAN), (g.SAMPLER_UNIFORM, oracle.UNIFORM, 0, 20_011)))
    sdims = (60, 50, 40)
    idx, vals = sparse_random(sdims, 4000, 3)
    h = g.Handle(g.DataTensor.coo(sdims, idx, vals))
    XO = oracle_sparse(sdims, idx, vals)
    out.append(("stratified", h, XO, sdims, 7, (g.LOSS_POISSON_LOG, oracle.POISSON_LOG),
                (g.SAMPLER_STRATIFIED, oracle.STRATIFIED, 9_001, 11_003)))
    out.append(("semi", h, XO, sdims, 7, (g.LOSS_POISSON_LOG, oracle.POISSON_LOG),
                (g.SAMPLER_SEMI_STRATIFIED, oracle.SEMI_STRATIFIED, 9_001, 11_003)))
    return out


@pytest.mark.parametrize("world", [1, 2, 3, 7])
def test_grad_ranges_sum_to_the_whole_gradient(world):
    from paper_1906_01687_gb300.parallel import draw_range
    g = gcp()
    for name, h, XO, dims, rank, (loss, oloss), (kind, okind, p, q) in _cases():
        A = rng_factors(dims, rank, 11, scale=0.3)
        F = g.Factors(A)
        S = g.Sampling(kind, p, q, seed=1687, stream=5)
        total = F.like()
        for r in range(world):
            first, count = draw_range(r, world, S.count())
            part = F.like()
            g.gcp_grad_range(h, F, loss, part, S, first, count)
            for t, x in zip(total, part):
                t += x
        torch.cuda.synchronize()
        assert g.gcp_get_device_status(h) == 0, name
        assert_pads_zero(total, rank)
        SO = oracle.sample(XO, okind, p, q, 1687, 5)
        ref = oracle.grad(dims, f64(A), oloss, SO)
        gabs = oracle.grad_abs(dims, f64(A), oloss, SO)
        assert_grad_close(grad_to_numpy(total, rank), ref, gabs)


def test_grad_range_of_a_slice_equals_the_oracle_on_that_slice():
    g = gcp()
    name, h, XO, dims, rank, (loss, oloss), (kind, okind, p, q) = _cases()[1]
    A = rng_factors(dims, rank, 12, scale=0.3)
    F = g.Factors(A)
    S = g.Sampling(kind, p, q, seed=99, stream=1)
    SO = oracle.sample(XO, okind, p, q, 99, 1)
    for first, count in ((0, 1), (p - 5, 10), (p, q), (123, 4567), (p + q - 1, 1), (p + q, 0)):
        G = F.like()
        g.gcp_grad_range(h, F, loss, G, S, first, count)
        torch.cuda.synchronize()
        sl = slice(first, first + count)
        part = oracle.Samples(SO.idx[sl], SO.x[sl], SO.w[sl], SO.cls[sl])
        ref = oracle.grad(dims, f64(A), oloss, part)
        if count == 0:
            assert all(torch.count_nonzero(x).item() == 0 for x in G)
        else:
            assert_grad_close(grad_to_numpy(G, rank), ref, oracle.grad_abs(dims, f64(A), oloss, part))


def test_grad_range_rejects_ranges_outside_the_spec():
    g = gcp()
    name, h, XO, dims, rank, (loss, _), (kind, _, p, q) = _cases()[0]
    F = g.Factors(rng_factors(dims, rank, 1))
    G = F.like()
    S = g.Sampling(kind, p, q, seed=1)
    for first, count in ((-1, 5), (0, S.count() + 1), (S.count(), 1), (10, -1)):
        with pytest.raises(g.GcpError) as e:
            g.gcp_grad_range(h, F, loss, G, S, first, count)
        assert e.value.status == g.ERR_INVALID_ARG


def test_sample_parallel_single_rank_follows_gcp_adam():
    """With one rank the sample-parallel optimizer (gradient, no exchange,
    standalone Adam step) takes the steps of the fused GcpAdam path."""
    g = gcp()
    from paper_1906_01687_gb300 import synth
    from paper_1906_01687_gb300.adam import GcpAdam
    from paper_1906_01687_gb300.parallel import SampleParallelGcpAdam
    X = synth.dense_small()[0].astype(np.float32)
    A0 = synth.initial_guess(X.shape, 3, seed=1, target_norm=float(np.linalg.norm(X)))
    kw = dict(seed=1, est_seed=2, tau=25, alpha=1e-2)
    a = SampleParallelGcpAdam(g.DataTensor.dense(X), A0, g.LOSS_GAUSSIAN, g.SAMPLER_UNIFORM, 0, 1000, 0, 500, **kw)
    b = GcpAdam(g.DataTensor.dense(X), A0, g.LOSS_GAUSSIAN, g.SAMPLER_UNIFORM, 0, 1000, 0, 500, **kw)
    for _ in range(3):
        a.run_epoch()
        b.run_epoch()
    sa, sb = a.status(), b.status()
    assert (sa["t"], sa["iter"], sa["bad"]) == (sb["t"], sb["iter"], sb["bad"])
    assert rel_norm(a.factors(), b.factors()) <= 1e-4
    assert abs(sa["F"] - sb["F"]) <= 1e-4 * abs(sb["F"]) and sa["status"] == 0


def test_two_emulated_ranks_take_the_single_rank_steps():
    """Two ranks of one problem, emulated in turn on one GPU: each computes
    its draw range's gradient, the device sum stands in for the all-reduce,
    both take the Adam step.  Both ranks' factors stay equal to each other
    and follow the single-rank run (summation order aside)."""
    g = gcp()
    from paper_1906_01687_gb300.parallel import SampleParallelGcpAdam, draw_range
    dims = (60, 50, 40)
    idx, vals = sparse_random(dims, 4000, 8)
    A0 = rng_factors(dims, 6, 4, scale=0.4, positive=True)
    kw = dict(seed=5, est_seed=6, tau=10, alpha=1e-2)
    args = (g.LOSS_POISSON_LOG, g.SAMPLER_STRATIFIED, 3000, 5000, 2000, 2000)
    ranks = [SampleParallelGcpAdam(g.DataTensor.coo(dims, idx, vals), A0, *args, **kw) for _ in range(2)]
    for r, run in enumerate(ranks):  # the split a two-rank process group would give
        run.world, run.rank = 2, r
        run.first, run.count = draw_range(r, 2, run.spec.count())
    single = SampleParallelGcpAdam(g.DataTensor.coo(dims, idx, vals), A0, *args, **kw)
    for _ in range(20):
        for run in ranks:
            run.partial_gradient()
        torch.cuda.synchronize()
        total = ranks[0].G_flat + ranks[1].G_flat
        for run in ranks:
            run.G_flat.copy_(total)
            g.gcp_adam_step(run.F, run.G, run.B, run.C, run.state, stream=run.stream, **run.adam)
        single.iteration()
    torch.cuda.synchronize()
    f0, f1, fs = ranks[0].factors(), ranks[1].factors(), single.factors()
    assert rel_norm(f0, f1) == 0.0
    assert rel_norm(f0, fs) <= 1e-4
    for run in ranks + [single]:
        assert g.gcp_get_device_status(run.h) == 0


def test_refresh_takes_up_new_tensor_contents():
    """A COO tensor rewritten in place and refreshed gives the stratified
    draws and the gradients of a handle made fresh from the new contents."""
    g = gcp()
    dims = (40, 30, 20)
    idx1, vals1 = sparse_random(dims, 3000, 1)
    idx2, vals2 = sparse_random(dims, 3000, 2)
    XT = g.DataTensor.coo(dims, idx1, vals1)
    h = g.Handle(XT)
    F = g.Factors(rng_factors(dims, 5, 3, scale=0.5))
    S = g.Sampling(g.SAMPLER_STRATIFIED, 2000, 2500, seed=3, stream=0)
    g.gcp_sample(h, S)  # builds the nonzero-key hash of the first contents
    for dst, src in zip(XT.idx, idx2):
        dst.copy_(torch.as_tensor(src))
    XT.vals.copy_(torch.as_tensor(vals2))
    g.gcp_refresh(h)
    L = g.gcp_sample(h, S)
    G = F.like()
    g.gcp_grad(h, F, g.LOSS_POISSON_LOG, G, S=S)
    torch.cuda.synchronize()
    assert g.gcp_get_device_status(h) == 0
    XO = oracle_sparse(dims, idx2, vals2)
    SO = oracle.sample(XO, oracle.STRATIFIED, 2000, 2500, 3, 0)
    assert_lists_equal(L, SO)
    A = f64([a[:, :5].cpu().numpy() for a in F.A])
    assert_grad_close(grad_to_numpy(G, 5), oracle.grad(dims, A, oracle.POISSON_LOG, SO),
                      oracle.grad_abs(dims, A, oracle.POISSON_LOG, SO))


def test_refresh_recounts_the_observed_entries():
    """Entry weights rewritten in place (more entries missing) and refreshed:
    the observed-entry sampler counts |Omega_obs| again and draws the
    oracle's list for the new weights (weights (|Omega_obs| / q) v_i)."""
    g = gcp()
    dims = (20, 15, 12)
    r = np.random.default_rng(40)
    X = r.standard_normal(dims).astype(np.float32)
    v1 = (r.random(dims) >= 0.2).astype(np.float32)
    v2 = np.where(r.random(dims) >= 0.5, v1, 0.0).astype(np.float32)
    XT = g.DataTensor.dense(X, weights=v1)
    h = g.Handle(XT)
    S = g.Sampling(g.SAMPLER_OBSERVED, 0, 3001, seed=8, stream=2)
    g.gcp_sample(h, S)  # counts the entries of nonzero weight of v1
    XT.weights.copy_(torch.as_tensor(v2.reshape(-1)))
    g.gcp_refresh(h)
    L = g.gcp_sample(h, S)
    torch.cuda.synchronize()
    assert g.gcp_get_device_status(h) == 0
    XO = oracle.Tensor(dims, dense=X.astype(np.float64), weights=v2.astype(np.float64))
    assert_lists_equal(L, oracle.sample(XO, oracle.OBSERVED, 0, 3001, 8, 2))
