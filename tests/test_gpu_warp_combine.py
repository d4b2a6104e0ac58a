"""Warp-level pre-reduction of row updates (gcp_tuning.warp_combine): within
one step of the group walk, the groups whose draws share row i_k of a short
mode sum their updates to each 16-byte chunk of G_k (a match on row and
chunk, then shuffles) and one lane issues the L2 reduction.  Only the
summation order changes, so every shape must still give the FP64 oracle's
sampled gradient (the MTTKRP of Eq. (4.3) over the draws of Algs. 1-3), with
and without the stratified zeros made in the launch, replica slabs and group
draws.
"""
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
    from paper_1906_01687_gb300 import build
    build.build()


def grad(h, F, loss, S, **tuning):
    g = gcp()
    g.gcp_set_tuning(h, **tuning)
    launch = g.gcp_get_launch(h, F, S.count())
    G = F.like()
    g.gcp_grad(h, F, loss, G, S=S)
    torch.cuda.synchronize()
    status = g.gcp_get_device_status(h)
    g.gcp_set_tuning(h, reset=True)
    return G, status, launch


def test_combined_updates_on_short_modes_dense():
    """Modes of 3, 4 and 500 rows, 20,011 uniform draws: in every warp step
    many groups hit the same rows of the two short modes."""
    g = gcp()
    dims = (3, 4, 500)
    X = np.random.default_rng(40).standard_normal(dims).astype(np.float32)
    h = g.Handle(g.DataTensor.dense(X))
    XO = oracle.Tensor(dims, dense=X.astype(np.float64))
    S = g.Sampling(g.SAMPLER_UNIFORM, 0, 20_011, seed=5, stream=1)
    SO = oracle.sample(XO, oracle.UNIFORM, 0, 20_011, 5, 1)
    for rank, shapes in [(3, [(1, 1), (2, 1), (4, 1)]), (10, [(4, 1), (2, 2), (1, 3), (8, 1)]),
                         (32, [(8, 1), (4, 2), (32, 1)])]:
        A = rng_factors(dims, rank, 41, scale=0.5)
        F = g.Factors(A)
        ref = oracle.grad(dims, f64(A), oracle.GAUSSIAN, SO)
        gabs = oracle.grad_abs(dims, f64(A), oracle.GAUSSIAN, SO)
        for lanes, chunks in shapes:
            for acc in (dict(), dict(max_replicas=0), dict(group_draws=1), dict(group_draws=1, max_replicas=0),
                        dict(grid_blocks=2)):
                G, st, launch = grad(h, F, g.LOSS_GAUSSIAN, S, lanes=lanes, chunks=chunks, warp_combine=100, **acc)
                assert st == 0
                assert launch["combine_mode_mask"] == 0b011  # the 3- and 4-row modes, not the 500-row one
                assert_grad_close(grad_to_numpy(G, rank), ref, gabs)


def test_combined_updates_with_zero_tiles_and_bf16():
    """Stratified sampling of a count tensor with short modes: the zeros made
    in the launch and the combine together, FP32 and BF16 rows, against the
    oracle on the same draws (at the factors the kernel reads)."""
    g = gcp()
    dims = (400, 6, 9, 5)
    idx, vals = sparse_random(dims, 9000, 42)
    h = g.Handle(g.DataTensor.coo(dims, idx, vals))
    XO = oracle_sparse(dims, idx, vals)
    A = rng_factors(dims, 10, 43, scale=0.4, positive=True)
    S = g.Sampling(g.SAMPLER_STRATIFIED, 6000, 7000, seed=9, stream=2)
    SO = oracle.sample(XO, oracle.STRATIFIED, 6000, 7000, 9, 2)
    for bf16 in (False, True):
        F = g.Factors(A, bf16=bf16)
        Ar = [a.float()[:, :10].double().cpu().numpy() for a in F.A_bf16] if bf16 else f64(A)
        ref = oracle.grad(dims, Ar, oracle.POISSON_LOG, SO)
        gabs = oracle.grad_abs(dims, Ar, oracle.POISSON_LOG, SO)
        for acc in (dict(), dict(max_replicas=0), dict(block=32), dict(zero_pass=1), dict(group_draws=1)):
            G, st, launch = grad(h, F, g.LOSS_POISSON_LOG, S, lanes=4, chunks=1, warp_combine=4096, **acc)
            assert st == 0
            assert launch["combine_mode_mask"] == 0b1111
            assert launch["zero_tiles"] == (0 if acc.get("zero_pass") else 1)
            assert_grad_close(grad_to_numpy(G, 10), ref, gabs)


def test_combine_leaves_shared_memory_modes_alone():
    """A mode accumulated in shared memory is not also combined."""
    g = gcp()
    dims = (25, 30, 35)
    X = np.random.default_rng(44).standard_normal(dims).astype(np.float32)
    h = g.Handle(g.DataTensor.dense(X))
    XO = oracle.Tensor(dims, dense=X.astype(np.float64))
    A = rng_factors(dims, 8, 45, scale=0.5)
    F = g.Factors(A)
    S = g.Sampling(g.SAMPLER_UNIFORM, 0, 5003, seed=3, stream=1)
    SO = oracle.sample(XO, oracle.UNIFORM, 0, 5003, 3, 1)
    G, st, launch = grad(h, F, g.LOSS_GAUSSIAN, S, lanes=2, chunks=1, warp_combine=4096, max_replicas=0,
                         smem_bytes=65536, smem_min_hits=0)
    assert st == 0
    assert launch["combine_mode_mask"] & launch["smem_mode_mask"] == 0
    assert launch["combine_mode_mask"] | launch["smem_mode_mask"] == 0b111
    assert_grad_close(grad_to_numpy(G, 8), oracle.grad(dims, f64(A), oracle.GAUSSIAN, SO))
