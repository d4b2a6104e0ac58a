"""The fold of replica slabs in gcp_grad: by a launch of its own
(tail_work = 0) or by the gradient kernel's last blocks to finish
(tail_work = 1, where at most 64 blocks suffice; a completion counter and a
bounded wait).  Either way G_k must be the FP64 oracle's sampled
gradient (Eq. (4.3)) and the slabs must be left zero for the next call, so
calls queued back to back give each its own gradient.
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


@pytest.mark.parametrize("tail_work", [0, 1])
@pytest.mark.parametrize("dims,rank", [((40, 30, 20), 8),      # 90 rows x 2 float4
                                       ((3000, 40, 30), 8),    # 6140 float4 elements
                                       ((12, 10, 9, 11), 32)])  # 42 rows x 8 float4, 4 modes
def test_replicated_gradient_queued_back_to_back(dims, rank, tail_work):
    g = gcp()
    X = np.random.default_rng(50).standard_normal(dims).astype(np.float32)
    h = g.Handle(g.DataTensor.dense(X))
    XO = oracle.Tensor(dims, dense=X.astype(np.float64))
    A = rng_factors(dims, rank, 51, scale=0.5)
    F = g.Factors(A)
    g.gcp_set_tuning(h, max_replicas=8, replica_target=1, tail_work=tail_work)
    assert all(r > 1 for r in g.gcp_get_launch(h, F, 7001)["replicas"])
    outs = []
    for it in range(5):
        G = F.like()
        g.gcp_grad(h, F, g.LOSS_GAUSSIAN, G, S=g.Sampling(g.SAMPLER_UNIFORM, 0, 7001, seed=4, stream=it))
        outs.append(G)
    torch.cuda.synchronize()
    assert g.gcp_get_device_status(h) == 0
    for it, G in enumerate(outs):
        SO = oracle.sample(XO, oracle.UNIFORM, 0, 7001, 4, it)
        assert_grad_close(grad_to_numpy(G, rank), oracle.grad(dims, f64(A), oracle.GAUSSIAN, SO),
                          oracle.grad_abs(dims, f64(A), oracle.GAUSSIAN, SO))


@pytest.mark.parametrize("tail_work", [0, 1])
def test_replicated_stratified_gradient_with_zero_tiles(tail_work):
    """The count-like case: short replicated modes, zeros made in the launch,
    the fold done by the last block."""
    g = gcp()
    dims = (600, 24, 7, 32)
    idx, vals = sparse_random(dims, 20000, 52)
    h = g.Handle(g.DataTensor.coo(dims, idx, vals))
    XO = oracle_sparse(dims, idx, vals)
    A = rng_factors(dims, 10, 53, scale=0.4, positive=True)
    F = g.Factors(A)
    g.gcp_set_tuning(h, max_replicas=32, replica_target=16, tail_work=tail_work)
    S = g.Sampling(g.SAMPLER_STRATIFIED, 8000, 9000, seed=6, stream=3)
    G = F.like()
    g.gcp_grad(h, F, g.LOSS_POISSON_LOG, G, S=S)
    torch.cuda.synchronize()
    assert g.gcp_get_device_status(h) == 0
    SO = oracle.sample(XO, oracle.STRATIFIED, 8000, 9000, 6, 3)
    assert_grad_close(grad_to_numpy(G, 10), oracle.grad(dims, f64(A), oracle.POISSON_LOG, SO),
                      oracle.grad_abs(dims, f64(A), oracle.POISSON_LOG, SO))
