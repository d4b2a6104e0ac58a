"""Parity at the full sizes of the standard workloads, in the launch shape
the benchmark uses (automatic tuning).  The oracle checks the whole sample
list bit for bit and the whole gradient of one iteration (it finishes those
in seconds at these draw counts); BF16 forms are checked against the oracle
at the BF16-rounded factors (1e-5) and at the FP32 factors (1e-2).
"""
import math

import numpy as np
import pytest

import oracle
from gpu_util import (BF16_RTOL, assert_grad_close, assert_lists_equal, f64, gcp, grad_to_numpy, oracle_sparse,
                      rel_norm)

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")


def check_iteration(h, XO, dims, A, loss, kind, p, q, seed, stream, bf16=False):
    g = gcp()
    rank = A[0].shape[1]
    F = g.Factors(A, bf16=bf16)
    S = g.Sampling(kind, p, q, seed, stream)
    G = F.like()
    g.gcp_grad(h, F, loss, G, S=S)
    L = g.gcp_sample(h, S)
    torch.cuda.synchronize()
    assert g.gcp_get_device_status(h) == 0
    SO = oracle.sample(XO, kind, p, q, seed, stream)
    assert_lists_equal(L, SO)
    got = grad_to_numpy(G, rank)
    if bf16:
        A_bf = [a.float()[:, :rank].double().cpu().numpy() for a in F.A_bf16]
        assert_grad_close(got, oracle.grad(dims, A_bf, loss, SO))
        assert rel_norm(got, oracle.grad(dims, f64(A), loss, SO)) <= BF16_RTOL
    else:
        assert_grad_close(got, oracle.grad(dims, f64(A), loss, SO))
    return L


def test_dense_small_workload():
    """20x30x40 FP64-generated tensor (FP32 on the device), rank 3, Gaussian,
    uniform 1000 draws, 500-entry loss estimate."""
    from paper_1906_01687_gb300 import synth
    g = gcp()
    X, _, _ = synth.dense_small()
    X32 = X.astype(np.float32)
    dims = X.shape
    h = g.Handle(g.DataTensor.dense(X32))
    XO = oracle.Tensor(dims, dense=X32.astype(np.float64))
    A = synth.initial_guess(dims, 3, 3, target_norm=float(np.linalg.norm(X32)))
    for it in (0, 1, 99):
        check_iteration(h, XO, dims, A, g.LOSS_GAUSSIAN, g.SAMPLER_UNIFORM, 0, 1000, 1687, it)
    est = g.gcp_sample(h, g.Sampling(g.SAMPLER_UNIFORM, 0, 500, 7, g.STREAM_EST))
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    g.gcp_loss_est(h, g.Factors(A), g.LOSS_GAUSSIAN, est, out)
    torch.cuda.synchronize()
    SO = oracle.sample(XO, oracle.UNIFORM, 0, 500, 7, 2**64 - 1)
    assert abs(out.item() - oracle.loss_estimate(dims, f64(A), oracle.GAUSSIAN, SO)) <= \
        2e-6 * oracle.loss_abs(dims, f64(A), oracle.GAUSSIAN, SO)


def test_dense_100_4_workload():
    """100^4 FP32 tensor (400 MB), rank 10, Gaussian, uniform 1e5 draws: the
    benchmark's workload and launch shape."""
    from paper_1906_01687_gb300 import synth
    g = gcp()
    X32, _ = synth.dense_100_4()
    dims = X32.shape
    h = g.Handle(g.DataTensor.dense(X32))
    XO = oracle.Tensor(dims, dense=X32.reshape(-1).astype(np.float64))
    A = synth.initial_guess(dims, 10, 3, target_norm=float(np.linalg.norm(X32)))
    for it in (0, 12345):
        check_iteration(h, XO, dims, A, g.LOSS_GAUSSIAN, g.SAMPLER_UNIFORM, 0, 100_000, 1687, it)
    est = g.gcp_sample(h, g.Sampling(g.SAMPLER_UNIFORM, 0, 100_000, 7, g.STREAM_EST))
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    g.gcp_loss_est(h, g.Factors(A), g.LOSS_GAUSSIAN, est, out)
    torch.cuda.synchronize()
    SO = oracle.sample(XO, oracle.UNIFORM, 0, 100_000, 7, 2**64 - 1)
    assert abs(out.item() - oracle.loss_estimate(dims, f64(A), oracle.GAUSSIAN, SO)) <= \
        2e-6 * oracle.loss_abs(dims, f64(A), oracle.GAUSSIAN, SO)


@pytest.mark.parametrize("bf16", [False, True])
def test_count_tensor_workload(bf16):
    """6186x24x77x32 count tensor with 5,330,673 nonzeros, rank 10,
    Poisson-log, stratified 1e5 nonzeros + 1e5 zeros."""
    from paper_1906_01687_gb300 import synth
    g = gcp()
    dims = (6186, 24, 77, 32)
    idx, vals, _ = synth.count_tensor()
    h = g.Handle(g.DataTensor.coo(dims, idx, vals))
    XO = oracle_sparse(dims, idx, vals)
    A = synth.initial_guess(dims, 10, 4, target_norm=float(np.linalg.norm(vals)), positive=True)
    A = [(a * 0.3).astype(np.float32) for a in A]
    check_iteration(h, XO, dims, A, g.LOSS_POISSON_LOG, g.SAMPLER_STRATIFIED, 100_000, 100_000, 1687, 5, bf16=bf16)


def test_binary_large_workload():
    """1e5 x 1e5 x 1e4 binary tensor with 1e8 nonzeros, rank 32,
    Bernoulli-logit, semi-stratified 1e6 + 1e6 draws, BF16 factor storage."""
    from paper_1906_01687_gb300 import synth
    g = gcp()
    dims = (100_000, 100_000, 10_000)
    idx, _, planted = synth.binary_tensor(device="cuda")
    h = g.Handle(g.DataTensor.coo(dims, idx, None))
    XO = oracle_sparse(dims, idx, None)
    A = synth.initial_guess(dims, 32, 5)
    A = [(a / math.sqrt(32) ** (1 / 3)).astype(np.float32) for a in A]
    check_iteration(h, XO, dims, A, g.LOSS_BERNOULLI_LOGIT, g.SAMPLER_SEMI_STRATIFIED, 1_000_000, 1_000_000,
                    1687, 3, bf16=True)
