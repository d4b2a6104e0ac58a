"""Parity where FP32 cancellation is worst: the 1e8-nonzero binary tensor
(1e5 x 1e5 x 1e4), Bernoulli-logit, semi-stratified 1e6 + 1e6 draws
(omega / q = 1e8, eta / p = 100), at factors near a fitted model.

Near a fit, sigma(m) of a zero is about the density, 1e-6, so a "zero"
draw's y = (omega / q) sigma(m) is about +100 while a nonzero draw's
y = (eta / p) [(sigma(m) - 1) - sigma(m)] is -100: the rows of G sum terms
of both signs that nearly cancel (Alg. 3).  The factors here are the
planted rank-32 logistic model with its first column replaced by a
constant whose cube is log(1e-6), so that m = log(1e-6) + (planted
structure).  The FP32 gradient must stay within 1e-5 of the FP64 oracle
norm-wise and within the element-wise bound of each element's sum of
|contributions|; the BF16 form within 1e-5 of the oracle at the BF16-rounded
factors.  Against the oracle at the FP32 factors the BF16 form is far from
1e-2 here: rounding a factor entry of about 2.4 to BF16 moves m by about
0.05, which moves sigma(m) = e^m of every zero term by about 5%, and the
terms cancel.  That is the storage format's own sensitivity, which the FP64
oracle shows just the same between the two sets of factors; the test checks
that the GPU's BF16 error equals it.
"""
import math

import numpy as np
import pytest

import oracle
from gpu_util import (BF16_RTOL, assert_grad_close, f64, gcp, grad_to_numpy, oracle_sparse, rel_norm)

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

DIMS, RANK, P, Q = (100_000, 100_000, 10_000), 32, 1_000_000, 1_000_000


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")


def near_fitted(planted):
    c = -(-math.log(1e-6)) ** (1.0 / 3.0)  # c^3 = log(1e-6): three negative entries
    A = [np.array(a, dtype=np.float32) for a in planted]
    for a in A:
        a[:, 0] = c
    return A


def test_semi_stratified_cancellation_near_a_fitted_model():
    from paper_1906_01687_gb300 import synth
    g = gcp()
    idx, _, planted = synth.binary_tensor(device="cuda")
    h = g.Handle(g.DataTensor.coo(DIMS, idx, None))
    XO = oracle_sparse(DIMS, idx, None)
    A = near_fitted(planted)
    S = g.Sampling(g.SAMPLER_SEMI_STRATIFIED, P, Q, 1687, 11)
    SO = oracle.sample(XO, oracle.SEMI_STRATIFIED, P, Q, 1687, 11)
    # the regime: most zero draws have sigma(m) of order 1e-6, so both kinds of term are about 100
    sub = SO.idx[P:P + 1000]
    m = np.zeros(len(sub))
    for j in range(RANK):
        m += A[0][sub[:, 0], j].astype(np.float64) * A[1][sub[:, 1], j] * A[2][sub[:, 2], j]
    assert np.median(np.abs(m - math.log(1e-6))) < 2.0
    ref = oracle.grad(DIMS, f64(A), oracle.BERNOULLI_LOGIT, SO)
    gabs = oracle.grad_abs(DIMS, f64(A), oracle.BERNOULLI_LOGIT, SO)
    for bf16 in (False, True):
        F = g.Factors(A, bf16=bf16)
        G = F.like()
        g.gcp_grad(h, F, g.LOSS_BERNOULLI_LOGIT, G, S=S)
        torch.cuda.synchronize()
        assert g.gcp_get_device_status(h) == 0
        got = grad_to_numpy(G, RANK)
        if bf16:
            A_bf = [a.float()[:, :RANK].double().cpu().numpy() for a in F.A_bf16]
            ref_bf = oracle.grad(DIMS, A_bf, oracle.BERNOULLI_LOGIT, SO)
            assert_grad_close(got, ref_bf)
            storage = rel_norm(ref_bf, ref)  # the FP64 oracle's own change from rounding the factors
            assert storage > BF16_RTOL  # the cancellation regime (about 0.2)
            assert abs(rel_norm(got, ref) - storage) <= 1e-4 * storage
        else:
            assert_grad_close(got, ref, gabs)
