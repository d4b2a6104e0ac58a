"""Edge cases of the CUDA path against the FP64 oracle: the most modes the
C ABI takes (d = 8: two Philox blocks per draw, 48-byte nonzero records), the
largest rank (256), BF16-stored rows with eight modes, and the fused GCP-Adam
iteration there.  Same bars as the parity tests: bit-exact sample lists,
gradients within 1e-5 norm-wise and the element-wise bound, loss estimates
within 2e-6 of the sum of |terms|.  (The fewest modes, d = 2, are covered by
the parity tests; d = 1 is rejected on the host.)
"""
import math

import numpy as np
import pytest

import oracle
from gpu_util import (BF16_RTOL, LOSS_RTOL, assert_grad_close, assert_lists_equal, assert_pads_zero, f64, gcp,
                      grad_to_numpy, oracle_sparse, rel_norm, rng_factors, sparse_random)

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

LOSS_IDS = {0: "gaussian", 1: "logit", 2: "poisson"}
DIMS_D8 = (3, 4, 2, 5, 3, 2, 4, 3)          # 8640 entries
DIMS_D8_SPARSE = (6, 5, 4, 7, 3, 5, 4, 6)   # 302,400 entries


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1906_01687_gb300 import build
    build.build()


def dense_for_loss(dims, seed, loss):
    X = np.random.default_rng(seed).standard_normal(dims).astype(np.float32)
    if loss == 1:
        X = (X > 0.5).astype(np.float32)
    elif loss == 2:
        X = np.floor(np.abs(X) * 2).astype(np.float32)
    return X, oracle.Tensor(dims, dense=X.astype(np.float64))


def check_uniform(dims, rank, loss, seed):
    """Uniform draws over a dense tensor: the list bit for bit, the fused
    gradient and the loss estimate against the oracle."""
    g = gcp()
    X, XO = dense_for_loss(dims, seed, loss)
    h = g.Handle(g.DataTensor.dense(X))
    A = rng_factors(dims, rank, seed + 1, scale=(0.5 / rank) ** (1 / len(dims)))
    F = g.Factors(A)
    S = g.Sampling(g.SAMPLER_UNIFORM, 0, 3001, seed=seed + 2, stream=4)
    SO = oracle.sample(XO, oracle.UNIFORM, 0, 3001, seed + 2, 4)
    L = g.gcp_sample(h, S)
    G = F.like()
    g.gcp_grad(h, F, loss, G, S=S)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    g.gcp_loss_est(h, F, loss, L, out)
    torch.cuda.synchronize()
    assert g.gcp_get_device_status(h) == 0
    assert_lists_equal(L, SO)
    assert_pads_zero(G, rank)
    assert_grad_close(grad_to_numpy(G, rank), oracle.grad(dims, f64(A), loss, SO),
                      oracle.grad_abs(dims, f64(A), loss, SO))
    ref = oracle.loss_estimate(dims, f64(A), loss, SO)
    assert abs(out.item() - ref) <= LOSS_RTOL * oracle.loss_abs(dims, f64(A), loss, SO)


def check_sparse(dims, nnz, rank, kind, loss, seed):
    g = gcp()
    idx, vals = sparse_random(dims, nnz, seed, binary=(loss == 1))
    h = g.Handle(g.DataTensor.coo(dims, idx, vals))
    XO = oracle_sparse(dims, idx, vals)
    A = rng_factors(dims, rank, seed + 1, scale=(0.5 / rank) ** (1 / len(dims)))
    F = g.Factors(A)
    S = g.Sampling(g.SAMPLERS[kind], 1500, 1700, seed=seed + 2, stream=6)
    SO = oracle.sample(XO, g.SAMPLERS[kind], 1500, 1700, seed + 2, 6)
    L = g.gcp_sample(h, S)
    G = F.like()
    g.gcp_grad(h, F, loss, G, S=S)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    g.gcp_loss_est(h, F, loss, L, out)
    torch.cuda.synchronize()
    assert g.gcp_get_device_status(h) == 0
    assert_lists_equal(L, SO)
    assert_grad_close(grad_to_numpy(G, rank), oracle.grad(dims, f64(A), loss, SO),
                      oracle.grad_abs(dims, f64(A), loss, SO))
    ref = oracle.loss_estimate(dims, f64(A), loss, SO)
    assert abs(out.item() - ref) <= LOSS_RTOL * oracle.loss_abs(dims, f64(A), loss, SO)


# ---------------------------------------------------------------------------
# d = 8: two Philox blocks per draw, three 16-byte words per nonzero record
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("loss", [0, 1, 2], ids=LOSS_IDS.get)
def test_eight_modes_dense(loss):
    check_uniform(DIMS_D8, 5, loss, 51)


@pytest.mark.parametrize("kind", ["stratified", "semi_stratified"])
@pytest.mark.parametrize("loss", [0, 2], ids=LOSS_IDS.get)
def test_eight_modes_sparse(kind, loss):
    check_sparse(DIMS_D8_SPARSE, 3000, 4, kind, loss, 61)


def test_eight_modes_bf16_rows():
    """BF16-stored factors with eight modes: within 1e-5 of the oracle at the
    BF16-rounded factors (arithmetic error), and within 2e-2 of it at the
    FP32 factors (storage error: each update multiplies d - 1 rounded rows
    and m sums products of d, so the four-way bound of 1e-2 is scaled by
    d / 4)."""
    g = gcp()
    dims, rank = DIMS_D8_SPARSE, 6
    idx, vals = sparse_random(dims, 3000, 71)
    h = g.Handle(g.DataTensor.coo(dims, idx, vals))
    XO = oracle_sparse(dims, idx, vals)
    A = rng_factors(dims, rank, 72, scale=(0.5 / rank) ** (1 / 8))
    F = g.Factors(A, bf16=True)
    S = g.Sampling(g.SAMPLER_STRATIFIED, 2000, 2000, seed=73, stream=1)
    G = F.like()
    g.gcp_grad(h, F, g.LOSS_POISSON_LOG, G, S=S)
    torch.cuda.synchronize()
    assert g.gcp_get_device_status(h) == 0
    SO = oracle.sample(XO, oracle.STRATIFIED, 2000, 2000, 73, 1)
    A_bf = [a.float()[:, :rank].double().cpu().numpy() for a in F.A_bf16]
    got = grad_to_numpy(G, rank)
    assert_grad_close(got, oracle.grad(dims, A_bf, oracle.POISSON_LOG, SO))
    assert rel_norm(got, oracle.grad(dims, f64(A), oracle.POISSON_LOG, SO)) <= BF16_RTOL * 8 / 4


# ---------------------------------------------------------------------------
# the largest rank: 64 float4 chunks per row (32 lanes x 2 chunks)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("loss", [0, 2], ids=LOSS_IDS.get)
def test_largest_rank(loss):
    check_uniform((30, 20, 10), 256, loss, 81)


def test_largest_rank_adam_step():
    g = gcp()
    dims, rank = (30, 20, 10), 256
    rs = np.random.default_rng(91)
    A = [rs.standard_normal((n, rank)).astype(np.float32) for n in dims]
    F = g.Factors(A)
    B, C, state = F.like(), F.like(), g.new_state()
    alpha = float(np.float32(0.01))
    g.gcp_state_init(state, alpha)
    Gs = [rs.standard_normal((n, rank)).astype(np.float32) for n in dims]
    G = F.like()
    for gd, gs in zip(G, Gs):
        gd[:, :rank] = torch.from_numpy(gs).cuda()
    b1, b2, eps = float(np.float32(0.9)), float(np.float32(0.999)), float(np.float32(1e-8))
    g.gcp_adam_step(F, G, B, C, state, beta1=b1, beta2=b2, eps=eps)
    Ao = np.concatenate([a.astype(np.float64).reshape(-1) for a in A])
    Bo, Co = np.zeros_like(Ao), np.zeros_like(Ao)
    oracle.adam_step(Ao, Bo, Co, np.concatenate([x.astype(np.float64).reshape(-1) for x in Gs]), alpha, b1, b2,
                     eps, -math.inf, 0, True)
    torch.cuda.synchronize()
    got = np.concatenate([a[:, :rank].double().cpu().numpy().reshape(-1) for a in F.A])
    np.testing.assert_allclose(got, Ao, rtol=2e-6, atol=1e-6 * np.abs(Ao).max())
    assert all(torch.count_nonzero(x).item() == 0 for x in G)


# ---------------------------------------------------------------------------
# the fused iteration (gradient, replica fold, Adam) with eight modes
# ---------------------------------------------------------------------------

def test_eight_modes_fused_iteration_equals_grad_then_adam():
    """Every row of these short modes is hit thousands of times per launch,
    so each mode is spread over replica slabs; gcp_iteration must give the
    factors of gcp_grad followed by gcp_adam_step (up to summation order)."""
    g = gcp()
    dims = DIMS_D8
    X = np.random.default_rng(101).standard_normal(dims).astype(np.float32)
    h = g.Handle(g.DataTensor.dense(X))
    A = rng_factors(dims, 6, 102, scale=0.8)
    runs = []
    for fused in (True, False):
        F = g.Factors(A)
        G, B, C, st = F.like(), F.like(), F.like(), g.new_state()
        g.gcp_state_init(st, 0.01)
        for it in range(3):
            S = g.Sampling(g.SAMPLER_UNIFORM, 0, 50000, seed=103, stream=it)
            if fused:
                g.gcp_iteration(h, F, g.LOSS_GAUSSIAN, S, G, B, C, st)
            else:
                g.gcp_grad(h, F, g.LOSS_GAUSSIAN, G, S=S)
                g.gcp_adam_step(F, G, B, C, st)
        torch.cuda.synchronize()
        assert g.gcp_get_device_status(h) == 0
        assert all(torch.count_nonzero(x).item() == 0 for x in G)
        assert g.read_state(st)["t"] == 3
        runs.append(np.concatenate([a[:, :6].double().cpu().numpy().reshape(-1) for a in F.A]))
    # entries of G that nearly cancel keep only rounding noise, which Adam's
    # normalised step can turn into a move of up to alpha per step
    diff = np.abs(runs[0] - runs[1])
    assert diff.max() <= 3 * 0.01 * 1.01
    assert np.count_nonzero(diff > 1e-5 * np.abs(runs[1]).max()) <= max(2, 1e-3 * diff.size)


def test_eight_modes_gcp_adam_matches_oracle_driver():
    """Graph-replayed GCP-Adam epochs (early draws, replica fold, device-side
    accept/revert) on a planted eight-way problem follow the oracle's Alg. 4
    loop: the same estimates per epoch and factors equal to FP32 accuracy."""
    from oracle.driver import gcp_adam as oracle_gcp_adam
    from paper_1906_01687_gb300.adam import GcpAdam
    g = gcp()
    dims, rank = DIMS_D8, 2
    rs = np.random.default_rng(111)
    true = [rs.standard_normal((n, rank)) for n in dims]
    M = np.zeros(dims)
    for j in range(rank):
        t = true[0][:, j]
        for a in true[1:]:
            t = np.multiply.outer(t, a[:, j])
        M += t
    X = (M + 0.1 * rs.standard_normal(dims)).astype(np.float32)
    A0 = rng_factors(dims, rank, 112, scale=0.8)
    alpha, b1, b2, eps = (float(np.float32(v)) for v in (0.01, 0.9, 0.999, 1e-8))
    run = GcpAdam(g.DataTensor.dense(X), A0, g.LOSS_GAUSSIAN, g.SAMPLER_UNIFORM, 0, 1000, 0, 500, seed=113,
                  est_seed=114, alpha=alpha, beta1=b1, beta2=b2, eps=eps, tau=20)
    run.fit(max_epochs=3)
    est, hist = oracle_gcp_adam(oracle.Tensor(dims, dense=X.astype(np.float64)), f64(A0), oracle.GAUSSIAN,
                                oracle.UNIFORM, 0, 1000, 0, 500, seed=113, est_seed=114, alpha=alpha, beta1=b1,
                                beta2=b2, eps=eps, tau=20, max_epochs=3)
    got = run.factors()
    num = sum(np.linalg.norm(a - b) ** 2 for a, b in zip(got, est))
    den = sum(np.linalg.norm(b) ** 2 for b in est)
    assert math.sqrt(num / den) < 1e-4
    np.testing.assert_allclose(run.history, hist, rtol=1e-5)
