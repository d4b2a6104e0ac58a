"""Parity of the optimizer kernels (Adam with projection, epoch accept and
revert of Alg. 4), the BF16-storage form and the autograd form with the
FP64 oracle, and planted recovery through the device-side GCP-Adam."""
import math
import os

import numpy as np
import pytest

import oracle
from gpu_util import (BF16_RTOL, GRAD_RTOL, assert_grad_close, f64, gcp, grad_to_numpy, oracle_sparse,
                      rel_norm, rng_factors, sparse_random)

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

B1, B2, EPS = float(np.float32(0.9)), float(np.float32(0.999)), float(np.float32(1e-8))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")


def flat(mats, rank):
    return np.concatenate([m[:, :rank].double().cpu().numpy().reshape(-1) for m in mats])


@pytest.mark.parametrize("rank,lower,inside", [(10, -math.inf, True), (3, 0.0, True), (32, -math.inf, False),
                                               (7, -0.05, True)])
@pytest.mark.parametrize("dims", [(37, 20, 9), (3001, 20, 9)], ids=["cluster", "ticket"])
def test_adam_steps_match_oracle(rank, lower, inside, dims):
    """Small factor sets take the one-cluster Adam launch (<= 8 blocks), large
    ones the completion-ticket launch; both match the oracle's Alg. 4 step."""
    g = gcp()
    rs = np.random.default_rng(rank)
    A = [rs.standard_normal((n, rank)).astype(np.float32) for n in dims]
    F = g.Factors(A)
    B, C = F.like(), F.like()
    state = g.new_state()
    alpha = float(np.float32(0.01))
    g.gcp_state_init(state, alpha)
    Ao = np.concatenate([a.astype(np.float64).reshape(-1) for a in A])
    Bo, Co = np.zeros_like(Ao), np.zeros_like(Ao)
    for t in range(4):
        Gs = [rs.standard_normal((n, rank)).astype(np.float32) * (t + 1) for n in dims]
        G = F.like()
        for gd, gs in zip(G, Gs):
            gd[:, :rank] = torch.from_numpy(gs).cuda()
        g.gcp_adam_step(F, G, B, C, state, beta1=B1, beta2=B2, eps=EPS, lower=lower, eps_inside_sqrt=inside)
        oracle.adam_step(Ao, Bo, Co, np.concatenate([x.astype(np.float64).reshape(-1) for x in Gs]), alpha, B1, B2,
                         EPS, lower, t, inside)
        torch.cuda.synchronize()
        assert all(torch.count_nonzero(x).item() == 0 for x in G)
        np.testing.assert_allclose(flat(F.A, rank), Ao, rtol=2e-6, atol=1e-6 * np.abs(Ao).max())
        np.testing.assert_allclose(flat(B, rank), Bo, rtol=2e-6, atol=1e-7 * np.abs(Bo).max())
        np.testing.assert_allclose(flat(C, rank), Co, rtol=2e-6, atol=1e-7 * np.abs(Co).max())
    st = g.read_state(state)
    assert st["t"] == 4 and st["iter"] == 4
    for a in F.A:  # padding columns stay zero
        assert torch.count_nonzero(a[:, rank:]).item() == 0


def test_epoch_accept_and_revert():
    g = gcp()
    dims = (11, 12, 13)
    F = g.Factors(rng_factors(dims, 6, 1))
    B, C = F.like(), F.like()
    SA, SB, SC = F.like(), F.like(), F.like()
    for x in B + C:
        x.normal_()
    state = g.new_state()
    g.gcp_state_init(state, 0.5)
    state[0] = 3.0  # F-hat of the start
    g.gcp_epoch_begin(F, B, C, SA, SB, SC, state)
    torch.cuda.synchronize()
    start = [a.clone() for a in F.A]
    assert g.read_state(state)["F_old"] == 3.0
    # an epoch that lowers F-hat is accepted and becomes the new snapshot
    for a in F.A:
        a[:, :6] += 1.0
    state[0] = 2.5
    state.view(torch.int64)[2] = 7  # t = 7
    g.gcp_epoch_end(F, B, C, SA, SB, SC, state, tau=7, nu=0.1, kappa=1)
    torch.cuda.synchronize()
    st = g.read_state(state)
    assert st["F_old"] == 2.5 and st["t"] == 7 and st["bad"] == 0 and st["alpha"] == 0.5
    accepted = [a.clone() for a in F.A]
    for s_, a in zip(SA, accepted):
        assert torch.equal(s_, a)
    # an epoch that raises it is reverted: factors restored, t wound back, alpha decayed
    for a in F.A:
        a[:, :6] -= 5.0
    state[0] = 2.75
    g.gcp_epoch_end(F, B, C, SA, SB, SC, state, tau=7, nu=0.1, kappa=1)
    torch.cuda.synchronize()
    st = g.read_state(state)
    assert st["F"] == 2.5 and st["t"] == 0 and st["bad"] == 1 and st["done"] == 0
    assert st["alpha"] == pytest.approx(0.05)
    for a, ref in zip(F.A, accepted):
        assert torch.equal(a, ref)
    # a non-finite estimate fails too; the second failure exceeds kappa = 1
    state[0] = float("nan")
    g.gcp_epoch_end(F, B, C, SA, SB, SC, state, tau=7, nu=0.1, kappa=1)
    torch.cuda.synchronize()
    st = g.read_state(state)
    assert st["bad"] == 2 and st["done"] == 1 and st["status"] == g.ERR_NONFINITE
    # once done, Adam steps leave the factors alone but still zero G
    G = F.like()
    for x in G:
        x.fill_(1.0)
    before = [a.clone() for a in F.A]
    g.gcp_adam_step(F, G, B, C, state)
    torch.cuda.synchronize()
    assert all(torch.equal(a, b) for a, b in zip(F.A, before))
    assert all(torch.count_nonzero(x).item() == 0 for x in G)


def test_bf16_form():
    """Gradient gathered from BF16-stored factors: within 1e-5 of the oracle
    at the BF16-rounded factors (arithmetic error) and within 1e-2 of the
    oracle at the FP32 factors (storage error)."""
    g = gcp()
    dims = (300, 40, 25, 12)
    idx, vals = sparse_random(dims, 20000, 3)
    h = g.Handle(g.DataTensor.coo(dims, idx, vals))
    XO = oracle_sparse(dims, idx, vals)
    rank = 10
    A = rng_factors(dims, rank, 4, scale=(0.5 / rank) ** 0.25)
    F = g.Factors(A, bf16=True)
    S = g.Sampling(g.SAMPLER_STRATIFIED, 4000, 4000, seed=5, stream=1)
    G = F.like()
    g.gcp_grad(h, F, g.LOSS_POISSON_LOG, G, S=S)
    torch.cuda.synchronize()
    SO = oracle.sample(XO, oracle.STRATIFIED, 4000, 4000, 5, 1)
    A_bf = [a.float()[:, :rank].double().cpu().numpy() for a in F.A_bf16]
    ref_bf = oracle.grad(dims, A_bf, oracle.POISSON_LOG, SO)
    ref_32 = oracle.grad(dims, f64(A), oracle.POISSON_LOG, SO)
    got = grad_to_numpy(G, rank)
    assert_grad_close(got, ref_bf, rtol=GRAD_RTOL)
    assert rel_norm(got, ref_32) <= BF16_RTOL
    # the loss estimate gathers the same BF16 rows
    est = g.gcp_sample(h, g.Sampling(g.SAMPLER_STRATIFIED, 5000, 5000, seed=6, stream=g.STREAM_EST))
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    g.gcp_loss_est(h, F, g.LOSS_POISSON_LOG, est, out)
    torch.cuda.synchronize()
    SOe = oracle.sample(XO, oracle.STRATIFIED, 5000, 5000, 6, 2**64 - 1)
    assert abs(out.item() - oracle.loss_estimate(dims, A_bf, oracle.POISSON_LOG, SOe)) <= \
        2e-6 * oracle.loss_abs(dims, A_bf, oracle.POISSON_LOG, SOe)
    # Adam keeps the BF16 copy equal to the rounded FP32 master
    B, C, state = F.like(), F.like(), g.new_state()
    g.gcp_state_init(state, 0.01)
    g.gcp_adam_step(F, G, B, C, state)
    torch.cuda.synchronize()
    for a, ab in zip(F.A, F.A_bf16):
        assert torch.equal(a.to(torch.bfloat16), ab)


def test_autograd_function():
    """GcpLoss: forward = F-hat on a fixed list, backward = the sampled
    gradient; checked against the oracle and against central differences."""
    from paper_1906_01687_gb300.autograd import gcp_loss
    g = gcp()
    dims = (20, 18, 16, 14)
    X = np.random.default_rng(7).standard_normal(dims).astype(np.float32)
    h = g.Handle(g.DataTensor.dense(X))
    rank = 10
    A = rng_factors(dims, rank, 8, scale=(0.5 / rank) ** 0.25)
    L = g.gcp_sample(h, g.Sampling(g.SAMPLER_UNIFORM, 0, 4000, seed=9, stream=g.STREAM_EST))
    At = [torch.tensor(a, device="cuda", requires_grad=True) for a in A]
    Fh = gcp_loss(h, g.LOSS_GAUSSIAN, L, *At)
    Fh.backward()
    XO = oracle.Tensor(dims, dense=X.astype(np.float64))
    SO = oracle.sample(XO, oracle.UNIFORM, 0, 4000, 9, 2**64 - 1)
    assert Fh.item() == pytest.approx(oracle.loss_estimate(dims, f64(A), oracle.GAUSSIAN, SO), rel=2e-6)
    grads = [a.grad.double().cpu().numpy() for a in At]
    assert_grad_close(grads, oracle.grad(dims, f64(A), oracle.GAUSSIAN, SO))
    # central differences of the CUDA forward itself (FP64 reduction, FP32 terms)
    rs = np.random.default_rng(0)
    for _ in range(6):
        k, i, j = int(rs.integers(4)), 0, int(rs.integers(rank))
        i = int(rs.integers(dims[k]))
        h_ = 1e-2
        vals = []
        for sgn in (1, -1):
            Ap = [a.detach().clone() for a in At]
            Ap[k][i, j] += sgn * h_
            vals.append(gcp_loss(h, g.LOSS_GAUSSIAN, L, *Ap).item())
        fd = (vals[0] - vals[1]) / (2 * h_)
        assert grads[k][i, j] == pytest.approx(fd, rel=2e-2, abs=2e-3 * max(1.0, abs(fd)))


def test_device_adam_matches_oracle_driver():
    """A short GCP-Adam run with device-side epochs (graph-replayed) follows
    the oracle's Alg. 4 loop: same draws, same accept/revert decisions, and
    factors that agree to FP32 accuracy."""
    from oracle.driver import gcp_adam as oracle_gcp_adam
    from paper_1906_01687_gb300.adam import GcpAdam
    g = gcp()
    dims = (20, 30, 40)
    rs = np.random.default_rng(1)
    true = [rs.standard_normal((n, 3)) for n in dims]
    X = np.einsum("ir,jr,kr->ijk", *true).astype(np.float32) + 0.1 * rs.standard_normal(dims).astype(np.float32)
    A0 = rng_factors(dims, 3, 2, scale=0.5)
    run = GcpAdam(g.DataTensor.dense(X), A0, g.LOSS_GAUSSIAN, g.SAMPLER_UNIFORM, 0, 1000, 0, 500, seed=11,
                  est_seed=12, alpha=float(np.float32(0.01)), beta1=B1, beta2=B2, eps=EPS, tau=20)
    st = run.fit(max_epochs=3)
    est, hist = oracle_gcp_adam(oracle.Tensor(dims, dense=X.astype(np.float64)), f64(A0), oracle.GAUSSIAN,
                                oracle.UNIFORM, 0, 1000, 0, 500, seed=11, est_seed=12, alpha=float(np.float32(0.01)),
                                beta1=B1, beta2=B2, eps=EPS, tau=20, max_epochs=3)
    got = run.factors()
    num = sum(np.linalg.norm(a - b) ** 2 for a, b in zip(got, est))
    den = sum(np.linalg.norm(b) ** 2 for b in est)
    assert math.sqrt(num / den) < 1e-4
    np.testing.assert_allclose(run.history, hist, rtol=1e-5)


def test_planted_recovery_on_gpu():
    """Planted rank-3 factors (noise at 10% of the model) are recovered with
    score >= 0.9 (App. E) by the device-side GCP-Adam."""
    from oracle.score import cosine_score
    from paper_1906_01687_gb300 import synth
    from paper_1906_01687_gb300.adam import GcpAdam
    g = gcp()
    dims, rank = (20, 30, 40), 3
    rs = np.random.default_rng(5)
    true = [rs.standard_normal((n, rank)) for n in dims]
    true = [a / np.linalg.norm(a, axis=0, keepdims=True) for a in true]
    M = synth.dense_from_factors(true, np.array([30.0, 25.0, 20.0]))
    X = (M + 0.1 * np.linalg.norm(M) / math.sqrt(M.size) * rs.standard_normal(M.shape)).astype(np.float32)
    A0 = synth.initial_guess(dims, rank, 6, target_norm=float(np.linalg.norm(X)))
    run = GcpAdam(g.DataTensor.dense(X), A0, g.LOSS_GAUSSIAN, g.SAMPLER_UNIFORM, 0, 1000, 0, 500, seed=7,
                  est_seed=8, alpha=0.01, tau=100)
    run.fit(max_epochs=40)
    assert cosine_score(true, run.factors()) >= 0.9


@pytest.mark.parametrize("kind", ["uniform", "stratified", "uniform_large", "semi_stream"])
def test_fused_iteration_equals_grad_then_adam(kind):
    """gcp_iteration (gradient + Adam with the replica fold inside Adam) gives
    the factors of gcp_grad followed by gcp_adam_step on the same draws: with
    more than 16 replicas per mode (the fold's tail), with factor sets small
    enough for the one-cluster Adam launch and large enough for the ticket
    launch, and (semi_stream: 1.2M float4 elements, short modes replicated)
    large enough for gcp_iteration's streaming Adam kernel."""
    g = gcp()
    if kind == "semi_stream":
        dims = (400_000, 40, 30)
        idx, vals = sparse_random(dims, 20000, 10)
        h = g.Handle(g.DataTensor.coo(dims, idx, vals))
        S = g.Sampling(g.SAMPLER_SEMI_STRATIFIED, 20000, 20000, seed=3, stream=5)
    elif kind in ("uniform", "uniform_large"):
        dims = (60, 50, 40, 30) if kind == "uniform" else (3000, 40, 30)
        X = np.random.default_rng(3).standard_normal(dims).astype(np.float32)
        h = g.Handle(g.DataTensor.dense(X))
        S = g.Sampling(g.SAMPLER_UNIFORM, 0, 50000, seed=3, stream=5)
    else:
        dims = (300, 40, 25)
        idx, vals = sparse_random(dims, 20000, 9)
        h = g.Handle(g.DataTensor.coo(dims, idx, vals))
        S = g.Sampling(g.SAMPLER_STRATIFIED, 20000, 20000, seed=3, stream=5)
    A = rng_factors(dims, 10, 4, scale=0.5)
    runs = []
    for fused in (True, False):
        F = g.Factors(A)
        G, B, C, st = F.like(), F.like(), F.like(), g.new_state()
        g.gcp_state_init(st, 0.01)
        for it in range(3):
            Sit = g.Sampling(S.kind, S.p, S.q, S.seed, it)
            if fused:
                g.gcp_iteration(h, F, g.LOSS_POISSON_LOG, Sit, G, B, C, st)
            else:
                g.gcp_grad(h, F, g.LOSS_POISSON_LOG, G, S=Sit)
                g.gcp_adam_step(F, G, B, C, st)
        torch.cuda.synchronize()
        assert all(torch.count_nonzero(x).item() == 0 for x in G)
        runs.append(flat(F.A, 10))
        assert g.read_state(st)["t"] == 3
    # The two runs add the same terms in different orders.  An entry of G that
    # nearly cancels (a row hit by few draws) keeps only rounding noise, and
    # Adam's normalised step turns it into a move of up to alpha per step, so
    # single entries may differ by up to steps * alpha while all others agree
    # to FP32 noise.
    diff = np.abs(runs[0] - runs[1])
    assert diff.max() <= 3 * 0.01 * 1.01
    assert np.count_nonzero(diff > 1e-5 * np.abs(runs[1]).max()) <= 1e-3 * diff.size


def test_profile_events_count_gradient_kernels():
    g = gcp()
    dims = (30, 20, 10)
    X = np.random.default_rng(1).standard_normal(dims).astype(np.float32)
    h = g.Handle(g.DataTensor.dense(X))
    F = g.Factors(rng_factors(dims, 8, 2))
    G = F.like()
    g.gcp_profile(h, True, 4)
    for i in range(6):  # only the first 4 launches are timed
        g.gcp_grad(h, F, 0, G, S=g.Sampling(g.SAMPLER_UNIFORM, 0, 5000, seed=1, stream=i))
    ms, n = g.gcp_profile_read(h)
    assert n == 4 and ms > 0
    ms, n = g.gcp_profile_read(h)
    assert n == 0
    B, C, st = F.like(), F.like(), g.new_state()
    g.gcp_state_init(st, 0.01)
    for x in G:
        x.zero_()
    g.gcp_iteration(h, F, 0, g.Sampling(g.SAMPLER_UNIFORM, 0, 5000, seed=1, stream=9), G, B, C, st)
    assert g.gcp_profile_read(h, 0)[1] == 1 and g.gcp_profile_read(h, 1)[1] == 1
    # with tail_work this small factor set's Adam step is taken by the gradient kernel: no Adam launch to time
    g.gcp_set_tuning(h, tail_work=1)
    g.gcp_iteration(h, F, 0, g.Sampling(g.SAMPLER_UNIFORM, 0, 5000, seed=1, stream=10), G, B, C, st)
    assert g.gcp_profile_read(h, 0)[1] == 1 and g.gcp_profile_read(h, 1)[1] == 0
    g.gcp_profile(h, False)


def test_gamma_problem_fits_with_projection():
    """App. C's gamma problem (scaled down): GCP-Adam with the gamma loss and
    the projection max(A, 0) lowers F-hat and keeps the factors nonnegative."""
    from paper_1906_01687_gb300 import synth
    from paper_1906_01687_gb300.adam import GcpAdam
    g = gcp()
    X, true = synth.gamma_problem(dims=(20, 15, 10, 5), rank=3)
    A0 = synth.initial_guess(X.shape, 3, 4, target_norm=float(np.linalg.norm(X)), positive=True)
    run = GcpAdam(g.DataTensor.dense(X), A0, g.LOSS_GAMMA, g.SAMPLER_UNIFORM, 0, 500, 0, 5000, seed=3, est_seed=4,
                  alpha=0.01, tau=100, lower=0.0)
    st = run.fit(max_epochs=10)
    assert run.history[-1] < run.history[0] and math.isfinite(run.history[-1])
    assert all((a >= 0).all() for a in run.factors())


def test_checkpoint_resume_reproduces_run(tmp_path):
    """Four epochs straight, or two epochs, a checkpoint through torch.save,
    and two more epochs in a fresh driver: the same draws and, up to the
    summation order of the atomics, the same factors and state."""
    from paper_1906_01687_gb300.adam import GcpAdam
    g = gcp()
    dims = (20, 30, 40)
    rs = np.random.default_rng(9)
    X = rs.standard_normal(dims).astype(np.float32)
    A0 = rng_factors(dims, 4, 10, scale=0.5)
    mk = lambda: GcpAdam(g.DataTensor.dense(X), A0, g.LOSS_GAUSSIAN, g.SAMPLER_UNIFORM, 0, 2000, 0, 1000, seed=5,
                         est_seed=6, alpha=0.01, tau=25)
    straight = mk()
    straight.fit(max_epochs=4)
    first = mk()
    first.fit(max_epochs=2)
    path = tmp_path / "ckpt.pt"
    torch.save(first.state_dict(), path)
    resumed = mk()
    resumed.load_state_dict(torch.load(path))
    resumed.fit(max_epochs=2)
    a, b = straight.factors(), resumed.factors()
    num = math.sqrt(sum(np.linalg.norm(x - y) ** 2 for x, y in zip(a, b)))
    assert num <= 1e-4 * math.sqrt(sum(np.linalg.norm(y) ** 2 for y in a))
    s1, s2 = straight.status(), resumed.status()
    assert (s1["t"], s1["iter"], s1["bad"]) == (s2["t"], s2["iter"], s2["bad"])


def test_python_example_runs():
    """The Python example (examples/fit_dense.py), as written, runs and lowers the estimated loss."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("fit_dense", os.path.join(ROOT, "examples", "fit_dense.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    state, history, A = mod.fit(max_epochs=50)
    assert len(A) == 3 and all(a.shape == (n, 3) for a, n in zip(A, (20, 30, 40)))
    assert state["status"] == 0 and math.isfinite(state["F"]) and state["F"] < history[0]


def test_gcp_adam_with_observed_sampler():
    """GCP-Adam on a tensor with 40% of its entries missing (weight 0), drawing
    only observed entries (Section 4.4) for the gradients and the fixed
    estimate set, through the captured epoch: the estimated loss falls and the
    run ends without a device error."""
    from paper_1906_01687_gb300 import gcp as G, synth
    from paper_1906_01687_gb300.adam import GcpAdam
    X = synth.dense_small()[0].astype(np.float32)
    r = np.random.default_rng(3)
    v = (r.random(X.shape) >= 0.4).astype(np.float32)
    A0 = synth.initial_guess(X.shape, 3, seed=2, target_norm=float(np.linalg.norm(X * v)))
    run = GcpAdam(G.DataTensor.dense(X, weights=v), A0, G.LOSS_GAUSSIAN, G.SAMPLER_OBSERVED, p=0, q=1000,
                  est_p=0, est_q=2000, seed=4, est_seed=5, tau=50)
    state = run.fit(max_epochs=20)
    # the planted model is fitted down to the noise floor (0.01 per observed entry, ~145 here)
    assert state["status"] == 0 and math.isfinite(state["F"]) and state["F"] < 0.7 * run.history[0]
