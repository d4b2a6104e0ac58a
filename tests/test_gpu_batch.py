"""The batched form (many independent problems, one launch per step) against
the single-problem path and the FP64 oracle: the same draws, gradients,
Adam steps, loss estimates and epoch decisions for every problem."""
import math

import numpy as np
import pytest

import oracle
from gpu_util import assert_grad_close, f64, gcp, grad_to_numpy, rng_factors

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SHAPES = [((40, 30, 20), 4, 0), ((25, 20, 15, 10), 8, 1), ((60, 50, 7), 16, 2), ((30, 30, 30), 32, 0),
          ((12, 11, 10, 9), 64, 1), ((55, 3, 40), 10, 2)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")


def make_specs(n_draws=3001):
    specs = []
    for i, (dims, rank, loss) in enumerate(SHAPES):
        rs = np.random.default_rng(100 + i)
        X = rs.standard_normal(dims).astype(np.float32)
        if loss == 1:
            X = (X > 0.3).astype(np.float32)
        elif loss == 2:
            X = np.floor(np.abs(X) * 2).astype(np.float32)
        A0 = rng_factors(dims, rank, 200 + i, scale=(0.5 / rank) ** (1 / len(dims)))
        specs.append(dict(X=X, A0=A0, loss=loss, s=n_draws + 17 * i, est=2000 + i, seed=7 + i, est_seed=9, problem=i))
    return specs


def test_batched_steps_match_single_problem_path():
    from paper_1906_01687_gb300.batch import GcpAdamBatch
    g = gcp()
    specs = make_specs()
    run = GcpAdamBatch(specs, tau=5, alpha=0.01)
    run.batch.grad()
    torch.cuda.synchronize()
    for i, (sp, p) in enumerate(zip(specs, run.problems)):
        dims, rank = sp["X"].shape, sp["A0"][0].shape[1]
        h = g.Handle(g.DataTensor.dense(sp["X"]))
        F = g.Factors(sp["A0"])
        G = F.like()
        S = g.Sampling(g.SAMPLER_UNIFORM, 0, sp["s"], sp["seed"], 0, i)
        g.gcp_grad(h, F, sp["loss"], G, S=S)
        torch.cuda.synchronize()
        got = grad_to_numpy(p["G"], rank)
        assert_grad_close(got, grad_to_numpy(G, rank), rtol=2e-6)
        XO = oracle.Tensor(dims, dense=sp["X"].astype(np.float64))
        SO = oracle.sample(XO, oracle.UNIFORM, 0, sp["s"], sp["seed"], 0, problem=i)
        assert_grad_close(got, oracle.grad(dims, f64(sp["A0"]), sp["loss"], SO))
        # loss estimate of the initial factors (computed at construction) vs the oracle
        SE = oracle.sample(XO, oracle.UNIFORM, 0, sp["est"], sp["est_seed"], 2**64 - 1, problem=i)
        ref = oracle.loss_estimate(dims, f64(sp["A0"]), sp["loss"], SE)
        assert abs(g.read_state(p["state"])["F"] - ref) <= 2e-6 * oracle.loss_abs(dims, f64(sp["A0"]), sp["loss"], SE)


def test_batched_adam_matches_single_problem_path():
    from paper_1906_01687_gb300.batch import GcpAdamBatch
    g = gcp()
    specs = make_specs()
    run = GcpAdamBatch(specs, tau=5, alpha=0.01)
    rs = np.random.default_rng(5)
    grads = []
    for p in run.problems:
        gs = [torch.tensor(rs.standard_normal(x.shape).astype(np.float32), device="cuda") for x in p["G"]]
        for x, v in zip(p["G"], gs):
            x.copy_(v)
            x[:, p["F"].rank:] = 0
        grads.append(gs)
    run.batch.adam_step()
    torch.cuda.synchronize()
    for sp, p, gs in zip(specs, run.problems, grads):
        rank = sp["A0"][0].shape[1]
        F = g.Factors(sp["A0"])
        B, C, st = F.like(), F.like(), g.new_state()
        g.gcp_state_init(st, 0.01)
        G = [x.clone() for x in gs]
        for x in G:
            x[:, rank:] = 0
        g.gcp_adam_step(F, G, B, C, st)
        torch.cuda.synchronize()
        for a, b in zip(p["F"].A, F.A):
            torch.testing.assert_close(a, b, rtol=1e-6, atol=1e-7)
        assert g.read_state(p["state"])["t"] == 1
        assert all(torch.count_nonzero(x).item() == 0 for x in p["G"])


def test_batched_runs_follow_single_runs():
    """Two epochs of the batched GCP-Adam give each problem the factors and
    F-hat history of its own single-problem GCP-Adam run."""
    from paper_1906_01687_gb300.adam import GcpAdam
    from paper_1906_01687_gb300.batch import GcpAdamBatch
    g = gcp()
    specs = make_specs(2000)
    run = GcpAdamBatch(specs, tau=10, alpha=0.01)
    run.fit(max_epochs=2)
    for i, sp in enumerate(specs):
        single = GcpAdam(g.DataTensor.dense(sp["X"]), sp["A0"], sp["loss"], g.SAMPLER_UNIFORM, 0, sp["s"], 0,
                         sp["est"], seed=sp["seed"], est_seed=sp["est_seed"], alpha=0.01, tau=10, problem=i)
        single.fit(max_epochs=2)
        a, b = run.factors(i), single.factors()
        num = math.sqrt(sum(np.linalg.norm(x - y) ** 2 for x, y in zip(a, b)))
        den = math.sqrt(sum(np.linalg.norm(y) ** 2 for y in b))
        assert num <= 1e-4 * den, (i, num / den)
        st_b, st_s = run.states()[i], single.status()
        assert st_b["t"] == st_s["t"] and st_b["bad"] == st_s["bad"]
        assert st_b["F"] == pytest.approx(st_s["F"], rel=1e-5)


def test_batch_autotune_and_graph_replay():
    from paper_1906_01687_gb300.batch import GcpAdamBatch
    specs = make_specs(5000)
    run = GcpAdamBatch(specs, tau=4, alpha=0.01, autotune=True)
    assert run.tuned["seconds_per_iteration"] > 0 and run.tuned["tried"] >= 8
    assert set(run.tuned["best"]) == {"fused", "block", "grid_blocks", "chunks_per_lane", "replica_target",
                                      "max_replicas"}
    assert len(run.tuned["shapes"]) == len(specs)
    sts = run.fit(max_epochs=3)
    assert all(st["iter"] == 12 for st in sts)
    assert all(math.isfinite(st["F"]) for st in sts)


@pytest.mark.parametrize("cpl,target,maxr", [(2, 0, 0), (4, 16, 32), (1, 0, 1), (8, 8, 64)])
def test_batch_shapes_give_the_same_gradients(cpl, target, maxr):
    """Every per-problem shape (chunks per lane, replica width) gives each
    problem the oracle's gradient on the same draws (only the summation order
    changes), and the lanes and replicas follow the rule gcp_batch_set_shape
    states."""
    from paper_1906_01687_gb300.batch import GcpAdamBatch
    specs = make_specs(20_000)
    run = GcpAdamBatch(specs, tau=5, alpha=0.01)
    run.set_shape(chunks_per_lane=cpl, replica_target=target, max_replicas=maxr)
    run.batch.grad()
    torch.cuda.synchronize()
    for i, (sp, p) in enumerate(zip(specs, run.problems)):
        dims, rank = sp["X"].shape, sp["A0"][0].shape[1]
        shape = run.batch.get_shape(i)
        chunks = (rank + 3) // 4
        per = -(-chunks // cpl)
        L = 1
        while L < per and L < 32:
            L *= 2
        assert shape["lanes"] == L and shape["chunks"] == -(-chunks // L)
        t, m = (target or 64), (maxr or 32)
        want = [max(1, min(math.ceil(sp["s"] / n / t), m)) for n in dims]
        assert shape["replicas"] == want
        XO = oracle.Tensor(dims, dense=sp["X"].astype(np.float64))
        SO = oracle.sample(XO, oracle.UNIFORM, 0, sp["s"], sp["seed"], 0, problem=i)
        assert_grad_close(grad_to_numpy(p["G"], rank), oracle.grad(dims, f64(sp["A0"]), sp["loss"], SO),
                          oracle.grad_abs(dims, f64(sp["A0"]), sp["loss"], SO))


def test_batch_rejects_sparse_and_wide_problems():
    g = gcp()
    dims = (5, 6, 7, 3, 2)
    X = np.zeros(dims, np.float32)
    F = g.Factors(rng_factors(dims, 4, 1))
    st = g.new_state()
    p = dict(X=g.DataTensor.dense(X), F=F, loss=0, S=g.Sampling(0, 0, 10, 1), est=g.SampleList.empty(5, 0),
             G=F.like(), B=F.like(), C=F.like(), SA=F.like(), SB=F.like(), SC=F.like(), state=st)
    with pytest.raises(g.GcpError):
        g.Batch([p])  # d = 5 > 4


@pytest.mark.parametrize("cpl,target,maxr", [(1, 0, 0), (2, 16, 32), (1, 0, 1)])
def test_fused_iteration_follows_two_launches(cpl, target, maxr):
    """The one-launch batched iteration (gradient batches, then Adam chunks that
    wait for their problem's gradient) gives every problem the factors, moments
    and counters of the two-launch iteration (summation order aside), and
    leaves its queue ready for the next launch (repeated iterations)."""
    from paper_1906_01687_gb300.batch import GcpAdamBatch
    g = gcp()
    specs = make_specs(20_000)
    runs = []
    for fused in (False, True):
        run = GcpAdamBatch(specs, tau=5, alpha=0.01, fused=fused)
        run.set_shape(chunks_per_lane=cpl, replica_target=target, max_replicas=maxr)
        for _ in range(6):
            run.iteration()
        torch.cuda.synchronize()
        runs.append(run)
    for i in range(len(specs)):
        a, b = runs[0].factors(i), runs[1].factors(i)
        num = math.sqrt(sum(np.linalg.norm(x - y) ** 2 for x, y in zip(a, b)))
        den = math.sqrt(sum(np.linalg.norm(y) ** 2 for y in a))
        assert num <= 1e-4 * den, (i, num / den)
        s0, s1 = runs[0].states()[i], runs[1].states()[i]
        assert (s0["t"], s0["iter"], s1["status"]) == (s1["t"], s1["iter"], 0) == (6, 6, 0)
        assert all(torch.count_nonzero(x).item() == 0 for x in runs[1].problems[i]["G"])


def test_fused_epochs_in_a_graph():
    from paper_1906_01687_gb300.batch import GcpAdamBatch
    specs = make_specs(5000)
    run = GcpAdamBatch(specs, tau=4, alpha=0.01, fused=True)
    sts = run.fit(max_epochs=3)
    assert all(st["iter"] == 12 and st["status"] == 0 for st in sts)
    assert all(math.isfinite(st["F"]) for st in sts)
