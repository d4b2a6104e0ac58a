"""GCP-Adam iterations whose Adam step (Alg. 4) is taken by the gradient
kernel's last blocks (gcp_tuning.tail_work = 1, small factor sets) against
the same iterations with a separate Adam launch (tail_work = 0, the
default): the same draws, the same replica fold order and the same
elementwise update, so the factors agree to the FP32 rounding of the
gradient's accumulation order, and the step and iteration counters exactly.
"""
import numpy as np
import pytest

from gpu_util import gcp, rel_norm, rng_factors, sparse_random

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1906_01687_gb300 import build
    build.build()


def run(make, tail_work, epochs, graph):
    g = gcp()
    r = make()
    g.gcp_set_tuning(r.h, early_draws=1, tail_work=tail_work)
    if graph:
        r.capture()
    for _ in range(epochs):
        r.run_epoch()
    st = r.status()
    assert st["status"] == 0 and g.gcp_get_device_status(r.h) == 0
    return r.factors(), st


@pytest.mark.parametrize("graph", [False, True])
def test_dense_uniform_adam_in_the_gradient_kernel(graph):
    from paper_1906_01687_gb300.adam import GcpAdam
    g = gcp()
    dims = (30, 20, 10, 8)
    X = np.random.default_rng(60).standard_normal(dims).astype(np.float32)
    A0 = rng_factors(dims, 6, 61, scale=0.5)

    def make():
        return GcpAdam(g.DataTensor.dense(X), A0, g.LOSS_GAUSSIAN, g.SAMPLER_UNIFORM, 0, 5000, 0, 2000, seed=7,
                       est_seed=8, alpha=1e-2, tau=15)
    r0 = make()
    g.gcp_set_tuning(r0.h, early_draws=1, tail_work=1)
    assert g.gcp_get_launch(r0.h, r0.F, 5000)["adam_tail_blocks"] > 0
    f0, s0 = run(make, 1, 3, graph)
    f1, s1 = run(make, 0, 3, graph)
    assert (s0["t"], s0["iter"], s0["bad"]) == (s1["t"], s1["iter"], s1["bad"]) and s0["iter"] == 45
    assert rel_norm(f0, f1) <= 1e-5
    assert abs(s0["F"] - s1["F"]) <= 1e-5 * abs(s1["F"])


def test_stratified_adam_in_the_gradient_kernel_bf16():
    """Zeros made in the launch, BF16 rows (the step writes the BF16 copy),
    nonnegativity: the same run either way."""
    from paper_1906_01687_gb300.adam import GcpAdam
    g = gcp()
    dims = (40, 30, 20)
    idx, vals = sparse_random(dims, 3000, 62)
    A0 = rng_factors(dims, 5, 63, scale=0.5, positive=True)

    def make():
        return GcpAdam(g.DataTensor.coo(dims, idx, vals), A0, g.LOSS_POISSON_LOG, g.SAMPLER_STRATIFIED, 2000, 2000,
                       3000, 3000, seed=9, est_seed=10, alpha=1e-2, tau=10, lower=0.0, bf16=True)
    f0, s0 = run(make, 1, 3, True)
    f1, s1 = run(make, 0, 3, True)
    assert (s0["t"], s0["iter"], s0["bad"]) == (s1["t"], s1["iter"], s1["bad"])
    assert rel_norm(f0, f1) <= 1e-5
    assert all((a >= 0).all() for a in f0)
