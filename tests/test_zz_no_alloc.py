"""gcp_loss_est_noalloc: the loss estimate for callers that must not allocate
device memory when they run it (a host whose GPU memory belongs to another
allocator, a loop that forbids allocation after start-up).  It keeps its
scratch in a static device array instead of handle memory; call after call
it must give the FP64 oracle's estimate and the handle version's.

This file is collected last on purpose: a failure here comes after every
other test has run.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

LOSS_RTOL = 2e-6  # against the sum of |terms|, as in the other loss-estimate tests


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1906_01687_gb300 import build
    build.build()


def _count_tensor(dims, nnz, seed):
    rs = np.random.default_rng(seed)
    keys = rs.permutation(np.unique(rs.integers(0, int(np.prod(dims)), nnz + nnz // 3)))[:nnz]
    idx, rem = [], keys.copy()
    for n in reversed(dims):
        idx.append((rem % n).astype(np.int32))
        rem //= n
    idx = idx[::-1]
    vals = (1 + rs.poisson(2.0, nnz)).astype(np.float32)
    return idx, vals, rs


def test_noalloc_loss_estimate_matches_oracle_and_handle_version_twice():
    from paper_1906_01687_gb300 import gcp
    dims = (40, 30, 20, 6)
    idx, vals, rs = _count_tensor(dims, 9000, 3)
    h = gcp.Handle(gcp.DataTensor.coo(dims, idx, vals))
    A = [(0.5 * rs.standard_normal((n, 10))).astype(np.float32) for n in dims]
    F = gcp.Factors(A)
    spec = gcp.Sampling(gcp.SAMPLER_STRATIFIED, 30001, 29999, seed=4, stream=gcp.STREAM_EST)
    L = gcp.gcp_sample(h, spec)
    ref = torch.zeros(1, dtype=torch.float64, device="cuda")
    gcp.gcp_loss_est(h, F, gcp.LOSS_POISSON_LOG, L, ref)
    torch.cuda.synchronize()
    # the FP64 oracle on the same draws (its sampler gives the same list bit for bit)
    XO = oracle.Tensor(dims, coo=np.stack([i.astype(np.int64) for i in idx], axis=1), vals=vals.astype(np.float64))
    SO = oracle.sample(XO, oracle.STRATIFIED, 30001, 29999, 4, gcp.STREAM_EST)
    A64 = [a.astype(np.float64) for a in A]
    F_orc = oracle.loss_estimate(dims, A64, oracle.POISSON_LOG, SO)
    scale = oracle.loss_abs(dims, A64, oracle.POISSON_LOG, SO)
    for call in range(2):
        out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        gcp.gcp_loss_est_noalloc(len(dims), F, gcp.LOSS_POISSON_LOG, L, out)
        torch.cuda.synchronize()
        got = out.item()
        assert abs(got - F_orc) <= LOSS_RTOL * scale, (call, got, F_orc)
        assert abs(got - ref.item()) <= LOSS_RTOL * scale, (call, got, ref.item())


def test_noalloc_rejects_lists_beyond_its_scratch_and_one_mode():
    from paper_1906_01687_gb300 import gcp
    F = gcp.Factors([np.ones((3, 4), np.float32)] * 3)
    L = gcp.SampleList.empty(3, 1024 * 256 + 1)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(gcp.GcpError) as e:
        gcp.gcp_loss_est_noalloc(3, F, gcp.LOSS_GAUSSIAN, L, out)
    assert e.value.status == gcp.ERR_INVALID_ARG
    # one mode: no tensor of the library has a single mode
    F1 = gcp.Factors([np.ones((3, 4), np.float32)])
    with pytest.raises(gcp.GcpError) as e:
        gcp.gcp_loss_est_noalloc(1, F1, gcp.LOSS_GAUSSIAN, gcp.SampleList.empty(1, 8), out)
    assert e.value.status == gcp.ERR_INVALID_ARG
