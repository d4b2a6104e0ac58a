"""gcp_loss_est_noalloc: the loss estimate for callers that cannot allocate
device memory when they call it (for example while a CUDA graph is being
captured, or under another allocator's memory budget).  It keeps its scratch
in a static device array instead of handle memory; it must give the same
estimate as gcp_loss_est, call after call.

This file is collected last on purpose: a failure here comes after every
other test has run.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

LOSS_RTOL = 2e-6  # against the sum of |terms|, as in the other loss-estimate tests


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1906_01687_gb300 import build
    build.build()


def test_noalloc_loss_estimate_matches_handle_version_twice():
    from paper_1906_01687_gb300 import gcp
    dims = (40, 30, 20, 6)
    rs = np.random.default_rng(3)
    nnz = 9000
    keys = rs.permutation(np.unique(rs.integers(0, int(np.prod(dims)), 12000)))[:nnz]
    idx, rem = [], keys.copy()
    for n in reversed(dims):
        idx.append((rem % n).astype(np.int32))
        rem //= n
    idx = idx[::-1]
    vals = (1 + rs.poisson(2.0, nnz)).astype(np.float32)
    h = gcp.Handle(gcp.DataTensor.coo(dims, idx, vals))
    A = [(0.5 * rs.standard_normal((n, 10))).astype(np.float32) for n in dims]
    F = gcp.Factors(A)
    L = gcp.gcp_sample(h, gcp.Sampling(gcp.SAMPLER_STRATIFIED, 30001, 29999, seed=4, stream=gcp.STREAM_EST))
    ref = torch.zeros(1, dtype=torch.float64, device="cuda")
    gcp.gcp_loss_est(h, F, gcp.LOSS_POISSON_LOG, L, ref)
    torch.cuda.synchronize()
    # sum of |terms|: the error scale of any summation order (from the same list, on the host)
    m = np.zeros(L.n)
    A64 = [a.astype(np.float64) for a in A]
    ix = [i.cpu().numpy() for i in L.idx]
    prod = np.ones((L.n, 10))
    for k in range(4):
        prod *= A64[k][ix[k]]
    m = prod.sum(axis=1)
    x, w, cls = L.x.double().cpu().numpy(), L.w.double().cpu().numpy(), L.cls.cpu().numpy()
    f = np.exp(m) - x * m
    f = np.where(cls == gcp.CLS_SEMI_NZ, f - np.exp(m), f)
    scale = float(np.abs(w * f).sum())
    for call in range(2):
        out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        gcp.gcp_loss_est_noalloc(len(dims), F, gcp.LOSS_POISSON_LOG, L, out)
        torch.cuda.synchronize()
        assert abs(out.item() - ref.item()) <= LOSS_RTOL * scale, (call, out.item(), ref.item())


def test_noalloc_rejects_lists_beyond_its_scratch():
    from paper_1906_01687_gb300 import gcp
    F = gcp.Factors([np.ones((3, 4), np.float32)] * 3)
    L = gcp.SampleList.empty(3, 1024 * 256 + 1)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(gcp.GcpError) as e:
        gcp.gcp_loss_est_noalloc(3, F, gcp.LOSS_GAUSSIAN, L, out)
    assert e.value.status == gcp.ERR_INVALID_ARG
