"""The sample-parallel split of one problem (paper_1906_01687_gb300/parallel.py)
on CPU: draw ranges partition the draw counter, and two gloo ranks that each
compute the oracle's gradient of their own range and sum the flat gradients
with the module's collective get the single-rank oracle gradient (FP64 sum
order aside), for uniform, stratified and semi-stratified draws."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
torch = pytest.importorskip("torch")


def test_draw_ranges_partition_the_counter():
    from paper_1906_01687_gb300.parallel import draw_range
    for n in (0, 1, 7, 1000, 2_000_001):
        for world in (1, 2, 3, 8):
            got = [draw_range(r, world, n) for r in range(world)]
            assert got[0][0] == 0 and sum(c for _, c in got) == n
            for (f0, c0), (f1, _) in zip(got, got[1:]):
                assert f0 + c0 == f1
            assert max(c for _, c in got) - min(c for _, c in got) <= 1
    with pytest.raises(ValueError):
        draw_range(2, 2, 10)


def test_flat_buffers_are_one_allocation_with_aligned_views():
    from paper_1906_01687_gb300.parallel import flat_buffers
    flat, views = flat_buffers((5, 3, 7), 8, device="cpu")
    assert flat.numel() == 15 * 8 and [v.shape for v in views] == [(5, 8), (3, 8), (7, 8)]
    views[1][2, 3] = 4.0
    assert flat[5 * 8 + 2 * 8 + 3] == 4.0
    assert all(v.data_ptr() % 16 == 0 for v in views)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem(kind):
    import oracle
    r = np.random.default_rng(5)
    dims = (9, 8, 7)
    if kind == "uniform":
        X = oracle.Tensor(dims, dense=r.standard_normal(dims))
        return X, dims, oracle.UNIFORM, 0, 601, oracle.GAUSSIAN
    keys = r.choice(int(np.prod(dims)), 60, replace=False)
    coo = np.stack(np.unravel_index(keys, dims), axis=1)
    X = oracle.Tensor(dims, coo=coo, vals=None)
    kind_id = oracle.STRATIFIED if kind == "stratified" else oracle.SEMI_STRATIFIED
    return X, dims, kind_id, 211, 390, oracle.BERNOULLI_LOGIT


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import oracle
    from paper_1906_01687_gb300.parallel import draw_range, flat_buffers, sum_across_ranks
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        for kind in ("uniform", "stratified", "semi"):
            X, dims, sampler, p, q, loss = _problem(kind)
            A = [np.random.default_rng(9 + k).standard_normal((n, 5)) * 0.4 for k, n in enumerate(dims)]
            S = oracle.sample(X, sampler, p, q, 17, 3)
            first, count = draw_range(dist.get_rank(), dist.get_world_size(), S.n)
            mine = oracle.Samples(S.idx[first:first + count], S.x[first:first + count], S.w[first:first + count],
                                  S.cls[first:first + count])
            part = oracle.grad(dims, A, loss, mine)
            flat, views = flat_buffers(dims, 8, device="cpu", dtype=torch.float64)
            for v, g in zip(views, part):
                v[:, :5] = torch.from_numpy(g)
            sum_across_ranks(flat)
            full = oracle.grad(dims, A, loss, S)
            err = max(float(np.abs(v[:, :5].numpy() - g).max() / max(np.abs(g).max(), 1e-300))
                      for v, g in zip(views, full))
            pad = max(float(v[:, 5:].abs().max()) for v in views)
            out.put((rank, kind, err, pad, count))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_sum_to_the_single_rank_gradient():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
        assert p.exitcode == 0
    res = [q.get(timeout=10) for _ in range(6)]
    counts = {}
    for rank, kind, err, pad, count in res:
        assert err <= 1e-12, (rank, kind, err)
        assert pad == 0.0
        counts.setdefault(kind, 0)
        counts[kind] += count
    assert counts == {"uniform": 601, "stratified": 601, "semi": 601}
