"""The N-rank benchmark path on CPU: two gloo ranks (127.0.0.1), each a
replica with its own seeds, timing reduced to the slowest rank, whole-job
rate over all ranks; the reference arm does no work on ranks other than 0."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, _ = bench.dist_env()
        seconds = bench.max_over_ranks(1.0 + rank, w)        # rank 1 is the slower one
        rate = bench.whole_job_rate(1000, w, seconds)
        seeds = bench.replica_seeds(r)
        out.put((rank, seconds, rate, seeds))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_benchmark():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, seconds, rate, seeds in res:
        assert seconds == 2.0            # max over ranks
        assert rate == 1000 * 2 / 2.0    # all ranks' units / slowest time
    assert res[0][3] != res[1][3]        # each replica has its own seeds


def test_reference_arm_is_rank0_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        steps, warmup, gpus = 1, 3, 2
    assert bench.reference_arm(A()) == 0


def test_reference_arm_line_keeps_the_contract(monkeypatch, capsys):
    """Rank 0 prints one JSON line with the arm's keys; the input and the
    oracle's timing are replaced by stand-ins here (the line's assembly is
    what is checked)."""
    import json
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    monkeypatch.setattr(bench, "large_input", lambda init_seed=3: (None, None, None))
    monkeypatch.setattr(bench, "oracle_large_tensor", lambda idx: None)
    monkeypatch.setattr(bench, "oracle_epoch_rate",
                        lambda XO, A0, cores, iters=1, seed=1687: (2.0e6, "a bounded sample"))

    class A:
        steps, warmup, gpus = 2, 3, 1
    assert bench.reference_arm(A()) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] == 2.0e6 and line["higher_is_better"] is True
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT and line["dtype"] == "f64"
    assert line["steps"] == 2 and line["warmup"] == 3 and line["n_gpus"] == 1
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == bench.host_cores()
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": 2.0e6, "unit": bench.UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert line["config"]["workload"] == bench.WORKLOAD
