"""Host logic of bench.py that needs no GPU: the recorded DRAM traffic of the
dominant kernel is reported only for the kernel sources and instance it was
measured on, the roofline's peak comes from the measured-peaks file when
there is one, the algorithmic byte counts follow their definition, and the
oracle's multi-threaded gradient equals its one-call gradient."""
import json

import numpy as np

import bench
import oracle

SHAPE = {"lanes": 8, "chunks": 1, "block": 128, "group_draws": 0, "prefetch": 0, "early_draws": 1}


def _record(tmp_path, source_hash):
    path = tmp_path / "traffic.json"
    path.write_text(json.dumps({"source_hash": source_hash, "launch_shape": SHAPE,
                                "dram_bytes_per_launch": 123456.0}))
    return str(path)


def test_traffic_follows_the_kernel_instance(tmp_path):
    path = _record(tmp_path, bench.kernel_source_hash())
    assert bench.recorded_traffic(dict(SHAPE), path) == 123456.0
    # the block size does not change the kernel's code or its DRAM traffic
    assert bench.recorded_traffic(dict(SHAPE, block=256), path) == 123456.0
    # another instance of the kernel: no figure
    for key, other in (("lanes", 16), ("chunks", 2), ("group_draws", 1), ("early_draws", 0)):
        assert bench.recorded_traffic(dict(SHAPE, **{key: other}), path) is None


def test_traffic_needs_the_recorded_sources(tmp_path):
    path = _record(tmp_path, "0" * 16)
    assert bench.recorded_traffic(dict(SHAPE), path) is None
    assert bench.recorded_traffic(dict(SHAPE), str(tmp_path / "missing.json")) is None


def test_peak_from_the_measured_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6651.4, "bf16_tflops": 1900.0}))
    assert bench.peaks() == (6651.4, "measured")


def test_whole_job_rate_counts_every_rank():
    assert bench.whole_job_rate(1000, 4, 2.0) == 2000.0
    assert bench.max_over_ranks(3.5, 1) == 3.5


def test_algorithmic_bytes():
    # a nonzero draw of the 3-way rank-32 tensor: 16-byte record, 3 rows of 32 FP32 gathered and updated
    assert bench.grad_bytes(1, 0, 3, 32, 4) == 16 + 3 * 32 * 8 == 784
    assert bench.grad_bytes(0, 1, 3, 32, 4) == 768
    assert bench.grad_bytes(0, 1, 3, 32, 2) == 3 * 32 * 6
    assert bench.grad_bytes(10, 20, 4, 10, 4, nz_extra=32, zero_extra=5) == 10 * (32 + 320) + 20 * (5 + 320)
    assert bench.adam_bytes((2, 3), 4) == 5 * 4 * 32 and bench.adam_bytes((2, 3), 4, bf16=True) == 5 * 4 * 34


def test_threaded_oracle_gradient_equals_one_call():
    """The all-core CPU baseline's split of the draws over threads gives the
    oracle's gradient and loss estimate (to FP64 summation order)."""
    dims = (7, 6, 5)
    r = np.random.default_rng(1)
    X = oracle.Tensor(dims, dense=r.standard_normal(dims))
    S = oracle.sample(X, oracle.UNIFORM, 0, 1001, 3, 0)
    A = [r.standard_normal((n, 4)) for n in dims]
    one = oracle.grad(dims, A, oracle.GAUSSIAN, S)
    for cores in (2, 3, 8):
        got = bench.oracle_grad_threads(dims, A, oracle.GAUSSIAN, S, cores)
        for a, b in zip(got, one):
            assert np.allclose(a, b, rtol=1e-12, atol=1e-12)
        f = bench.oracle_loss_threads(dims, A, oracle.GAUSSIAN, S, cores)
        assert abs(f - oracle.loss_estimate(dims, A, oracle.GAUSSIAN, S)) <= 1e-12 * abs(f)
    assert bench.host_cores() >= 1


def test_code_hash_ignores_comments_not_code():
    import bench
    base = "int f(int x) {\n    return x + 1;  // one more\n}\n/* a note */\n"
    h = bench.code_hash([base])
    assert bench.code_hash([base.replace("// one more", "// the successor")]) == h
    assert bench.code_hash([base.replace("/* a note */", "/* another\n   note */")]) == h
    assert bench.code_hash([base.replace("    return", "\treturn")]) == h
    assert bench.code_hash([base.replace("x + 1", "x + 2")]) != h
    assert bench.code_hash([base, base]) != h


def test_stratified_call_bytes():
    """The count tensor's call: 32-byte records, ~1.12 hash probes of 8 B per
    zero, 160 B of rows gathered and 160 B updated per draw (rank 10, 4 modes,
    FP32); BF16 rows gather half."""
    import bench
    dims, nnz = (6186, 24, 77, 32), 5_330_673
    omega = 6186 * 24 * 77 * 32
    probes = 1.1 * omega / (omega - nnz)
    fp32 = bench.stratified_call_bytes(dims, nnz, 100_000, 100_000, 10, 4)
    assert abs(fp32 - (100_000 * (32 + 320) + 100_000 * (8 * probes + 320))) < 1e-3
    assert 68.0e6 < fp32 < 68.2e6
    bf16 = bench.stratified_call_bytes(dims, nnz, 100_000, 100_000, 10, 2)
    assert abs((fp32 - bf16) - 200_000 * 4 * 10 * 2) < 1e-3
