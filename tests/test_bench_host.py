"""Host logic of bench.py that needs no GPU: the recorded DRAM traffic of the
dominant kernel is reported only for the kernel sources and instance it was
measured on, and the roofline's peak comes from the measured-peaks file when
there is one."""
import json

import bench


def recorded():
    with open(bench.TRAFFIC_FILE) as f:
        return json.load(f)


def test_traffic_follows_the_kernel_instance():
    rec = recorded()
    launch = dict(rec["launch_shape"])
    expected = rec["dram_bytes_per_launch"] if rec["source_hash"] == bench.kernel_source_hash() else None
    assert bench.recorded_traffic(launch) == expected
    # the block size does not change the kernel's code or its DRAM traffic
    assert bench.recorded_traffic(dict(launch, block=launch.get("block", 128) * 2)) == expected
    # another instance of the kernel: no figure
    for key, other in (("lanes", launch["lanes"] * 2), ("chunks", launch["chunks"] + 1),
                       ("group_draws", 1 - launch["group_draws"]), ("early_draws", 1 - launch["early_draws"])):
        assert bench.recorded_traffic(dict(launch, **{key: other})) is None


def test_traffic_needs_the_recorded_sources(monkeypatch):
    rec = recorded()
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench.recorded_traffic(dict(rec["launch_shape"])) is None


def test_peak_from_the_measured_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6651.4, "bf16_tflops": 1900.0}))
    assert bench.peaks() == (6651.4, "measured")


def test_whole_job_rate_counts_every_rank():
    assert bench.whole_job_rate(1000, 4, 2.0) == 2000.0
    assert bench.max_over_ranks(3.5, 1) == 3.5
