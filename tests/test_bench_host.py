"""Host-side logic of the benchmark: the clock record counts only samples from the timed region,
and the committed DRAM-traffic record applies only to its own workload and kernel source."""
import json

import bench


def test_clock_summary_uses_timed_region_samples():
    c = bench.ClockSampler(0)
    idle = "0, 345, 2070, 80.0, 0x0, Not Active, Not Active, Not Active, Not Active"
    busy = "0, 2070, 2070, 900.0, 0x4, Not Active, Not Active, Not Active, Active"
    c.lines = [idle, idle, busy, busy, busy]
    c.first = 2
    s = c.summary()
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "samples": 3, "reasons": ["sw_power_cap"]}
    c.first = 5                     # no sample inside the region: the last one stands in
    assert c.summary()["samples"] == 1
    c.lines = []
    assert c.summary() is None


def test_traffic_record_applies_to_its_workload_and_source_only(tmp_path, monkeypatch):
    rec = {"workload": bench.workload("splash").name, "kernel_hash": bench.kernel_hash(), "dram_bytes_per_lu": 117.5}
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_hash", lambda: rec["kernel_hash"])
    splash, large = bench.workload("splash"), bench.workload("large")
    assert bench.traffic_per_launch(splash) == 117.5 * splash.cells
    assert bench.traffic_per_launch(large) is None                 # another workload
    monkeypatch.setattr(bench, "kernel_hash", lambda: "changed")
    assert bench.traffic_per_launch(splash) is None                # another kernel source
    # the committed form: one record per profiled workload
    big = dict(rec, workload=large.name, dram_bytes_per_lu=150.8)
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps([rec, big]))
    monkeypatch.setattr(bench, "kernel_hash", lambda: rec["kernel_hash"])
    assert bench.traffic_per_launch(splash) == 117.5 * splash.cells
    assert bench.traffic_per_launch(large) == 150.8 * large.cells
