"""Host-side logic of the benchmark: the clock record counts only samples from the timed region."""
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
