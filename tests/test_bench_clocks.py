"""The benchmark's clock record: samples parsed from nvidia-smi's CSV lines,
throttle reasons collected, and the samples inside the timed region counted
apart from those of the loaded window around it."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_clock_summary_counts_timed_samples_and_reasons():
    c = bench.ClockSampler(0)
    c.lines = [
        (0.0, "2070, 2070, 900.1, Not Active, Not Active, Not Active, Not Active"),
        (1.0, "2040, 2070, 1350.0, Not Active, Not Active, Not Active, Active"),
        (1.1, "2055, 2070, 1320.0, Not Active, Not Active, Not Active, Not Active"),
        (2.0, "[N/A], 2070, 10.0, Not Active, Not Active, Not Active, Not Active"),
        (3.0, "truncated"),
    ]
    c.t_start, c.t_end = 0.5, 1.5
    s = c.summary()
    assert s["samples"] == 3
    assert s["samples_timed"] == 2
    assert s["sm_mhz"] == 2055.0
    assert s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]


def test_clock_summary_without_samples():
    s = bench.ClockSampler(0).summary()
    assert s["sm_mhz"] is None and s["samples"] == 0 and s["samples_timed"] == 0
