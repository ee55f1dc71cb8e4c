"""The clock record of bench.py on the host: which samples count for the timed
region, and how the slowdown reasons and the SM clock are summarised."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_samples_inside_the_window_only():
    rows = [(0.5, 900.0, 2070.0, {"sw_thermal_slowdown"}),      # before: ignored
            (1.0, 2070.0, 2070.0, set()),
            (1.1, 2040.0, 2070.0, {"sw_power_cap"}),
            (1.2, 2055.0, 2070.0, set()),
            (2.5, 1000.0, 2070.0, {"hw_slowdown"})]              # after: ignored
    c = bench.summarize_clocks(rows, 0.9, 1.3, "test")
    assert c["samples"] == 3 and c["in_window"]
    assert c["sm_mhz"] == 2055.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"]


def test_nearest_samples_stand_in_for_a_short_window():
    rows = [(0.5, 2000.0, 2070.0, set()), (0.8, 1990.0, 2070.0, set()),
            (1.5, 2010.0, 2070.0, {"hw_thermal_slowdown"})]
    c = bench.summarize_clocks(rows, 1.0, 1.02, "test")
    assert c["samples"] == 2 and not c["in_window"]
    assert c["sm_mhz"] == 2000.0
    assert c["reasons"] == ["hw_thermal_slowdown"]


def test_no_samples():
    c = bench.summarize_clocks([], 1.0, 2.0, "test")
    assert c["sm_mhz"] is None and c["samples"] == 0 and not c["in_window"]


def test_reason_bits_are_distinct_and_named():
    bits = bench._NVML_REASON_BITS
    assert set(bits) == set(bench.CLOCK_REASONS)
    vals = list(bits.values())
    assert all(v & (v - 1) == 0 for v in vals) and len(set(vals)) == len(vals)
