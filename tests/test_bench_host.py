"""bench.py host logic without a GPU: the nvidia-smi clock summary (median SM clock under load,
max clock, throttle reasons that were Active, never 'Not Active')."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _summary(rows):
    c = bench.ClockSampler(0)
    c.samples = [[x.strip() for x in r.split(",")] for r in rows]
    return c.stop()


def test_clock_summary_reasons_and_median():
    s = _summary(["2070, 2070, 950.1, Not Active, Not Active, Not Active, Not Active",
                  "1980, 2070, 1399.0, Not Active, Not Active, Not Active, Active",
                  "2070, 2070, 1012.5, Not Active, Not Active, Not Active, Not Active"])
    assert s["sm_mhz"] == 2070 and s["sm_max_mhz"] == 2070 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]


def test_clock_summary_thermal_and_empty():
    s = _summary(["1500, 2070, 1300, Active, Not Active, Active, Not Active"])
    assert s["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    e = _summary([])
    assert e["sm_mhz"] is None and e["reasons"] == [] and e["samples"] == 0
