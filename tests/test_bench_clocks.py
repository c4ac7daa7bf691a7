"""Host logic of bench.py's clock record: samples are selected by nvidia-smi's
timestamps inside the timed region, and slowdown reasons are reported only
when a sample in the region shows them (the rejection rule for a benchmark
run)."""
import datetime

import bench


def _line(t, sm, reasons=("Not Active",) * 4):
    ts = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    return f"{ts}, 0, {sm}, 2070, 180.5, 0x0, " + ", ".join(reasons)


def test_samples_inside_the_region_only():
    t0 = 1_800_000_000.0
    lines = [_line(t0 - 0.10, 1000), _line(t0 + 0.01, 2070), _line(t0 + 0.05, 2070), _line(t0 + 0.50, 900)]
    s = bench.clock_summary(lines, t0, t0 + 0.10)
    assert s["samples_in_region"] == 2 and s["samples"] == 2
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == []


def test_slowdown_reasons_and_fallback_to_last_sample():
    t0 = 1_800_000_000.0
    hot = ("Not Active", "Active", "Not Active", "Active")      # hw_thermal_slowdown, sw_power_cap
    lines = ["garbage line", _line(t0 + 0.02, 1500, hot)]
    s = bench.clock_summary(lines, t0, t0 + 0.05)
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"] and s["sm_mhz"] == 1500.0
    # nothing inside the interval: the last sample stands in, and says so
    s = bench.clock_summary(lines, t0 + 1.0, t0 + 2.0)
    assert s["samples_in_region"] == 0 and s["samples"] == 1
    assert bench.clock_summary(["no samples"], t0, t0 + 1.0) is None
