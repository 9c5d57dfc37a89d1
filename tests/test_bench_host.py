"""Host-side logic of bench.py that decides whether a timed run is valid and how
much work it did, checked on the CPU: the clock record parsed from nvidia-smi's
CSV (median SM clock, maximum, throttle reasons) and the algorithmic
dist-evals of a step."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _line(sm, mx=2070, active="0x0000000000000000", hw="Not Active", hwt="Not Active", swt="Not Active",
          cap="Not Active"):
    return f"0, {sm}, {mx}, 812.45, {active}, {hw}, {hwt}, {swt}, {cap}"


def test_clock_record_median_max_and_no_reason():
    out = "\n".join([_line(2070), _line(1965), _line(2070), _line(2055)])
    rec = bench.ClockSampler.parse(out)
    assert rec == {"sm_mhz": 2062.5, "sm_max_mhz": 2070.0, "reasons": [], "samples": 4}


def test_clock_record_collects_throttle_reasons():
    out = "\n".join([_line(2070), _line(1500, cap="Active"), _line(1400, hwt="Active"), _line(2070)])
    rec = bench.ClockSampler.parse(out)
    assert rec["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"] and rec["samples"] == 4
    assert rec["sm_mhz"] == 1785.0


def test_clock_record_skips_malformed_lines():
    out = "\n".join(["", "garbage", "0, [N/A], 2070, 1, 0, Not Active, Not Active, Not Active, Not Active",
                     _line(2070)])
    rec = bench.ClockSampler.parse(out)
    assert rec["samples"] == 1 and rec["sm_mhz"] == 2070.0
    assert bench.ClockSampler.parse("") is None


def test_dist_evals_of_a_step():
    """init n; each round n |C'_i|; recluster k m; Lloyd n k per assignment
    (iterations + 1 assignments, the first with the seed centers)."""
    stats = {"round_added": [1000, 999, 1001, 1000, 1000], "m": 5001}
    total, parts = bench.count_dist_evals(10, 7, stats, 3)
    assert parts == {"init": 10, "rounds": 10 * 5000, "recluster": 7 * 5001, "lloyd": 4 * 10 * 7}
    assert total == sum(parts.values())
