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


def test_traffic_record_is_used_only_for_the_captured_source(tmp_path, monkeypatch):
    """roofline.traffic comes from a committed ncu summary row
    (kernel | workload | precision | bytes per launch | source sha16) and is
    dropped once the kernel source no longer has the captured hash."""
    import hashlib
    src = tmp_path / "paper_1203_6402_gb300" / "csrc"
    src.mkdir(parents=True)
    (src / "nearest_tc_kernel.cuh").write_bytes(b"kernel v1")
    sha = hashlib.sha256(b"kernel v1").hexdigest()[:16]
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.md").write_text(
        "| kernel | workload | precision | bytes | sha |\n|---|---|---|---|---|\n"
        f"| tc::nearest_tc_kernel (assign) | w1 | bf16 | 1.5e9 | {sha} |\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_record("tc::nearest_tc_kernel (assign)", "w1", "bf16") == (1.5e9, sha)
    assert bench.traffic_record("tc::nearest_tc_kernel (round)", "w1", "bf16") == (None, None)
    (src / "nearest_tc_kernel.cuh").write_bytes(b"kernel v2")
    assert bench.traffic_record("tc::nearest_tc_kernel (assign)", "w1", "bf16") == (None, sha)


def test_oracle_sample_keeps_points_per_cluster():
    import argparse
    a = argparse.Namespace(workload="gmm_n10M_d128_k10000", n=0, ell_factor=0, cpu_sample_n=50000,
                           cpu_lloyd_iters=10)
    assert bench.oracle_sample(a) == dict(n=50000, k=50, ell=100.0, rounds=5, lloyd=10)
    a = argparse.Namespace(workload="gmm_n10k_d15_k50", n=0, ell_factor=0, cpu_sample_n=50000,
                           cpu_lloyd_iters=10)
    assert bench.oracle_sample(a) == dict(n=10000, k=50, ell=100.0, rounds=5, lloyd=10)


def test_default_precision_by_dimension():
    assert bench.default_precision("kdd_n1M_d42_k500") == "bf16x3"
    assert bench.default_precision("gmm_n10M_d128_k10000") == "bf16"
