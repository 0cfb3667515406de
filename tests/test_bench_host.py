"""Host logic of bench.py that needs no GPU: the clock-sample summary that
decides whether a timed run is kept, and the lookup of the recorded DRAM
traffic of the product kernel."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _line(sm, mx, hw="Not Active", thermal="Not Active", sw_thermal="Not Active", cap="Not Active"):
    return "0, %d, %d, 640.0, 0x0, %s, %s, %s, %s\n" % (sm, mx, hw, thermal, sw_thermal, cap)


def test_clock_summary_median_and_reasons():
    lines = [_line(2070, 2070), _line(1900, 2070, cap="Active"), _line(2070, 2070),
             "garbage line\n", _line(2000, 2070, thermal="Active")]
    s = bench.parse_clock_samples(lines)
    assert s["samples"] == 4
    assert s["sm_mhz"] == 2035.0                 # median of 2070, 1900, 2070, 2000
    assert s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


def test_clock_summary_without_samples():
    assert bench.parse_clock_samples([]) is None
    assert bench.parse_clock_samples(["[N/A], [N/A]\n"]) is None


def test_traffic_record_matches_workload_only():
    d = bench._traffic("fp64", bench.WORKLOAD["workload"])
    with open(os.path.join(ROOT, "profiles", "filter_traffic_fp64.txt")) as f:
        rec = json.load(f)
    assert d == rec
    Np = 50048
    assert d["bytes_per_launch"] > 24 * Np * Np       # at least the slices of H
    assert bench._traffic("fp64", "chase_N20000_nev100_nex40") is None
    assert bench._traffic("nonexistent", bench.WORKLOAD["workload"]) is None


def test_projected_solve_time():
    """cpu_baseline projection: build + per-column product time x products +
    iterations x (QR + Rayleigh-Ritz)."""
    smp = dict(t_build=4.0, t_mv=0.05, t_qr=1.0, t_rr=0.5)
    assert bench.project_solve(smp, dict(iters=8, matvecs=47231)) == \
        4.0 + 0.05 * 47231 + 8 * 1.5
