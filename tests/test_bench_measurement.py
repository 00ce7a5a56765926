"""Host logic of the benchmark's measurement (bench.py, no GPU): the roofline
of the dominant kernel class (binding roof, peaks, traffic, L2 residency) and
the clock sampler's reading of nvidia-smi samples (median clock, throttle
reasons that reject a run)."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _peaks():
    """The measured peaks bench.py reads, with its fallbacks when the file
    (written per GPU pool) is absent."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
    except OSError:
        p = {}
    return {"hbm_gbs": p.get("hbm_gbs", 6800.0), "sm_max_mhz": p.get("sm_max_mhz", 2070.0)}


def test_every_timer_class_has_roofline_info():
    # every timed class, and the Gram-Schmidt projection formed from two of them
    assert set(bench.CLASS_INFO) == set(bench.TIMER_NAMES) | {"gram_schmidt"}
    for name, arith, sms in bench.CLASS_INFO.values():
        assert arith in ("fp32", "fp64") and 1 <= sms <= 152 and name


def test_fp64_class_is_bound_by_the_derived_fp64_peak():
    p = _peaks()
    # 436 launches, 10 ms, 50 MB and 12 MFLOP each: arithmetic binds
    launches, ms = 436, 10.0
    r = bench.roofline_for("dot", ms, launches, 50e6 * launches, 12e6 * launches)
    peak = 152 * 2 * 2 * p["sm_max_mhz"] * 1e6 / 1e9
    assert r["bound"] == "alu" and r["unit"] == "GFLOP/s"
    assert r["peak"] == pytest.approx(peak)
    avg_s = ms * 1e-3 / launches
    assert r["achieved"] == pytest.approx(12e6 / avg_s / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / peak)
    assert r["other_roof"]["unit"] == "GB/s" and r["other_roof"]["peak"] == pytest.approx(p["hbm_gbs"])
    # traffic from the committed ncu ratio, per launch like achieved (null
    # while the kernel has changed since its counters were taken)
    if "dot" in bench.TRAFFIC_RATIO:
        assert r["traffic"] == pytest.approx(bench.TRAFFIC_RATIO["dot"] * 50e6)
    else:
        assert r["traffic"] is None
    # a 50 MB working set per launch fits the L2
    assert "resident" in r


def test_streaming_class_is_bound_by_measured_hbm():
    p = _peaks()
    # 20 launches of 535 MB each at 0.15 ms: bytes bind, no L2 label, no
    # traffic figure for a class without a committed capture
    launches = 20
    r = bench.roofline_for("matvec", 0.15 * launches, launches, 535e6 * launches, 2e7 * launches)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(535e6 / 0.15e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / p["hbm_gbs"])
    assert "resident" not in r
    assert r["traffic"] is None
    assert r["alg_bytes_per_launch"] == pytest.approx(535e6)


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _sampler_with(tmp_path, rows):
    path = tmp_path / "clocks.csv"
    path.write_text("".join(", ".join(r) + "\n" for r in rows))
    s = bench.ClockSampler(0)
    s.proc = _FakeProc()
    s.path = str(path)
    return s


def test_clock_sampler_reports_median_and_no_reasons(tmp_path):
    idle = "Not Active"
    rows = [["0", str(mhz), "2070", "900.0", "0x0", idle, idle, idle, idle] for mhz in (2070, 2055, 2070, 1980, 2070)]
    out = _sampler_with(tmp_path, rows).stop()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == [] and out["samples"] == 5


def test_clock_sampler_flags_throttle_reasons(tmp_path):
    idle, act = "Not Active", "Active"
    rows = [["0", "2070", "2070", "1390.0", "0x4", idle, idle, idle, act],
            ["0", "1800", "2070", "1400.0", "0x48", idle, act, idle, act],
            ["0", "2070", "2070", "1000.0", "0x0", idle, idle, idle, idle]]
    out = _sampler_with(tmp_path, rows).stop()
    assert out["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert out["sm_mhz"] == 2070.0
