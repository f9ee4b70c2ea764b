"""Host-side pieces of bench.py on the CPU: the clock-sample summary (median
SM clock, the throttle reasons that reject a run), the traffic record lookup
keyed by the kernel sources, the peak file fallback, and the oracle timing
used by the CPU baseline."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_clock_summary_reports_median_and_active_reasons():
    cs = bench.ClockSampler(0)
    cs.lines = ["2070, 2070, Not Active, Not Active, Not Active, Not Active",
                "1980, 2070, Not Active, Not Active, Not Active, Active",
                "2070, 2070, Not Active, Not Active, Not Active, Not Active",
                "garbage line",
                "1500, 2070, Active, Not Active, Not Active, Not Active"]
    s = cs.summary()
    assert s["samples"] == 4 and s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap"]
    empty = bench.ClockSampler(0)
    assert empty.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_traffic_record_follows_the_kernel_sources(tmp_path, monkeypatch):
    n = 384 * 96 * 96
    got = bench.recorded_traffic("c2", "fp32", "pair", n)
    rec = json.load(open(os.path.join(ROOT, "profiles", "step_kernel_traffic.json")))
    if rec["source_hash"] == bench.kernel_source_hash():
        assert got == pytest.approx(rec["entries"]["c2_fp32_pair"]["bytes_per_cell"] * n)
    else:
        assert got is None
    assert bench.recorded_traffic("c3", "fp32", "pair", n) is None        # no entry: null
    # a record for other kernel sources is not used
    fake = tmp_path / "profiles"
    fake.mkdir()
    rec["source_hash"] = "0" * 16
    (fake / "step_kernel_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "f" * 16)
    assert bench.recorded_traffic("c2", "fp32", "pair", n) is None


def test_peaks_fall_back_when_the_file_is_absent(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    peaks, kind = bench.measured_peaks()
    assert kind == "fallback" and peaks["hbm_gbs"] == 6800.0


def test_cpu_baseline_times_the_oracle():
    cfg = dict(bench.CONFIGS["c1"])
    m, thr, sample, dt, n = bench.cpu_oracle_mlups(cfg, steps=2, nz_sample=4)
    assert m > 0 and thr >= 1 and n == 2 and dt > 0 and "64x32x4" in sample
