"""Host logic of bench.py that the benchmark line rests on (no GPU): the clock record kept for the
timed region, and the traffic record's validity rule."""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _line(sm, reason_power="Not Active", reason_thermal="Not Active"):
    return f"0, {sm}, 2032, 900, 0x0, Not Active, {reason_thermal}, Not Active, {reason_power}"


def test_clock_record_keeps_the_timed_region_only():
    c = bench.ClockSampler(0)
    t = time.monotonic()
    c.lines = [(t - 2.0, _line(600)),                              # idle, before the warm-up
               (t - 1.0, _line(1200, reason_thermal="Active")),    # warm-up: a slowdown outside the window
               (t + 0.05, _line(2032)), (t + 0.15, _line(1990, reason_power="Active")), (t + 0.25, _line(2010)),
               (t + 5.0, _line(700))]                              # after the timed region
    c.window = [t, t + 0.3]
    s = c.summary()
    assert s["samples"] == 3 and s["sm_mhz"] == 2010 and s["sm_max_mhz"] == 2032
    assert s["reasons"] == ["sw_power_cap"]                        # the warm-up's slowdown is not reported


def test_clock_record_of_a_window_shorter_than_one_period_takes_the_nearest_samples():
    c = bench.ClockSampler(0)
    t = time.monotonic()
    c.lines = [(t - 2.0, _line(600)), (t - 0.15, _line(2000)), (t + 0.25, _line(2032))]
    c.window = [t, t + 0.02]                                       # no sample inside the window
    s = c.summary()
    assert s["samples"] == 2 and s["sm_mhz"] == 2016                 # the idle sample 2 s before is left out


def test_clock_record_without_samples_says_unavailable():
    c = bench.ClockSampler(0)
    assert c.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}


def test_traffic_record_counts_only_for_the_kernel_source_it_was_taken_on(tmp_path, monkeypatch):
    rec = {"kernel_source_sha256_16": bench.fused_source_hash(), "dram_bytes_per_full_launch": 8.4e9}
    p = tmp_path / "traffic.json"
    p.write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "TRAFFIC_RECORD", str(p))
    assert bench.traffic_from_record() == 8.4e9
    rec["kernel_source_sha256_16"] = "0" * 16
    p.write_text(json.dumps(rec))
    assert bench.traffic_from_record() is None


def test_committed_traffic_record_matches_the_committed_kernel():
    with open(bench.TRAFFIC_RECORD) as f:
        rec = json.load(f)
    assert rec["kernel_source_sha256_16"] == bench.fused_source_hash()
    assert rec["captured_samples"] > 0 and rec["dram_bytes_per_full_launch"] > 6.8e9   # >= the algorithmic bytes
