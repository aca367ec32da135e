"""Host-side logic of bench.py that needs no GPU: the clock record's
throttle reasons, the gate on recorded DRAM traffic, the workload config."""

import json
import os

import bench


def _clock_summary(tmp_path, lines):
    path = tmp_path / "clocks.csv"
    path.write_text("".join(line + "\n" for line in lines))
    s = bench.ClockSampler(0)
    s.path = str(path)
    return s.summary()


def test_clock_summary_reasons_and_median(tmp_path):
    idle = "0, 2070, 2070, 310.0, 0x0, Not Active, Not Active, Not Active, Not Active"
    capped = "0, 1965, 2070, 1390.5, 0x4, Not Active, Not Active, Not Active, Active"
    hot = "0, 1800, 2070, 1399.0, 0x40, Not Active, Not Active, Active, Not Active"
    out = _clock_summary(tmp_path, [idle, capped, hot, "garbage line"])
    assert out["samples"] == 3
    assert out["sm_mhz"] == 1965.0
    assert out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap", "sw_thermal_slowdown"]
    assert not os.path.exists(str(tmp_path / "clocks.csv"))  # consumed


def test_clock_summary_without_samples(tmp_path):
    out = _clock_summary(tmp_path, [])
    assert out["samples"] == 0 and out["reasons"] == ["unsampled"]


def test_recorded_traffic_is_gated_by_source_hash(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    rec = {"source_hash": "abc", "n1": {"dram_bytes_per_launch": 1.5e8},
           "n4": {"dram_bytes_per_launch": 7.0e7}}
    (prof / "trace_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "trace_source_hash", lambda: "abc")
    assert bench.recorded_traffic(1) == 1.5e8
    assert bench.recorded_traffic(4) == 7.0e7
    assert bench.recorded_traffic(2) is None  # no capture for that launch
    monkeypatch.setattr(bench, "trace_source_hash", lambda: "changed")
    assert bench.recorded_traffic(1) is None  # kernel changed since the capture


def test_source_hash_covers_the_trace_sources():
    h = bench.trace_source_hash()
    assert len(h) == 16 and int(h, 16) >= 0


def test_config_names_the_workload():
    cfg = bench.config_dict(None, 2)
    assert cfg["workload"] == "shell-1M-1080p"
    assert (cfg["gaussians"], cfg["width"], cfg["height"]) == (1_000_000, 1920, 1080)
    assert (cfg["spp"], cfg["n_hits"]) == (bench.SPP_N1, 1) == (64, 1)
    assert cfg["parallelism"].startswith("dp2")
    assert "flushed" in cfg["l2"]
