"""Host-side logic of bench.py that needs no GPU: the clock record's
throttle reasons, the ncu counter record (parsing and its gate on the kernel
source), the workload config."""

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


def test_recorded_counters_are_gated_by_source_hash(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    rec = {"source_hash": "abc", "launches": {"n1_spp64": {"dram_bytes": 1.5e8,
                                                          "inst_executed": 3.0e10},
                                             "n4_spp16": {"dram_bytes": 7.0e7}}}
    (prof / "trace_counters.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "trace_source_hash", lambda: "abc")
    assert bench.recorded_traffic("n1_spp64") == 1.5e8
    assert bench.recorded_counters("n1_spp64")["inst_executed"] == 3.0e10
    assert bench.recorded_traffic("n4_spp16") == 7.0e7
    assert bench.recorded_traffic("n2_spp8") is None  # no capture for that launch
    monkeypatch.setattr(bench, "trace_source_hash", lambda: "changed")
    assert bench.recorded_traffic("n1_spp64") is None  # kernel changed since the capture


_NCU_CSV = """==PROF== Connected to process 1
"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size","Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"
"0","7","python","h","k_trace","1","7","(128, 1, 1)","(1216, 1, 1)","0","10.3","Command line profiler metrics","dram__bytes_read.sum","byte","67,495,680"
"0","7","python","h","k_trace","1","7","(128, 1, 1)","(1216, 1, 1)","0","10.3","Command line profiler metrics","dram__bytes_write.sum","Mbyte","54.9"
"0","7","python","h","k_trace","1","7","(128, 1, 1)","(1216, 1, 1)","0","10.3","Command line profiler metrics","gpu__time_duration.sum","msecond","52.33"
"0","7","python","h","k_trace","1","7","(128, 1, 1)","(1216, 1, 1)","0","10.3","Command line profiler metrics","lts__t_bytes.sum","Gbyte","1.5"
"0","7","python","h","k_trace","1","7","(128, 1, 1)","(1216, 1, 1)","0","10.3","Command line profiler metrics","smsp__inst_executed.sum","inst","26,000,000,000"
"0","7","python","h","k_trace","1","7","(128, 1, 1)","(1216, 1, 1)","0","10.3","Command line profiler metrics","smsp__issue_active.avg.pct_of_peak_sustained_active","%","77.4"
"0","7","python","h","k_trace","1","7","(128, 1, 1)","(1216, 1, 1)","0","10.3","Command line profiler metrics","smsp__thread_inst_executed_per_inst_executed.ratio","","16.8"
"""


def test_record_counters_parses_ncu_csv(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    log = tmp_path / "c.csv"
    log.write_text(_NCU_CSV)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "trace_source_hash", lambda: "h1")
    e = bench.record_counters(str(log), "n1_spp64", layout={"samples_per_lane": 1})
    assert e["dram_read_bytes"] == 67495680.0
    assert e["dram_write_bytes"] == 54.9e6
    assert e["dram_bytes"] == 67495680.0 + 54.9e6
    assert e["lts_bytes"] == 1.5e9
    assert e["duration_ns_under_ncu"] == 52.33e6
    assert e["inst_executed"] == 2.6e10
    assert e["issue_active_pct"] == 77.4 and e["thread_inst_per_inst"] == 16.8
    assert bench.recorded_counters("n1_spp64")["layout"] == {"samples_per_lane": 1}
    # a record for another source is replaced, not merged
    monkeypatch.setattr(bench, "trace_source_hash", lambda: "h2")
    bench.record_counters(str(log), "n4_spp16")
    assert bench.recorded_counters("n1_spp64") is None
    assert bench.recorded_counters("n4_spp16")["launches"] == 1


def test_source_hash_covers_the_trace_sources():
    h = bench.trace_source_hash()
    assert len(h) == 16 and int(h, 16) >= 0


def test_code_tokens_ignore_comments_only():
    a = "int f(int x) {  // the answer\n    return x + 1; /* one */ }\n"
    b = "int f(int x) {\n  /* a different comment */ return x + 1;\n}"
    c = "int f(int x) { return x + 2; }"
    assert bench.code_tokens(a) == bench.code_tokens(b)
    assert bench.code_tokens(a) != bench.code_tokens(c)


def test_config_names_the_workload():
    cfg = bench.config_dict(None, 2)
    assert cfg["workload"] == "shell-1M-1080p"
    assert (cfg["gaussians"], cfg["width"], cfg["height"]) == (1_000_000, 1920, 1080)
    assert (cfg["spp"], cfg["n_hits"]) == (bench.SPP_N1, 1) == (64, 1)
    assert cfg["parallelism"].startswith("dp2")
    assert "flushed" in cfg["l2"]
