"""The ncu summaries behind the benchmark's roofline objects (no GPU): parsing of a launch
list and of a raw counter page, the per-launch DRAM traffic of a one-pass capture, the
JSON the benchmark reads, and the benchmark's choice of the memory level."""
import json
import os

import pytest

from paper_1607_06283_gb300 import profiling

LAUNCH_HEAD = ('"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream",'
               '"Block Size","Grid Size","Device","CC","Section Name","Metric Name",'
               '"Metric Unit","Metric Value"')


def _launch_row(i, kernel, metric, unit, value):
    return (f'"{i}","1","python3","host","{kernel}","1","13","(1024, 1, 1)","(150, 1, 1)",'
            f'"0","10.3","Command line profiler metrics","{metric}","{unit}","{value}"')


def test_launch_list_units_shares_and_exclusions(tmp_path):
    p = tmp_path / "launches.csv"
    rows = ["==PROF== Connected to process 1", LAUNCH_HEAD,
            _launch_row(0, "k_tiled<1>", "gpu__time_duration.sum", "ns", "10,000"),
            _launch_row(1, "k_tiled<1>", "gpu__time_duration.sum", "ns", "12000"),
            _launch_row(2, "k_push_one_cta", "gpu__time_duration.sum", "us", "6"),
            _launch_row(3, "FillFunctor", "gpu__time_duration.sum", "ms", "0.04")]
    p.write_text("\n".join(rows) + "\n")
    kl = profiling.launch_list(str(p))
    assert kl["k_tiled<1>"] == (2, pytest.approx(22.0))
    assert kl["k_push_one_cta"] == (1, pytest.approx(6.0))
    assert kl["FillFunctor"] == (1, pytest.approx(40.0))
    table = profiling.launch_table(str(p), exclude=("FillFunctor",))
    assert "FillFunctor" not in table
    assert "78.6 %" in table and "21.4 %" in table  # 22 / 28 and 6 / 28


def test_traffic_of_a_one_pass_capture(tmp_path):
    p = tmp_path / "traffic.csv"
    rows = [LAUNCH_HEAD,
            _launch_row(7, "k", "dram__bytes_read.sum", "Mbyte", "2.5"),
            _launch_row(7, "k", "dram__bytes_write.sum", "Kbyte", "500"),
            _launch_row(7, "k", "gpu__time_duration.sum", "ns", "9000"),
            _launch_row(8, "k", "dram__bytes_read.sum", "byte", "1000"),
            _launch_row(8, "k", "dram__bytes_write.sum", "byte", "0"),
            _launch_row(8, "k", "gpu__time_duration.sum", "us", "8.5")]
    p.write_text("\n".join(rows) + "\n")
    tr = profiling.traffic(str(p))
    assert [d["dram"] for d in tr] == [pytest.approx(3.0e6), pytest.approx(1000.0)]
    assert [d["us"] for d in tr] == [pytest.approx(9.0), pytest.approx(8.5)]


def test_raw_counters_and_the_json_entry(tmp_path):
    names = ["ID", "Kernel Name", "dram__bytes_read.sum", "dram__bytes_write.sum",
             "gpu__time_duration.sum", "smsp__issue_active.avg.pct_of_peak_sustained_active",
             "sm__warps_active.avg.pct_of_peak_sustained_active", "launch__registers_per_thread"]
    units = ["", "", "Mbyte", "byte", "us", "%", "%", "register/thread"]
    data = [["0", "k_tiled<1,2,32>", "3.0", "0", "14.0", "45.5", "49.0", "64"],
            ["1", "k_tiled<1,2,32>", "1.0", "1000", "12.0", "44.5", "50.0", "64"]]
    p = tmp_path / "raw.csv"
    p.write_text("\n".join(",".join(f'"{v}"' for v in r) for r in [names, units] + data) + "\n")
    rows, summary = profiling.summarise_counters(str(p), scale=2.0)
    assert [r[1] for r in rows] == [pytest.approx(6.0e6), pytest.approx(2.002e6)]
    assert summary["issue_active"] == pytest.approx(0.45)
    assert summary["warps_active"] == pytest.approx(0.495)
    assert summary["duration_us"] == pytest.approx(13.0)
    out = tmp_path / "counters.json"
    profiling.update_json(str(out), dict(summary, workload="w", solver="s", source_sha="x"))
    profiling.update_json(str(out), dict(summary, workload="w", solver="s", source_sha="y"))
    entries = json.loads(out.read_text())
    assert len(entries) == 1 and entries[0]["source_sha"] == "y"  # replaced, not appended


def test_sources_keying_each_kernel_family():
    assert "evr_staged.cu" in profiling.sources_for("staged 32x32 R4 (512 threads, 304 CTAs)")
    assert profiling.sources_for("k_rev_tiled")[0] == "evr_grad.cu"
    tiled = profiling.sources_for("tiled 32x64 R9 (1024 threads, 150 CTAs)")
    assert "evr_tile.cuh" in tiled and "evr_grad.cu" not in tiled
    assert len(profiling.source_hash(tiled)) == 16


def test_committed_counters_are_well_formed():
    path = os.path.join(profiling.ROOT, "profiles", "counters.json")
    entries = json.load(open(path))
    for e in entries:
        for k in ("workload", "solver", "source_sha", "dram_bytes_per_launch", "issue_active",
                  "command"):
            assert k in e, (e.get("workload"), k)
        assert 0.0 < e["issue_active"] <= 1.0
        assert e["dram_bytes_per_launch"] >= 0


def test_roofline_level_of_each_solver():
    import sys
    sys.argv = ["bench.py"]
    import bench
    level, peak, _ = bench.roofline_level("cluster 4x4 of 32x32 R0 (512 threads, 16 CTAs)", 152,
                                          12000.0, 38000.0)
    assert level == "smem" and peak == pytest.approx(38000.0 * 16 / 152)
    level, peak, _ = bench.roofline_level("cluster 4x2 of 32x32 R6 (512 threads, 120 CTAs)", 152,
                                          12000.0, 38000.0)
    assert level == "l2" and peak == 12000.0
    level, peak, _ = bench.roofline_level("tiled 32x64 R9 (1024 threads, 150 CTAs)", 152,
                                          12000.0, 38000.0)
    assert level == "l2" and peak == 12000.0
