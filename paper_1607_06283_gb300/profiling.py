"""Summaries of ncu output for the committed profiles.

Two inputs, both produced by ncu on the GPU machine and read here without a GPU:

  launch list: ``ncu --metrics gpu__time_duration.sum --clock-control none --csv
  --log-file launches.csv <cmd>`` -> per kernel: launches, total device time, share;

  counters: ``ncu -i <capture>.ncu-rep --page raw --csv > raw.csv`` of a capture of the
  dominant kernel -> per launch the DRAM bytes, duration, issue-active and warps-active
  fractions and registers per thread.

``python -m paper_1607_06283_gb300.profiling launches launches.csv [--exclude a,b]``
prints the launch-list table; ``python -m paper_1607_06283_gb300.profiling counters
raw.csv [--traffic traffic.csv] --workload W --solver S [--scale X] [--update
profiles/counters.json]`` prints the counters of the captured launches and, with
--update, records their mean under (workload, solver, kernel source hash) in the JSON
that bench.py reads for the roofline's ``traffic`` and ``issue_active``.  --traffic
takes the DRAM bytes from a one-pass capture in the program's own sequence (caches as
the program leaves them) instead of the full capture's cold-cache replay.  --scale
multiplies the DRAM bytes (a capture of a smaller case scaled to a full launch by the
units it processes).
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import json
import os
import statistics
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1607_06283_gb300", "csrc")
# the device sources the counters of the iteration kernels depend on (bench.py hashes the
# same lists, through sources_for)
SOLVER_SOURCES = ("evr_kernels.cu", "evr_solvers.cu", "evr_cluster.cu", "evr_tile.cuh",
                  "evr_push.cuh", "evr_internal.cuh")
STAGED_SOURCES = SOLVER_SOURCES + ("evr_staged.cu", "evr_tma.cuh")
REVERSE_SOURCES = ("evr_grad.cu", "evr_tma.cuh")
PERSIST_SOURCES = SOLVER_SOURCES + ("evr_persist.cu", "evr_persist.cuh")


def sources_for(solver: str):
    """The device sources whose hash keys the counters of `solver` (a solver name as the
    library reports it, or k_rev_tiled)."""
    if solver.startswith("staged"):
        return STAGED_SOURCES
    if solver.startswith("k_rev_tiled"):
        return REVERSE_SOURCES
    if solver.startswith("persistent step"):
        return PERSIST_SOURCES
    return SOLVER_SOURCES


def source_hash(files=SOLVER_SOURCES) -> str:
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _rows(path):
    with open(path, newline="") as fh:
        lines = [ln for ln in fh if ln.startswith('"')]  # skip ncu's ==PROF== lines
    return list(csv.reader(lines))


def launch_list(path):
    """{kernel: (launches, total_us)} from a --csv --log-file launch list."""
    rows = _rows(path)
    head = rows[0]
    k_name, k_metric, k_unit, k_val = (head.index("Kernel Name"), head.index("Metric Name"),
                                       head.index("Metric Unit"), head.index("Metric Value"))
    out = {}
    for r in rows[1:]:
        if r[k_metric] != "gpu__time_duration.sum":
            continue
        v = float(r[k_val].replace(",", ""))
        unit = r[k_unit]
        us = (v / 1e3 if unit in ("ns", "nsecond") else v * 1e3 if unit in ("ms", "msecond")
              else v)
        n, t = out.get(r[k_name], (0, 0.0))
        out[r[k_name]] = (n + 1, t + us)
    return out


def launch_table(path, exclude=()) -> str:
    """Markdown table of the launch list; kernels whose name contains one of `exclude`
    are left out of the table and of the shares."""
    kl = {k: v for k, v in launch_list(path).items() if not any(e in k for e in exclude)}
    total = sum(t for _, t in kl.values())
    lines = ["| kernel | launches | total µs | share | avg µs |", "|---|---|---|---|---|"]
    for name, (n, t) in sorted(kl.items(), key=lambda kv: -kv[1][1]):
        short = name if len(name) < 70 else name[:67] + "..."
        lines.append(f"| `{short}` | {n} | {t:.1f} | {100 * t / total:.1f} % | {t / n:.2f} |")
    return "\n".join(lines)


METRICS = {
    "dram_read": "dram__bytes_read.sum",
    "dram_write": "dram__bytes_write.sum",
    "duration": "gpu__time_duration.sum",
    "issue_active": "smsp__issue_active.avg.pct_of_peak_sustained_active",
    "warps_active": "sm__warps_active.avg.pct_of_peak_sustained_active",
    "registers": "launch__registers_per_thread",
}
SCALE = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "nsecond": 1e-3, "ns": 1e-3,
         "usecond": 1.0, "us": 1.0, "msecond": 1e3, "ms": 1e3, "%": 0.01}


def counters(path):
    """Per captured launch: kernel name and the METRICS above (bytes, µs, fractions)."""
    rows = _rows(path)
    head, units = rows[0], rows[1]
    cols = {k: head.index(m) for k, m in METRICS.items() if m in head}
    k_name = head.index("Kernel Name")
    out = []
    for r in rows[2:]:
        d = {"kernel": r[k_name]}
        for k, c in cols.items():
            try:
                v = float(r[c].replace(",", ""))
            except ValueError:
                continue
            d[k] = v * SCALE.get(units[c], 1.0)
        out.append(d)
    return out


def traffic(path):
    """Per launch (ID order): DRAM bytes read + written and duration (µs) from a
    metric-per-row --csv --log-file capture (dram__bytes_read.sum, dram__bytes_write.sum,
    gpu__time_duration.sum), e.g. one pass per launch in the program's own sequence."""
    rows = _rows(path)
    head = rows[0]
    k_id, k_metric, k_unit, k_val = (head.index("ID"), head.index("Metric Name"),
                                     head.index("Metric Unit"), head.index("Metric Value"))
    per = {}
    for r in rows[1:]:
        v = float(r[k_val].replace(",", "")) * SCALE.get(r[k_unit], 1.0)
        d = per.setdefault(int(r[k_id]), {"dram": 0.0, "us": None})
        if r[k_metric] in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            d["dram"] += v
        elif r[k_metric] == "gpu__time_duration.sum":
            d["us"] = v
    return [per[i] for i in sorted(per)]


def summarise_counters(path, scale=1.0):
    cs = counters(path)
    rows = []
    for d in cs:
        dram = (d.get("dram_read", 0.0) + d.get("dram_write", 0.0)) * scale
        rows.append((d["kernel"], dram, d.get("duration"), d.get("issue_active"),
                     d.get("warps_active"), d.get("registers")))
    mean = lambda i: statistics.mean(r[i] for r in rows if r[i] is not None)  # noqa: E731
    summary = {"dram_bytes_per_launch": mean(1), "duration_us": mean(2),
               "issue_active": mean(3), "warps_active": mean(4),
               "registers": mean(5), "launches_captured": len(rows),
               "kernel": rows[0][0] if rows else None}
    return rows, summary


def update_json(path, entry):
    entries = []
    if os.path.exists(path):
        with open(path) as fh:
            entries = json.load(fh)
    entries = [e for e in entries if not (e["workload"] == entry["workload"] and
                                          e["solver"] == entry["solver"])]
    entries.append(entry)
    with open(path, "w") as fh:
        json.dump(entries, fh, indent=1, sort_keys=True)
        fh.write("\n")


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["launches", "counters"])
    ap.add_argument("csv")
    ap.add_argument("--workload")
    ap.add_argument("--solver")
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--update")
    ap.add_argument("--traffic", default=None,
                    help="counters: a metric-per-row capture of DRAM bytes in the program's "
                         "own sequence; its mean per launch is the entry's DRAM bytes")
    ap.add_argument("--command", default="", help="the ncu command, recorded with the entry")
    ap.add_argument("--alg-bytes", type=float, default=None,
                    help="algorithmic bytes of one captured launch, recorded with the entry")
    ap.add_argument("--exclude", default="",
                    help="launches: comma-separated name parts of kernels to leave out")

    a = ap.parse_args(argv)
    if a.what == "launches":
        print(launch_table(a.csv, tuple(e for e in a.exclude.split(",") if e)))
        return 0
    rows, summary = summarise_counters(a.csv, a.scale)
    print("| launch | kernel | DRAM bytes | µs | issue active | warps active | registers |")
    print("|---|---|---|---|---|---|---|")
    for i, r in enumerate(rows):
        print(f"| {i} | `{r[0][:50]}` | {r[1]:.0f} | {r[2]:.2f} | {r[3]:.3f} | {r[4]:.3f} | "
              f"{r[5]:.0f} |")
    if a.traffic:
        tr = traffic(a.traffic)
        print()
        print("| launch (program's own sequence) | DRAM bytes | µs |")
        print("|---|---|---|")
        for i, d in enumerate(tr):
            print(f"| {i} | {d['dram'] * a.scale:.0f} | {d['us']:.2f} |")
        summary["dram_bytes_per_launch"] = statistics.mean(d["dram"] for d in tr) * a.scale
        summary["dram_source"] = "one-pass capture in the program's own sequence"
        print(f"mean DRAM bytes per launch: {summary['dram_bytes_per_launch']:.0f}")
    if a.update:
        entry = dict(summary, workload=a.workload, solver=a.solver,
                     source_sha=source_hash(sources_for(a.solver)),
                     dram_scale=a.scale, command=a.command, alg_bytes_per_launch=a.alg_bytes)
        update_json(a.update, entry)
        print(f"recorded {a.workload} / {a.solver} in {a.update}")
    return 0


if __name__ == "__main__":
    sys.exit(main())
