"""Per-kernel hardware counters (Nsight Compute) of the current kernel sources,
kept as data for ``bench.py``.

    python -m paper_2105_13678_gb300.ncu_counters RAW.csv --names mmh.p3_fwd_col,mh.p3_fwd_col \\
        --command "ncu --metrics ... python bench.py ..."

RAW.csv is ``ncu -i <report> --page raw --csv``; its launches, in order, are
given the trace names of ``--names`` (stage.kernel, as ``pa_trace_collect``
reports them).  The script records, per name, the DRAM bytes read + written,
the duration, the ALU-pipe warp instructions and the issue-active fraction,
together with the SHA-256 of every kernel source file at the time it is run.
``bench.py`` uses a kernel's figures only while the sources still hash the
same, so they are written right after a capture, never edited by hand.
"""
from __future__ import annotations

import argparse
import csv
import datetime
import hashlib
import json
import os

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "kernel_counters.json")

METRICS = {
    "dram__bytes_read.sum": "dram_read_bytes",
    "dram__bytes_write.sum": "dram_write_bytes",
    "gpu__time_duration.sum": "duration_ns",
    "sm__inst_executed_pipe_alu.sum": "alu_warp_inst",
    "sm__inst_executed_pipe_fma.sum": "fma_warp_inst",
    "smsp__inst_executed.sum": "warp_inst",
    "smsp__issue_active.avg.pct_of_peak_sustained_active": "issue_active_pct",
    "sm__pipe_alu_cycles_active.avg.pct_of_peak_sustained_active": "alu_pipe_pct",
    "sm__cycles_elapsed.avg.per_second": "sm_hz",
    "launch__grid_size": "grid",
}


def source_hashes() -> dict:
    """SHA-256 (first 16 hex digits) of every CUDA source and header of the library."""
    out = {}
    for f in sorted(os.listdir(CSRC)):
        if f.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(CSRC, f), "rb") as fh:
                out[f] = hashlib.sha256(fh.read()).hexdigest()[:16]
    return out


def _num(s: str):
    s = s.replace(",", "").strip()
    try:
        return float(s)
    except ValueError:
        return None


def _scale(unit: str) -> float:
    unit = unit.strip().lower()
    return {"byte": 1, "kbyte": 1e3, "mbyte": 1e6, "gbyte": 1e9, "nsecond": 1, "usecond": 1e3, "msecond": 1e6,
            "second": 1e9, "ns": 1, "us": 1e3, "ms": 1e6, "s": 1e9, "hz": 1, "khz": 1e3, "mhz": 1e6,
            "ghz": 1e9}.get(unit, 1.0)


def parse_raw(path: str) -> list[dict]:
    """Launches of an ncu raw-page CSV export, with the metrics above in base units."""
    with open(path, newline="") as f:
        rows = list(csv.reader(f))
    hdr = rows[0]
    units = rows[1] if len(rows) > 1 and not rows[1][0].strip().isdigit() else [""] * len(hdr)
    data = rows[2:] if units is rows[1] else rows[1:]
    col = {name: i for i, name in enumerate(hdr)}
    out = []
    for r in data:
        if len(r) < len(hdr):
            continue
        rec = {"kernel": r[col["Kernel Name"]] if "Kernel Name" in col else ""}
        for m, key in METRICS.items():
            if m in col:
                v = _num(r[col[m]])
                if v is not None:
                    rec[key] = v * _scale(units[col[m]])
        out.append(rec)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("raw", nargs="+", help="ncu --page raw --csv exports")
    ap.add_argument("--names", required=True, help="comma-separated trace names, one per captured launch, in order")
    ap.add_argument("--command", required=True, help="the ncu command line that produced the reports")
    ap.add_argument("--workload", default="plain block n = 2.6e8, r = 0.1 n (config 2)")
    args = ap.parse_args()
    launches = [rec for p in args.raw for rec in parse_raw(p)]
    names = args.names.split(",")
    if len(names) != len(launches):
        raise SystemExit(f"{len(launches)} launches in the reports, {len(names)} names given")
    try:
        with open(OUT) as f:
            doc = json.load(f)
    except (OSError, ValueError):
        doc = {"kernels": {}}
    hashes = source_hashes()
    for name, rec in zip(names, launches):
        rec = dict(rec)
        rec["dram_bytes"] = int(rec.get("dram_read_bytes", 0) + rec.get("dram_write_bytes", 0))
        rec["sources"] = hashes
        rec["command"] = args.command
        rec["workload"] = args.workload
        rec["written"] = datetime.datetime.now(datetime.timezone.utc).strftime("%Y-%m-%dT%H:%M:%SZ")
        doc["kernels"][name] = rec
    with open(OUT, "w") as f:
        json.dump(doc, f, indent=1, sort_keys=True)
    print(f"{OUT}: {', '.join(names)}")


def lookup(name: str):
    """The recorded counters of trace name `name`, or None when absent or when
    any kernel source changed since they were recorded."""
    try:
        with open(OUT) as f:
            rec = json.load(f)["kernels"].get(name)
    except (OSError, ValueError, KeyError):
        return None
    if not rec or rec.get("sources") != source_hashes():
        return None
    return rec


if __name__ == "__main__":
    main()
