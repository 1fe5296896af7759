"""Summarise an ncu capture of one scan-kernel launch into the figures the benchmark's roofline
uses: instructions per state, the issue roofline, DRAM bytes per state, issue activity.

    python -m paper_2607_04857_gb300.ncu_summary CSV --states 2^36 [--sms 152 --clock-mhz 2070]
        [--acc i32f --variant 1 --workload n50_int32 --command "..."
         --update profiles/scan_kernel_counters.json]

CSV is the `--csv --log-file` output of `ncu --metrics ...` for one launch (`-c 1`).  With
--update, the entry of accumulator --acc in the counters file is replaced, tagged with the hash of
the kernel sources the capture was taken on (bench.kernel_source_hash) and the benchmark workload
whose plan it was taken in, so the benchmark only uses counters that still match the code, on that
workload.
"""
from __future__ import annotations

import argparse
import csv
import json
import os
import sys


def read_metrics(path: str) -> dict:
    """Metric name -> float value of the first (only) launch in an ncu CSV log."""
    with open(path) as fh:
        lines = fh.read().splitlines()
    start = next(i for i, line in enumerate(lines) if line.startswith('"ID"'))
    out = {}
    for row in csv.DictReader(lines[start:]):
        name, val = row["Metric Name"], row["Metric Value"].replace(",", "")
        try:
            out.setdefault(name, float(val))
        except ValueError:
            pass
    return out


def summarise(m: dict, states: int, sms: int = 152, clock_mhz: float = 2070.0) -> dict:
    inst = m["sm__inst_executed.sum"] * 32 / states  # thread instructions per state
    dram = m.get("dram__bytes_read.sum", 0.0) + m.get("dram__bytes_write.sum", 0.0)
    dur = m.get("gpu__time_duration.sum", 0.0) * 1e-9  # ncu reports ns
    return {
        "inst_per_state": inst,
        "issue_roofline_states_per_s": sms * 128 * clock_mhz * 1e6 / inst,
        "dram_bytes_per_launch": dram,
        "dram_bytes_per_state": dram / states,
        "issue_active_pct": m.get("smsp__issue_active.avg.pct_of_peak_sustained_active"),
        "states_per_s_under_ncu": states / dur if dur else None,
    }


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("csv")
    ap.add_argument("--states", required=True, help="states scanned by the launch, e.g. 2^36")
    ap.add_argument("--sms", type=int, default=152)
    ap.add_argument("--clock-mhz", type=float, default=2070.0)
    ap.add_argument("--acc")
    ap.add_argument("--variant", type=int, default=0)
    ap.add_argument("--workload", default="")
    ap.add_argument("--command", default="")
    ap.add_argument("--update")
    a = ap.parse_args(argv)
    states = 2 ** int(a.states[2:]) if a.states.startswith("2^") else int(a.states)
    s = summarise(read_metrics(a.csv), states, a.sms, a.clock_mhz)
    print(json.dumps(s, indent=1))
    if a.update:
        if not a.acc:
            raise SystemExit("--update needs --acc")
        root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
        sys.path.insert(0, root)
        import bench

        d = json.load(open(a.update)) if os.path.exists(a.update) else {}
        d[a.acc] = {"kernel_hash": bench.kernel_source_hash(a.acc), "workload": a.workload, "variant": a.variant,
                    "captured_states": states,
                    "inst_per_state": round(s["inst_per_state"], 7),
                    "dram_bytes_per_launch": s["dram_bytes_per_launch"],
                    "dram_bytes_per_state": s["dram_bytes_per_state"],
                    "issue_active_pct": s["issue_active_pct"], "command": a.command}
        with open(a.update, "w") as fh:
            json.dump(d, fh, indent=1)
    return 0


if __name__ == "__main__":
    sys.exit(main())
