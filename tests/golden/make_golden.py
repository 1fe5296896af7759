"""Write the stored expected results of the benchmark configurations, using only the CPU oracle.

    python tests/golden/make_golden.py cfg2      # n=36 int32, min + ties + 16 lowest (~2 min, 8 cores)
    python tests/golden/make_golden.py cfg4      # 4096 batched instances (~1 h, 8 cores)
    python tests/golden/make_golden.py cfg5_sub  # n=50, one 2^40-state sub-cube (~1 h, 8 cores)
    python tests/golden/make_golden.py cfg3_sub  # n=44 FP32, one 2^40-state sub-cube (~1 h, 8 cores)
    python tests/golden/make_golden.py cfg3_step # n=44 FP32, one benchmark step of 2^42 states (~4 h)
    python tests/golden/make_golden.py cfg5_step # n=50, one benchmark step of 2^43 states (~9 h, 8 cores)

The inputs come from the seeded generators in paper_2607_04857_gb300/workloads.py; the paper's
benchmark matrices are uniformly random (Sec. 5.3), so the instances are synthetic stand-ins of
the stated shapes.  Every value written here is computed by oracle/ (Gray-walk exhaustive search
with the direct evaluator defining float energies); nothing comes from the CUDA path.
"""
from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2607_04857_gb300 import workloads as wl  # noqa: E402


def cfg2():
    Q = wl.config2()
    t = time.time()
    r = oracle.solve(Q, method=oracle.GRAY, topk=16, cap=1 << 16)
    out = {"config": 2, "generator": "workloads.config2()", "n": 36, "seed": 2, "oracle": "gray",
           "seconds": round(time.time() - t, 1), "min": r.min, "n_ties": r.n_ties,
           "ties": [int(c) for c in r.ties], "topk": [int(c) for c in r.topk],
           "topk_E": [int(e) for e in r.topk_E]}
    with open(os.path.join(HERE, "cfg2_n36_top16.json"), "w") as fh:
        json.dump(out, fh, indent=1)


def cfg4():
    insts = wl.config4()
    rows = []
    t = time.time()
    for i, Q in enumerate(insts):
        r = oracle.solve(Q.astype(np.int32), method=oracle.GRAY, cap=64)
        rows.append({"i": i, "n": int(Q.shape[0]), "min": r.min, "n_ties": r.n_ties,
                     "ties": [int(c) for c in r.ties]})
        if i % 256 == 0:
            print(f"{i} {time.time() - t:.0f}s", file=sys.stderr, flush=True)
    out = {"config": 4, "generator": "workloads.config4()", "count": len(insts), "seed": 4, "oracle": "gray",
           "cap": 64, "seconds": round(time.time() - t, 1), "instances": rows}
    with open(os.path.join(HERE, "cfg4_batched.json"), "w") as fh:
        json.dump(out, fh, separators=(",", ":"))


def subcube(name, Q, n, seed, generator, fix_bits, fix_value, is_float):
    """One sub-cube (top fix_bits code bits = fix_value) of a benchmark instance: min, exact tie
    count, up to 4096 tie codes, the 16 lowest states."""
    t = time.time()
    r = oracle.solve(Q, method=oracle.GRAY, topk=16, cap=4096, fix_bits=fix_bits, fix_value=fix_value)
    conv = float if is_float else int
    out = {"generator": generator, "n": n, "seed": seed, "fix_bits": fix_bits, "fix_value": fix_value,
           "oracle": "gray" + (" (candidates rescored by the direct FP64 evaluator)" if is_float else ""),
           "seconds": round(time.time() - t, 1), "min": conv(r.min), "n_ties": r.n_ties,
           "ties": [int(c) for c in r.ties], "topk": [int(c) for c in r.topk],
           "topk_E": [conv(e) for e in r.topk_E]}
    with open(os.path.join(HERE, name), "w") as fh:
        json.dump(out, fh, indent=1)


def cfg5_sub():
    subcube("cfg5_n50_sub40.json", wl.config5(), 50, 5, "workloads.config5()", 10, 613, False)


def cfg3_sub():
    subcube("cfg3_n44_sub40.json", wl.config3(), 44, 3, "workloads.config3()", 4, 9, True)


def cfg3_step():
    subcube("cfg3_n44_step42.json", wl.config3(), 44, 3, "workloads.config3()", 2, 1, True)


def cfg5_step():
    # the first timed step of the default benchmark: top 7 bits fixed, sub-cube 5 (after 5 warm-ups)
    subcube("cfg5_n50_step43.json", wl.config5(), 50, 5, "workloads.config5()", 7, 5, False)


if __name__ == "__main__":
    for what in sys.argv[1:]:
        {"cfg2": cfg2, "cfg4": cfg4, "cfg5_sub": cfg5_sub, "cfg3_sub": cfg3_sub, "cfg3_step": cfg3_step,
         "cfg5_step": cfg5_step}[what]()
