"""Build and run the arithmetic-throughput probe (csrc/pipe_probe.cu) on the current GPU.

    python -m paper_2607_04857_gb300.pipe_probe [--clock-mhz 2070]

It reports, per SM scheduler with two warps (the occupancy of the scan kernels), the cycles that
16 independent FP32 adds, 2- and 3-input FP32 mins, paired adds, integer adds and mins, and one
Gray step of each scan's mix take.  The scan is bound by these operations, not by memory: the
probe tells which of them share a pipe, hence the roofline the scan kernels are held to.  It is a
measurement tool, not part of the library.
"""
from __future__ import annotations

import argparse
import os
import subprocess
import sys

from . import build as qbuild

SRC = os.path.join(qbuild.CSRC, "pipe_probe.cu")
BIN = os.path.join(qbuild.PKG, "_build", "pipe_probe")


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--clock-mhz", type=float, default=2070.0)
    a = ap.parse_args(argv)
    os.makedirs(os.path.dirname(BIN), exist_ok=True)
    if not os.path.exists(BIN) or os.path.getmtime(BIN) < os.path.getmtime(SRC):
        subprocess.run([qbuild._nvcc(), *qbuild.ARCH, "-O3", "-std=c++20", SRC, "-o", BIN], check=True)
    return subprocess.run([BIN, str(a.clock_mhz)]).returncode


if __name__ == "__main__":
    sys.exit(main())
