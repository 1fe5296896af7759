#!/usr/bin/env python
"""Benchmark of the exhaustive dense-QUBO scan on GB300.

Default workload: the n=50 dense QUBO with int32 entries uniform in [-32768, 32767] (seed 5),
int32 energies, tie set and the 16 lowest states.  One step is one full pass of the path
(table build, Gray-walk enumeration, reduction and extraction) over one sub-cube of that
instance with its top `--fix-bits` code bits fixed (2^(50-fix_bits) states); consecutive steps
take consecutive sub-cubes, so 2^fix_bits steps cover the whole instance.  The rate is states
per second (2^n / total time, the paper's convention, Sec. 5.3).

  python bench.py [--gpus N] [--steps K] [--warmup W]
                  [--workload n50_int32|n44_fp32|maxcut_n48|sparse_n56|sparse_f32_n56|window_n50|wide_n80|
                              batched]
  python bench.py --impl reference ...   (the CPU oracle on the host cores, same workload)

Under torchrun every rank takes disjoint sub-cubes (no data-path collective; weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2607_04857_gb300 import workloads as wl  # noqa: E402

LANES_PER_SM = 128          # FP32/INT32 lanes per Blackwell SM
ALG_OPS_PER_STATE = 2       # one add and one min per state (Sec. 3.2; Sec. 4.2 on the min)
PAPER_CONTEXT = "7.47e12 states/s, int16 energies, 1x H100 (paper Tab. 1); other machine and dtype"
PROFILE_JSON = os.path.join(ROOT, "profiles", "scan_kernel_counters.json")
# arithmetic type of each accumulator the library reports (integer results are exact in all)
ACC_DTYPE = {"i32": "int32", "i64": "int64", "f32": "f32", "f64": "f64", "i32f": "f32 (integer-valued)",
             "i16p": "u16x2 (integer-valued, packed)", "i32z": "int32 (factored sparse scan)",
             "f32z": "f32 (factored sparse scan)"}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ---------------------------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------------------------

def make_workload(name: str, fix_bits: int | None):
    if name == "n50_int32":
        fb = 7 if fix_bits is None else fix_bits
        return dict(name=name, Q=wl.config5(), n=50, topk=16, fix_bits=fb, metric="states/s (n=50 int32 dense QUBO)",
                    unit="states/s", dtype="int32",
                    config={"workload": "n50_int32_top16", "n": 50, "topk": 16, "seed": 5,
                            "entries": "upper-triangular int32 uniform [-32768, 32767]",
                            "step": f"one sub-cube of 2^{50 - fb} states (top {fb} code bits fixed)"})
    if name == "n44_fp32":
        fb = 2 if fix_bits is None else fix_bits
        return dict(name=name, Q=wl.config3(), n=44, topk=0, fix_bits=fb, metric="states/s (n=44 FP32 SK-like QUBO)",
                    unit="states/s", dtype="f32",
                    config={"workload": "n44_fp32_sk", "n": 44, "seed": 3, "margin": 1e-3,
                            "entries": "symmetric FP32, off-diagonal N(0,1)/sqrt(44), diagonal N(0,1)",
                            "anchor": "re-anchored every 2^10 Gray steps inside 2^14-step walks",
                            "step": f"one sub-cube of 2^{44 - fb} states (top {fb} code bits fixed)"})
    if name == "maxcut_n48":
        fb = 6 if fix_bits is None else fix_bits
        return dict(name=name, Q=wl.maxcut_qubo(48, 0.5, seed=48), n=48, topk=16, fix_bits=fb,
                    metric="states/s (n=48 Max-Cut QUBO)", unit="states/s", dtype="int32",
                    config={"workload": "maxcut_n48_top16", "n": 48, "topk": 16, "seed": 48,
                            "entries": "Max-Cut of G(48, 0.5), edge weights +-1 (int16)",
                            "step": f"one sub-cube of 2^{48 - fb} states (top {fb} code bits fixed)"})
    if name == "sparse_n56":
        fb = 10 if fix_bits is None else fix_bits
        return dict(name=name, Q=wl.sparse_int(56, 0.05, -1000, 1000, seed=56), n=56, topk=16, fix_bits=fb,
                    metric="states/s (n=56 sparse int32 QUBO)", unit="states/s", dtype="int32",
                    config={"workload": "sparse_n56_top16", "n": 56, "topk": 16, "seed": 56,
                            "entries": "upper-triangular int32: diagonal uniform [-1000, 1000], off-diagonal "
                                       "present with probability 0.05, uniform [-1000, 1000]",
                            "step": f"one sub-cube of 2^{56 - fb} states (top {fb} code bits fixed)"})
    if name == "sparse_f32_n56":
        fb = 10 if fix_bits is None else fix_bits
        return dict(name=name, Q=wl.sparse_float32(56, 0.05, seed=56), n=56, topk=16, fix_bits=fb,
                    metric="states/s (n=56 sparse FP32 QUBO)", unit="states/s", dtype="f32",
                    config={"workload": "sparse_f32_n56_top16", "n": 56, "topk": 16, "seed": 56, "margin": 1e-3,
                            "entries": "symmetric FP32: diagonal N(0,1), off-diagonal pairs present with "
                                       "probability 0.05, N(0,1)/sqrt(2.8)",
                            "step": f"one sub-cube of 2^{56 - fb} states (top {fb} code bits fixed)"})
    if name == "window_n50":
        fb = 7 if fix_bits is None else fix_bits
        return dict(name=name, Q=wl.config5(), n=50, topk=0, fix_bits=fb, window=20000,
                    metric="states/s (n=50 int32 dense QUBO, low-energy window)", unit="states/s", dtype="int32",
                    config={"workload": "window_n50_delta20000", "n": 50, "seed": 5, "window": 20000,
                            "entries": "upper-triangular int32 uniform [-32768, 32767]",
                            "outputs": "every state with E <= E_min + 20000 of the sub-cube, (E, code) order",
                            "step": f"one sub-cube of 2^{50 - fb} states (top {fb} code bits fixed)"})
    if name == "wide_n80":
        outer = 64 if fix_bits is None else (1 << fix_bits)
        return dict(name=name, Q=wl.upper_int(80, -1000, 1000, seed=80), n=80, n_inner=40, outer=outer, topk=16,
                    metric="states/s (n=80 int32 dense QUBO, sub-problems of 40 variables)", unit="states/s",
                    dtype="int32",
                    config={"workload": "wide_n80_inner40_top16", "n": 80, "n_inner": 40, "topk": 16, "seed": 80,
                            "entries": "upper-triangular int32 uniform [-1000, 1000]",
                            "step": f"{outer} consecutive outer values (2^40 states each, one batched launch)"})
    if name == "batched":
        return dict(name=name, Qs=wl.config4(), topk=0, metric="instances/s (4096 QUBOs, n uniform in 16..32)",
                    unit="instances/s", dtype="int32",
                    config={"workload": "batched_4096_n16_32", "count": 4096, "seed": 4,
                            "entries": "even: int16 uniform [-127,127]; odd: Max-Cut G(n,0.5) weights +-1",
                            "step": "one persistent launch over all 4096 instances"})
    raise SystemExit(f"unknown workload {name}")


# ---------------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------------------------

ACC_SOURCE = {"i32": ["scan_i32.cu"], "i64": ["scan_i64.cu"], "f32": ["scan_f32.cu"], "f64": ["scan_f64.cu"],
              "i32f": ["scan_i32f.cu"], "i16p": ["scan_i16p.cu"], "i32z": ["scan_sparse.cu", "zscan.h"], "f32z": ["scan_sparse.cu", "zscan.h"]}


def kernel_source_hash(acc: str) -> str:
    """Hash of the sources the accumulator's scan kernel is compiled from."""
    h = hashlib.sha256()
    for f in ["scan_impl.cuh", "internal.h"] + ACC_SOURCE.get(acc, ["scan_i32.cu"]):
        with open(os.path.join(ROOT, "paper_2607_04857_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profile_counters(acc: str, workload: str):
    """ncu counters committed under profiles/ for the scan kernel, if they were taken on the
    current kernel source in this workload's plan; else None."""
    try:
        with open(PROFILE_JSON) as fh:
            d = json.load(fh)
    except (OSError, ValueError):
        return None
    e = d.get(acc)
    if not e or e.get("kernel_hash") != kernel_source_hash(acc) or e.get("workload") != workload:
        return None
    return e


def flush_l2(buf):
    if buf is not None:
        buf.add_(1)


def cpu_oracle_rate(Q, n: int, target_s: float, fix_hint: int):
    """Time the CPU oracle (Gray-walk, all host cores) on sub-cubes of the same instance."""
    import oracle

    fb = max(0, n - 28)
    t = time.perf_counter()
    oracle.solve(Q, method=oracle.GRAY, topk=16, fix_bits=fb, fix_value=1)
    dt = time.perf_counter() - t
    rate = (1 << (n - fb)) / dt
    # grow the sample to about target_s seconds
    free = n - fb
    while free < n and (1 << (free + 1)) / rate < target_s:
        free += 1
    fb2 = n - free
    t = time.perf_counter()
    oracle.solve(Q, method=oracle.GRAY, topk=16, fix_bits=fb2, fix_value=2 if fb2 > 1 else 0)
    dt = time.perf_counter() - t
    return (1 << free) / dt, dt, fb2, oracle.max_threads()


def cpu_oracle_rate_one_core(Q, n: int, target_s: float):
    """The same oracle on one thread (a sub-cube of about target_s seconds)."""
    import oracle

    free = min(n, 22)
    t = time.perf_counter()
    oracle.solve(Q, method=oracle.GRAY, topk=16, fix_bits=n - free, fix_value=1, nthreads=1)
    rate = (1 << free) / (time.perf_counter() - t)
    while free < n and (1 << (free + 1)) / rate < target_s:
        free += 1
    t = time.perf_counter()
    oracle.solve(Q, method=oracle.GRAY, topk=16, fix_bits=n - free, fix_value=0, nthreads=1)
    dt = time.perf_counter() - t
    return (1 << free) / dt, dt, n - free


# ---------------------------------------------------------------------------------------------
# secondary measurements on the same GPU (default workload, one GPU)
# ---------------------------------------------------------------------------------------------

def _timed_problem(q, torch, stream, l2buf, Q, fix_bits, values, **kw):
    """Device-resident problem over the sub-cubes `values` (first one untimed): states/s from CUDA
    events on the launching stream around run + fetch, and the last result's info."""
    prob = q.Problem(Q, **kw)
    prob.run(fix_bits, values[0], stream)
    prob.fetch()
    ev = []
    infos = []
    for v in values[1:]:
        flush_l2(l2buf)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        prob.run(fix_bits, v, stream)
        r = prob.fetch()
        b.record(stream)
        ev.append((a, b))
        infos.append(r.info)
    torch.cuda.synchronize()
    prob.close()
    secs = sum(a.elapsed_time(b) for a, b in ev) / 1000.0
    states = sum(i["states_scanned"] for i in infos)
    scan = sum(i["seconds_scan"] for i in infos)
    return {"value": states / secs, "unit": "states/s", "states_per_step": infos[0]["states_scanned"],
            "steps": len(infos), "scan_kernel_states_per_s": states / scan if scan > 0 else None,
            "acc": infos[-1]["acc"]}, infos[-1]


def _timed_batch(q, torch, stream, l2buf, mats, reps):
    """The 4096-instance batch resident on the device, replayed as its CUDA graph: instances/s
    from CUDA events around replay + fetch, and the per-instance plans used."""
    batch = q.Batch(mats, topk=0, states_cap=64)
    batch.run(stream)
    batch.fetch()
    ev = []
    for _ in range(reps):
        flush_l2(l2buf)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        batch.run(stream)
        rs = batch.fetch()
        b.record(stream)
        ev.append((a, b))
    torch.cuda.synchronize()
    secs = sum(a.elapsed_time(b) for a, b in ev) / 1000.0
    walks = {}
    for i, Q in enumerate(mats):
        walks.setdefault(int(Q.shape[0]), set()).add(int(rs[i].info["walk_bits"]))
    mins = [int(rs[i].min) for i in range(len(mats))]
    batch.close()
    return {"value": reps * len(mats) / secs, "unit": "instances/s", "steps": reps,
            "walk_bits_per_n": {n: sorted(w) for n, w in sorted(walks.items())}}, mins


def secondary(q, torch, stream, l2buf, dev, gpu_index):
    """The same-GPU comparisons: the int32 kernel on the default n=50 step; the n=44 FP32 scan
    with FP64 rescoring against the plain FP64 scan; the 4096-instance batch as one graph replay
    (with the default and the autotuned per-n plans) against a host loop of single solves."""
    out = {}
    sampler = ClockSampler(gpu_index)
    sampler.start()
    # int32 kernel on the benchmark's own n=50 step (2^43 states, top 7 bits fixed)
    r, _ = _timed_problem(q, torch, stream, l2buf, wl.config5(), 7, [4, 5, 6, 7], topk=16, int32=True)
    r["how"] = "QUBO_FLAG_INT32 (int32 lanes), 2^43-state sub-cubes 5..7 of the n=50 instance, top 16"
    out["n50_int32_kernel"] = r
    # n=44 FP32 + FP64 rescore on 2^40-state sub-cubes; plain FP64 on 2^36-state sub-cubes
    Q3 = wl.config3()
    r32, i32 = _timed_problem(q, torch, stream, l2buf, Q3, 4, [0, 1, 2, 3])
    r32["how"] = "FP32 scan + FP64 rescore (margin 1e-3), 2^40-state sub-cubes 1..3 of the n=44 instance"
    r32["fp32_max_abs_err"] = i32["fp32_max_abs_err"]
    r32["fp32_max_drift"] = i32["fp32_max_drift"]
    r32["anchor_bits"] = i32["anchor_bits"]
    rr, ir = _timed_problem(q, torch, stream, l2buf, Q3, 4, [0, 1, 2, 3], rigorous=True)
    rr["how"] = ("FP32 scan + FP64 rescore with QUBO_FLAG_RIGOROUS (re-anchored where the rounding bound "
                 "proves the candidates), 2^40-state sub-cubes 1..3 of the n=44 instance")
    rr["anchor_bits"] = ir["anchor_bits"]
    rr["fp32_err_bound"] = ir["fp32_err_bound"]
    rr["fp32_max_drift"] = ir["fp32_max_drift"]
    out["n44_fp32_rigorous"] = rr
    r32["fp32_err_bound"] = i32["fp32_err_bound"]
    r64, _ = _timed_problem(q, torch, stream, l2buf, Q3, 8, [16, 17, 18], plain=True)
    r64["how"] = "plain FP64 scan (QUBO_FLAG_PLAIN), 2^36-state sub-cubes 17..18 of the n=44 instance"
    out["n44_fp32_rescore"] = r32
    out["n44_fp64_plain"] = r64
    out["fp32_rescore_over_fp64"] = r32["value"] / r64["value"]
    # 4096-instance batch: graph replay, default plans, then autotuned; host loop of single solves
    mats = [q.as_qubo_matrix(Q)[0] for Q in wl.config4()]
    q.autotune_clear()
    rb, mins0 = _timed_batch(q, torch, stream, l2buf, mats, 3)
    rb["how"] = "one CUDA-graph replay per step over all 4096 instances (qubo_batch_run), default plans"
    t = time.perf_counter()
    tuned = q.autotune_batched(mats)
    tune_s = time.perf_counter() - t
    rt, mins1 = _timed_batch(q, torch, stream, l2buf, mats, 3)
    rt["how"] = "as batched_graph, after qubo_autotune_batched on the batch"
    rt["tuner"] = dict(tuned, seconds=tune_s)
    rt["same_minima_as_default"] = mins0 == mins1
    q.autotune_clear()
    torch.cuda.synchronize(dev)
    t = time.perf_counter()
    for Q in mats:
        q.solve(Q, states_cap=64, stream=stream)
    torch.cuda.synchronize(dev)
    loop = len(mats) / (time.perf_counter() - t)
    out["batched_graph"] = rb
    out["batched_graph_tuned"] = rt
    out["batched_loop"] = {"value": loop, "unit": "instances/s",
                           "how": "qubo_solve per instance, looped on the host (host clock)"}
    out["batched_over_loop"] = max(rb["value"], rt["value"]) / loop
    out["clocks"] = sampler.stop()
    return out


def datapath_probe(clock_mhz: float):
    """Cycles one Gray step's operation mix takes on one scheduler in isolation (the arithmetic
    probe, csrc/pipe_probe.cu): the floor the scan kernels are held to.  None if it cannot run."""
    try:
        r = subprocess.run([sys.executable, "-m", "paper_2607_04857_gb300.pipe_probe", "--clock-mhz",
                            f"{clock_mhz:.0f}"], cwd=ROOT, capture_output=True, text=True, timeout=300)
    except (OSError, subprocess.TimeoutExpired):
        return None
    out = {}
    for line in r.stdout.splitlines():
        for key, label in (("fp32_lane_step", "FP32-lane Gray step"), ("int32_step", "int32 Gray step"),
                           ("packed_step", "packed 16-bit Gray step"), ("fadd", "FADD "), ("fadd2", "FADD2 ("),
                           ("fmin3", "FMNMX3 (3 inputs)")):
            if line.startswith(label):
                try:
                    out[key] = float(line.split("ms")[1].split("cycles")[0])
                except (IndexError, ValueError):
                    pass
    return out if r.returncode == 0 and out else None


# ---------------------------------------------------------------------------------------------
# reference arm: the CPU oracle
# ---------------------------------------------------------------------------------------------

def run_reference(args, W):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle

    oracle.build()
    if W["name"] == "batched":
        Qs = W["Qs"]
        order = np.random.default_rng(0).permutation(len(Qs))
        # bounded sample: instances solved one by one until each step takes ~2 s
        i = 0
        times = []
        for s in range(args.warmup + args.steps):
            ts = time.perf_counter()
            cnt = 0
            while time.perf_counter() - ts < 2.0:
                Q = Qs[order[i % len(Qs)]]
                oracle.solve(Q.astype(np.int32), method=oracle.GRAY)
                i += 1
                cnt += 1
            if s >= args.warmup:
                times.append((cnt, time.perf_counter() - ts))
        value = sum(c for c, _ in times) / sum(t for _, t in times)
        sample = "instances of the 4096-instance batch, solved one by one on the host cores"
        ms = 1000 * sum(t for _, t in times) / len(times)
    else:
        Q, n = W["Q"], W["n"]
        if W["name"] == "wide_n80":  # the sub-problem of outer value 0 (40 variables)
            Q, _ = oracle.reduce(W["Q"], W["n_inner"], 0)
            n = W["n_inner"]
        # each step: one sub-cube of about 1 s of oracle work
        fb = max(0, n - 28)
        t = time.perf_counter()
        oracle.solve(Q, method=oracle.GRAY, topk=W["topk"], fix_bits=fb, fix_value=3)
        rate = (1 << (n - fb)) / (time.perf_counter() - t)
        free = n - fb
        while (1 << (free + 1)) / rate < 1.0:
            free += 1
        fb = n - free
        times = []
        for s in range(args.warmup + args.steps):
            t = time.perf_counter()
            oracle.solve(Q, method=oracle.GRAY, topk=W["topk"], fix_bits=fb, fix_value=s % (1 << fb))
            if s >= args.warmup:
                times.append(time.perf_counter() - t)
        value = args.steps * (1 << free) / sum(times)
        sample = f"sub-cubes of 2^{free} states (top {fb} bits fixed) of the same instance per step"
        ms = 1000 * sum(times) / len(times)
    cores = oracle.max_threads()
    line = {"impl": "reference", "metric": W["metric"], "value": value, "unit": W["unit"], "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": W["dtype"], "data": "synthetic",
            "config": W["config"],
            "cpu_baseline": {"value": value, "unit": W["unit"], "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": W["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------------------------

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="n50_int32",
                    choices=["n50_int32", "n44_fp32", "maxcut_n48", "sparse_n56", "sparse_f32_n56", "window_n50",
                             "wide_n80", "batched"])
    ap.add_argument("--fix-bits", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--compare-loop", action="store_true",
                    help="batched workload: also time a host loop of single solves")
    ap.add_argument("--by-size", action="store_true",
                    help="batched workload: also time sub-batches of the instances grouped by size n")
    ap.add_argument("--no-secondary", action="store_true",
                    help="default workload: skip the same-GPU comparisons (int32 kernel, FP32 vs FP64, batched)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    W = make_workload(args.workload, args.fix_bits)
    if args.impl == "reference":
        return run_reference(args, W)

    import torch

    import paper_2607_04857_gb300 as q
    from paper_2607_04857_gb300 import build as qbuild

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if rank == 0:
        qbuild.build()
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group(backend="nccl")
        dist.barrier(device_ids=[local])  # the other ranks wait for rank 0's build
        if rank != 0:
            qbuild.build()
    q.load_library()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    sms = q.device_sm_count()
    l2buf = torch.zeros(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 129 MB L2

    def barrier():
        if dist is not None:
            dist.barrier(device_ids=[local])
        torch.cuda.synchronize(dev)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and W["name"] != "batched":
        # the oracle runs on the host cores before the GPU timing (it uses threads, no fork)
        Qc, nc = W["Q"], W["n"]
        if W["name"] == "wide_n80":
            import oracle

            Qc, _ = oracle.reduce(W["Q"], W["n_inner"], 0)  # the sub-problem of outer value 0
            nc = W["n_inner"]
        rate, dt, fb, cores = cpu_oracle_rate(Qc, nc, 12.0, 0)
        rate1, dt1, fb1 = cpu_oracle_rate_one_core(Qc, nc, 3.0)
        cpu = {"value": rate, "unit": "states/s", "cores": cores, "kind": "oracle",
               "sample": f"Gray-walk oracle on one sub-cube of 2^{nc - fb} states of the same instance "
                         + ("(outer value 0's sub-problem) " if nc != W["n"] else "") + f"({dt:.1f} s)",
               "one_core": {"value": rate1, "unit": "states/s",
                            "sample": f"one thread, one sub-cube of 2^{nc - fb1} states ({dt1:.1f} s)"}}
        log(f"cpu oracle: {rate:.3e} states/s on {cores} threads")

    launches = 0
    scan_s = []
    states_per_step = 0
    sampler = ClockSampler(local)

    if W["name"] == "batched":
        Qs = W["Qs"]
        mats = [q.as_qubo_matrix(Q)[0] for Q in Qs]
        # value: the batch resident on the device, one CUDA-graph replay per step
        batch = q.Batch(mats, topk=0, states_cap=64)
        for s in range(args.warmup):
            batch.run(stream)
            batch.fetch()
        barrier()
        sampler.start()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        infos = []
        for s in range(args.steps):
            flush_l2(l2buf)
            ev[s][0].record(stream)
            batch.run(stream)
            rs = batch.fetch()
            ev[s][1].record(stream)
            infos.append(rs[0].info)
        barrier()
        clocks = sampler.stop()
        batch.close()
        t_dev = sum(a.elapsed_time(b) for a, b in ev) / 1000.0
        units = args.steps * len(Qs)
        launches = sum(i["kernel_launches"] for i in infos)
        scan_s = [i["seconds_scan"] for i in infos]
        states_per_step = sum(1 << Q.shape[0] for Q in Qs)
        # e2e: qubo_solve_batched from host buffers in its packed input layout (the library's
        # host preparation and the copies in every step)
        packed = q.pack_batch(mats)
        q.solve_batched(packed, topk=0, states_cap=64, stream=stream)
        barrier()
        t = time.perf_counter()
        for s in range(args.steps):
            rs = q.solve_batched(packed, topk=0, states_cap=64, stream=stream)
        torch.cuda.synchronize(dev)
        e2e_val = units / (time.perf_counter() - t)
        h2d, d2h = rs[0].info["h2d_bytes"], rs[0].info["d2h_bytes"]
        e2e_note = ("qubo_solve_batched from host buffers in its packed layout (host preparation and copies "
                    "inside every step)")
        loop_rate = None
        by_size = None
        if args.by_size:
            # where the batch's time goes: each size group alone as a device-resident batch
            by_size = []
            for lo, hi in ((16, 20), (21, 24), (25, 28), (29, 30), (31, 32)):
                sub = [Q for Q in mats if lo <= Q.shape[0] <= hi]
                if not sub:
                    continue
                b = q.Batch(sub, topk=0, states_cap=64)
                b.run(stream)
                b.fetch()
                best = None
                for _ in range(3):
                    a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    b.run(stream)
                    b.fetch()
                    c.record(stream)
                    torch.cuda.synchronize(dev)
                    best = min(best or 1e9, a.elapsed_time(c) / 1000.0)
                b.close()
                st = sum(1 << Q.shape[0] for Q in sub)
                by_size.append({"n": [lo, hi], "instances": len(sub), "states": st, "ms": best * 1000,
                                "states_per_s": st / best, "instances_per_s": len(sub) / best})
        if args.compare_loop:
            # the plain form: one qubo_solve per instance, looped on the host
            t = time.perf_counter()
            for Q in mats:
                q.solve(Q, states_cap=64, stream=stream)
            torch.cuda.synchronize(dev)
            loop_rate = len(mats) / (time.perf_counter() - t)
    elif W["name"] in ("window_n50", "wide_n80"):
        # host-buffer entry points (no device-resident form): value = states / the device time the
        # library measures with CUDA events on the launching stream (tables, scan, reduction);
        # e2e = states / wall time of the calls
        loop_rate = None
        Q = W["Q"]
        if W["name"] == "window_n50":
            my = q.shard_subcubes(W["fix_bits"], world, rank)

            def call(s):
                cnt, codes, E, info = q.solve_window(Q, W["window"], cap=1 << 16, fix_bits=W["fix_bits"],
                                                     fix_value=my[s % len(my)], stream=stream)
                info["window_count"] = cnt
                return info
        else:
            n_outer_vals = 1 << (W["n"] - W["n_inner"])

            def call(s):
                begin = ((s * world + rank) * W["outer"]) % n_outer_vals
                r = q.solve_wide(Q, W["n_inner"], outer_begin=begin, outer_count=W["outer"], topk=W["topk"],
                                 stream=stream)
                return r.info
        for s in range(args.warmup):
            call(s)
        barrier()
        sampler.start()
        infos = []
        for s in range(args.steps):
            flush_l2(l2buf)
            infos.append(call(args.warmup + s))
        barrier()
        clocks = sampler.stop()
        t_dev = sum(i["seconds_gpu"] for i in infos)
        states_per_step = infos[0]["states_scanned"]
        units = sum(i["states_scanned"] for i in infos)
        launches = sum(i["kernel_launches"] for i in infos)
        scan_s = [i["seconds_scan"] for i in infos]
        # e2e: the same calls timed by the host clock (after the clock sampler has stopped, as for
        # the other workloads)
        t = time.perf_counter()
        walls = []
        for s in range(args.steps):
            tc = time.perf_counter()
            call(args.warmup + s)
            walls.append(time.perf_counter() - tc)
        torch.cuda.synchronize(dev)
        t_wall = time.perf_counter() - t
        log("e2e call walls (s): " + " ".join(f"{w:.4f}" for w in walls))
        e2e_val = units / t_wall
        h2d, d2h = infos[-1]["h2d_bytes"], infos[-1]["d2h_bytes"]
        e2e_note = ("qubo_solve_window" if W["name"] == "window_n50" else "qubo_solve_wide") + \
            " from host buffers (host preparation and copies inside every step)"
        if W["name"] == "window_n50":
            W["config"]["window_states_per_step"] = [i["window_count"] for i in infos]
    else:
        loop_rate = None
        Q, n, topk, fb = W["Q"], W["n"], W["topk"], W["fix_bits"]
        my = q.shard_subcubes(fb, world, rank)

        def sub(s):
            return my[s % len(my)]

        # value: device-resident problem, inputs uploaded before the timed region
        prob = q.Problem(Q, topk=topk)
        for s in range(args.warmup):
            prob.run(fb, sub(s), stream)
            prob.fetch()
        barrier()
        sampler.start()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        infos = []
        for s in range(args.steps):
            flush_l2(l2buf)
            ev[s][0].record(stream)
            prob.run(fb, sub(args.warmup + s), stream)
            r = prob.fetch()
            ev[s][1].record(stream)
            infos.append(r.info)
        barrier()
        clocks = sampler.stop()
        prob.close()
        t_dev = sum(a.elapsed_time(b) for a, b in ev) / 1000.0
        states_per_step = 1 << (n - fb)
        units = args.steps * states_per_step
        launches = sum(i["kernel_launches"] for i in infos)
        scan_s = [i["seconds_scan"] for i in infos]
        # e2e: the public call with host buffers, copies inside every step
        q.solve(Q, topk=topk, fix_bits=fb, fix_value=sub(0), stream=stream)
        barrier()
        t = time.perf_counter()
        for s in range(args.steps):
            r = q.solve(Q, topk=topk, fix_bits=fb, fix_value=sub(args.warmup + s), stream=stream)
        torch.cuda.synchronize(dev)
        t_e2e = time.perf_counter() - t
        e2e_val = units / t_e2e
        h2d, d2h = r.info["h2d_bytes"], r.info["d2h_bytes"]
        e2e_note = "qubo_solve_ex from host buffers (Q upload and result download inside every step)"

    # max over ranks
    t_max = t_dev
    if dist is not None:
        tt = torch.tensor([t_dev], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_max = float(tt.item())
        ee = torch.tensor([e2e_val], dtype=torch.float64, device=dev)
        dist.all_reduce(ee, op=dist.ReduceOp.SUM)
        e2e_val = float(ee.item())
    value = units * world / t_max
    if W["name"] in ("window_n50", "wide_n80"):
        W["config"]["value_timing"] = "device time of each call's kernels (CUDA events on the launching stream)"

    # roofline of the enumeration kernel: algorithmic ALU ops per launch / its event-timed duration
    mean_scan = sum(scan_s) / len(scan_s)
    per_launch_states = states_per_step  # one enumeration launch per step
    acc = infos[0].get("acc", "i32")
    W["dtype"] = ACC_DTYPE.get(acc, acc)
    # the packed scan holds two 16-bit columns in each 32-bit lane: twice the lane-ops per cycle
    halves = 2 if acc == "i16p" else 1
    ops_per_state = ALG_OPS_PER_STATE
    grouped = bool(infos[0].get("grouped"))
    if grouped:
        # grouped form: one add per state, and one min per column per group of 16 Gray steps (the
        # exact minimum at the group's first state); the min tree of a group runs only when its
        # lower bound reaches the threshold
        ops_per_state = 1.0 + 1.0 / 16
    if acc in ("i32z", "f32z"):
        # factored scan: one add and one min per column per block of 2^Z walk steps, and one
        # add and one min per walk step per 2^B columns (the block minima of E_L)
        Zr, Bs = infos[0]["zero_rows"], infos[0]["suffix_bits"]
        ops_per_state = 2.0 / 2 ** Zr + 2.0 / 2 ** Bs
    achieved = ops_per_state * per_launch_states / mean_scan / 1e9
    clk_max = (clocks or {}).get("sm_max_mhz") or 2070.0
    peak = halves * sms * LANES_PER_SM * clk_max * 1e6 / 1e9
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gop/s", "frac": achieved / peak,
            "traffic": None, "kernel": "scan_kernel",
            "peak_basis": f"{sms} SMs x {LANES_PER_SM} lanes" + (" x 2 packed 16-bit halves" if halves == 2 else "")
                          + f" x {clk_max:.0f} MHz; {ops_per_state:.4g} ops/state"
                          + (" (grouped form: one add per state and one min per column per group of 16 Gray steps;"
                             " a group's min tree runs only when its lower bound reaches the threshold; one operation"
                             " per lane and cycle: paper_2607_04857_gb300.pipe_probe)" if grouped else
                             " (one add and one min-reduction per state; adds and mins share the 32-lane datapath,"
                             " one operation per lane and cycle: paper_2607_04857_gb300.pipe_probe)"
                             if acc not in ("i32z", "f32z") else
                             f" (factored scan: 2/2^Z + 2/2^B, Z = {infos[0]['zero_rows']}, B = {infos[0]['suffix_bits']})")}
    if clocks and clocks.get("sm_mhz"):
        roof["frac_at_sampled_clock"] = achieved / (halves * sms * LANES_PER_SM * clocks["sm_mhz"] * 1e-3)
    prof = profile_counters(acc, W["name"])
    if prof:
        # DRAM bytes per launch, scaled from the captured launch by the states it processed
        roof["traffic"] = prof["dram_bytes_per_state"] * per_launch_states
        roof["traffic_basis"] = (f"ncu capture of {prof['captured_states']} states scaled to "
                                 f"{per_launch_states} states per launch")
        if prof.get("inst_per_state") and clocks:
            ips = prof["inst_per_state"]
            issue = sms * LANES_PER_SM * clocks["sm_mhz"] * 1e6 / ips
            roof["issue_roofline"] = {"inst_per_state": ips, "states_per_s": issue,
                                      "frac": (per_launch_states / mean_scan) / issue}
            if grouped and acc == "i32f":
                roof["issue_roofline"]["note"] = (
                    "the column adds issue as paired f32x2 instructions (two columns per instruction, two "
                    "datapath cycles), so instruction issue is not this kernel's bound: the FP32 add datapath is "
                    "(roofline.frac); the same form with scalar adds (QUBO_SCAN_VARIANT=22) issues twice the adds "
                    "and runs slower")

    sec = None
    if W["name"] == "n50_int32" and world == 1 and not args.no_secondary:
        sec = secondary(q, torch, stream, l2buf, dev, local)
        # the dense scan's step floor on this GPU: cycles per 16-column step (512 states per warp)
        # of the kernel against the same operation mix timed alone
        clk = (clocks or {}).get("sm_mhz") or 2070.0
        probe = datapath_probe(clk)
        key = "fadd2" if grouped else "fp32_lane_step"
        if probe and acc == "i32f" and probe.get(key):
            kernel_cycles = sms * 4 * clk * 1e6 / ((per_launch_states / mean_scan) / 512.0)
            roof["datapath"] = {"kernel_cycles_per_step": kernel_cycles,
                                "probe_cycles_per_step": probe[key],
                                "probe_cycles_per_16_fadd": probe.get("fadd"),
                                "probe_cycles_per_16_fmnmx3": probe.get("fmin3"),
                                "basis": "one Gray step = 16 columns x 32 lanes = 512 states per warp; probe: "
                                         + ("the step's 16 column adds as 8 paired f32x2 adds alone (the grouped "
                                            "form's floor)" if grouped else "the step's adds and mins alone")
                                         + " with a loop counter (python -m paper_2607_04857_gb300.pipe_probe)"}

    if rank == 0:
        line = {"metric": W["metric"], "value": value, "unit": W["unit"], "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1000 * t_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": W["dtype"], "data": "synthetic",
                "config": dict(W["config"], parallelism=f"{world} GPU(s), disjoint sub-cubes per rank" if world > 1
                               else "1 GPU", l2="256 MiB buffer written between timed steps (L2 is 129 MB)",
                               states_per_step=states_per_step),
                "e2e": {"value": e2e_val, "unit": W["unit"], "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                        "how": e2e_note},
                "gpu_launches": launches, "roofline": roof, "clocks": clocks,
                "scan_kernel_ms_mean": mean_scan * 1000, "context": PAPER_CONTEXT}
        if cpu:
            line["cpu_baseline"] = cpu
        if sec:
            line["secondary"] = sec
        if W["name"] == "batched" and by_size:
            line["by_size"] = by_size
        if loop_rate:
            line["loop_baseline"] = {"value": loop_rate, "unit": "instances/s",
                                     "how": "qubo_solve per instance, looped on the host"}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
