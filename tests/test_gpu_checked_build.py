"""The checked build of the library (libqubo_debug.so, compiled with QUBO_DEBUG): every device
check is compiled in (work items inside their instance, walked rows inside the walk, the walk
inside its E_L table); a failed check records its site in the instance's state and the call
returns QUBO_ERR_INTERNAL instead of touching memory out of range; nothing traps.  Here every
kernel family runs through it on small instances, in a separate process that loads only the
checked library, and must return the oracle's results with no check failed."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import numpy as np
import oracle
import paper_2607_04857_gb300 as q
from paper_2607_04857_gb300 import build as qb, workloads as wl

q.load_library(qb.DEBUG_LIB)
assert any("libqubo_debug.so" in line for line in open("/proc/self/maps"))

def same(r, o):
    assert r.min == o.min and r.n_ties == o.n_ties, (r.min, o.min, r.n_ties, o.n_ties)
    assert np.array_equal(r.ties, o.ties) and np.array_equal(r.topk, o.topk)

kernels = set()
for Q, kw in ((wl.upper_int(26, -30000, 30000, seed=1), {}),          # integers in FP32 lanes
              (wl.upper_int(25, -60, 60, seed=2), {}),                # packed 16-bit lanes
              (wl.upper_int(26, -30000, 30000, seed=3), {"int32": True}),
              (wl.upper_int(27, -500, 500, seed=4), {"walk_bits": 5}),  # fewer register rows
              (wl.upper_int(24, -500, 500, seed=5), {"plain": True}),   # int64
              (wl.sparse_int(28, 0.08, -500, 500, seed=6), {})):        # factored scan
    r = q.solve(Q, topk=8, **kw)
    same(r, oracle.solve(Q, topk=8))
    kernels.add(r.info["acc"])
F = wl.sk_float32(23, seed=7)
for kw in ({}, {"rigorous": True}, {"plain": True}):
    r = q.solve(F, topk=4, **kw)
    o = oracle.solve(F, topk=4)
    assert np.array_equal(r.ties, o.ties) and np.array_equal(r.topk, o.topk)
    kernels.add(r.info["acc"])
Qs = wl.config4(count=24, seed=8)
for Qb, rb in zip(Qs, q.solve_batched(Qs, topk=2)):
    same(rb, oracle.solve(Qb.astype(np.int32), topk=2, cap=64))
Qn = wl.upper_int(30, -400, 400, seed=9)
rn = q.solve_noalloc(Qn, states_cap=64)
on = oracle.solve(Qn, cap=64)
assert rn.min == on.min and rn.n_ties == on.n_ties
print("checked build clean:", sorted(kernels))
"""


def test_checked_build_runs_every_kernel_clean():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_04857_gb300 import build as qbuild

    qbuild.build(debug=True)
    env = dict(os.environ, PYTHONPATH=os.pathsep.join([ROOT, os.path.join(ROOT, "tests")]))
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "checked build clean" in r.stdout
    for acc in ("i32f", "i16p", "i32", "i64", "i32z", "f32", "f64"):
        assert acc in r.stdout, r.stdout
