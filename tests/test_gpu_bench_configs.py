"""Parity on the benchmark's own instances in the benchmark's own launch plans.

Where the oracle can finish (sub-cubes of 2^28 states) the results are compared with it directly,
in the plan the benchmark uses (same kernel, walk length, anchoring).  At the full benchmark step
sizes, which the oracle cannot enumerate, the kernel the benchmark times is checked against other,
independent kernels of the library on the same step (the dense scans against the factored one,
FP32 with FP64 rescoring against the plain FP64 scan), and every returned state's energy is
re-evaluated directly by the oracle.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2607_04857_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

FLOAT_RTOL = 1e-9


@pytest.fixture(scope="module")
def q():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_04857_gb300 import build as qbuild

    qbuild.build()
    import paper_2607_04857_gb300 as q

    q.load_library()
    return q


def same_int(a, b):
    assert a.min == b.min, (a.min, b.min)
    assert a.n_ties == b.n_ties, (a.n_ties, b.n_ties)
    assert np.array_equal(a.ties, b.ties)
    assert np.array_equal(a.topk, b.topk), (a.topk, b.topk)
    assert np.array_equal(a.topk_E, b.topk_E)


def same_float(a, b):
    assert abs(a.min - b.min) <= FLOAT_RTOL * max(1.0, abs(b.min)), (a.min, b.min)
    assert a.n_ties == b.n_ties
    assert np.array_equal(a.ties, b.ties)
    assert np.array_equal(a.topk, b.topk), (a.topk, b.topk)
    assert np.allclose(a.topk_E, b.topk_E, rtol=FLOAT_RTOL, atol=FLOAT_RTOL)


def energies_direct(Q, r):
    """The oracle's direct energy of every returned K-lowest state equals the reported one."""
    for code, e in zip(r.topk.tolist(), r.topk_E.tolist()):
        d = oracle.energy(Q, int(code))
        if isinstance(d, float):
            assert abs(d - e) <= FLOAT_RTOL * max(1.0, abs(d)), (code, d, e)
        else:
            assert d == e, (code, d, e)


@pytest.mark.parametrize("v", [0, 40000, (1 << 16) - 1])
def test_n44_fp32_bench_plan_against_oracle(q, v):
    """n = 44 SK instance, the benchmark's plan (2^14-step walks re-anchored every 2^10 steps,
    9 suffix bits) on 2^28-state sub-cubes."""
    Q = wl.config3()
    r = q.solve(Q, topk=16, fix_bits=16, fix_value=v, walk_bits=14)
    i = r.info
    assert (i["acc"], i["walk_bits"], i["anchor_bits"], i["suffix_bits"]) == ("f32", 14, 10, 9), i
    same_float(r, oracle.solve(Q, topk=16, fix_bits=16, fix_value=v))


def test_n44_fp32_bench_plan_against_fp64_scan(q):
    """A 2^38-state sub-cube in the benchmark's plan against the plain FP64 scan of the library."""
    Q = wl.config3()
    r = q.solve(Q, topk=16, fix_bits=6, fix_value=37)
    assert (r.info["acc"], r.info["walk_bits"], r.info["anchor_bits"]) == ("f32", 14, 10), r.info
    p = q.solve(Q, topk=16, fix_bits=6, fix_value=37, plain=True)
    assert p.info["acc"] == "f64"
    same_float(r, p)
    energies_direct(Q, r)


def test_maxcut_n48_bench_step_three_kernels(q, monkeypatch):
    """One benchmark step of the n = 48 Max-Cut instance (2^42 states): the factored scan the
    benchmark times, the packed 16-bit scan and the FP32-lane scan agree exactly."""
    Q = wl.maxcut_qubo(48, 0.5, seed=48)
    r = q.solve(Q, topk=16, states_cap=1024, fix_bits=6, fix_value=21)
    assert r.info["acc"] == "i32z"
    monkeypatch.setenv("QUBO_NO_I32Z", "1")
    rp = q.solve(Q, topk=16, states_cap=1024, fix_bits=6, fix_value=21)
    assert rp.info["acc"] == "i16p"
    same_int(r, rp)
    monkeypatch.setenv("QUBO_NO_I16P", "1")
    rf = q.solve(Q, topk=16, states_cap=1024, fix_bits=6, fix_value=21)
    assert rf.info["acc"] == "i32f"
    same_int(r, rf)
    energies_direct(Q, r)


def test_sparse_n56_bench_step_factored_vs_dense(q, monkeypatch):
    """One benchmark step of the n = 56 sparse int32 instance (2^46 states): the factored scan
    (one block per unit, 14 factored rows) against the dense scan of the same step."""
    Q = wl.sparse_int(56, 0.05, -1000, 1000, seed=56)
    r = q.solve(Q, topk=16, fix_bits=10, fix_value=513)
    i = r.info
    assert i["acc"] == "i32z" and i["zero_rows"] == 14 and i["walk_bits"] == 14, i
    monkeypatch.setenv("QUBO_NO_I32Z", "1")
    d = q.solve(Q, topk=16, fix_bits=10, fix_value=513)
    assert d.info["acc"] in ("i16p", "i32f", "i32")
    same_int(r, d)
    energies_direct(Q, r)


def test_sparse_f32_n56_bench_step_factored_vs_dense(q, monkeypatch):
    """One benchmark step of the n = 56 sparse FP32 instance (2^46 states): the factored FP32
    scan against the dense FP32 scan, both rescored in FP64."""
    Q = wl.sparse_float32(56, 0.05, seed=56)
    r = q.solve(Q, topk=16, fix_bits=10, fix_value=77)
    assert r.info["acc"] == "f32z", r.info
    monkeypatch.setenv("QUBO_NO_I32Z", "1")
    d = q.solve(Q, topk=16, fix_bits=10, fix_value=77)
    assert d.info["acc"] == "f32"
    same_float(r, d)
    energies_direct(Q, r)


def load_golden(name):
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)
    if not os.path.exists(path):
        pytest.skip(f"{name} not written yet (tests/golden/make_golden.py)")
    with open(path) as fh:
        return json.load(fh)


def test_n50_bench_plan_subcube_golden(q):
    """A 2^40-state sub-cube of the n = 50 instance (the benchmark's plan: FP32 lanes, 14 walked
    bits, 9 suffix bits) against the oracle's stored result (tests/golden/make_golden.py)."""
    g = load_golden("cfg5_n50_sub40.json")
    Q = wl.config5()
    r = q.solve(Q, topk=16, states_cap=4096, fix_bits=g["fix_bits"], fix_value=g["fix_value"])
    i = r.info
    assert (i["acc"], i["walk_bits"], i["suffix_bits"]) == ("i32f", 14, 9), i
    assert r.min == g["min"] and r.n_ties == g["n_ties"]
    assert r.ties.tolist() == g["ties"] and r.topk.tolist() == g["topk"] and r.topk_E.tolist() == g["topk_E"]


def test_n44_fp32_bench_plan_subcube_golden(q):
    """A 2^40-state sub-cube of the n = 44 FP32 instance (the benchmark's plan: 2^14-step walks
    re-anchored every 2^10 steps) against the oracle's stored FP64 result."""
    g = load_golden("cfg3_n44_sub40.json")
    Q = wl.config3()
    r = q.solve(Q, topk=16, states_cap=4096, fix_bits=g["fix_bits"], fix_value=g["fix_value"])
    i = r.info
    assert (i["acc"], i["walk_bits"], i["anchor_bits"]) == ("f32", 14, 10), i
    assert abs(r.min - g["min"]) <= FLOAT_RTOL * max(1.0, abs(g["min"]))
    assert r.n_ties == g["n_ties"] and r.ties.tolist() == g["ties"] and r.topk.tolist() == g["topk"]
    assert np.allclose(r.topk_E, g["topk_E"], rtol=FLOAT_RTOL, atol=FLOAT_RTOL)


def test_n44_fp32_rigorous_subcube_golden(q):
    """The same 2^40-state sub-cube with QUBO_FLAG_RIGOROUS: 2^14-step walks re-anchored every
    2^6 steps, where the rounding bound alone proves the candidate set at the 1e-3 margin."""
    g = load_golden("cfg3_n44_sub40.json")
    Q = wl.config3()
    r = q.solve(Q, topk=16, states_cap=4096, fix_bits=g["fix_bits"], fix_value=g["fix_value"], rigorous=True)
    i = r.info
    assert (i["acc"], i["walk_bits"], i["anchor_bits"]) == ("f32", 14, 6), i
    assert 2 * i["fp32_err_bound"] <= 1e-3 and i["fp32_max_drift"] <= 2 * i["fp32_err_bound"]
    assert abs(r.min - g["min"]) <= FLOAT_RTOL * max(1.0, abs(g["min"]))
    assert r.n_ties == g["n_ties"] and r.ties.tolist() == g["ties"] and r.topk.tolist() == g["topk"]
    assert np.allclose(r.topk_E, g["topk_E"], rtol=FLOAT_RTOL, atol=FLOAT_RTOL)


def test_n44_fp32_bench_step_golden(q):
    """One whole benchmark step of the n = 44 FP32 instance (2^42 states, top 2 bits = 1), in the
    benchmark's plan, against the oracle's stored FP64 result."""
    g = load_golden("cfg3_n44_step42.json")
    Q = wl.config3()
    r = q.solve(Q, topk=16, states_cap=4096, fix_bits=g["fix_bits"], fix_value=g["fix_value"])
    i = r.info
    assert (i["acc"], i["walk_bits"], i["anchor_bits"]) == ("f32", 14, 10), i
    assert i["states_scanned"] == 1 << 42
    assert abs(r.min - g["min"]) <= FLOAT_RTOL * max(1.0, abs(g["min"]))
    assert r.n_ties == g["n_ties"] and r.ties.tolist() == g["ties"] and r.topk.tolist() == g["topk"]
    assert np.allclose(r.topk_E, g["topk_E"], rtol=FLOAT_RTOL, atol=FLOAT_RTOL)


def test_n50_bench_step_golden(q):
    """One whole timed step of the default benchmark (the n = 50 instance, 2^43 states, top 7 bits
    = 5, the first sub-cube after the warm-ups) through the two calls the benchmark times: the
    device-resident problem (value) and qubo_solve_ex from host buffers (e2e), against the
    oracle's stored result."""
    g = load_golden("cfg5_n50_step43.json")
    Q = wl.config5()
    prob = q.Problem(Q, topk=16)
    try:
        prob.run(g["fix_bits"], g["fix_value"])
        rp = prob.fetch(states_cap=4096)
    finally:
        prob.close()
    rs = q.solve(Q, topk=16, states_cap=4096, fix_bits=g["fix_bits"], fix_value=g["fix_value"])
    for r in (rp, rs):
        i = r.info
        assert (i["acc"], i["walk_bits"], i["suffix_bits"]) == ("i32f", 14, 9), i
        assert i["states_scanned"] == 1 << 43
        assert r.min == g["min"] and r.n_ties == g["n_ties"]
        assert r.ties.tolist() == g["ties"] and r.topk.tolist() == g["topk"] and r.topk_E.tolist() == g["topk_E"]
