"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer Q: minimum, exact tie count, tie codes and K lowest states must be bit-exact.
Float Q: the tie set and the K lowest codes must be identical and the minimum within 1e-9
relative of the oracle's FP64 value (both sides evaluate the final energies with the same
fixed-order FP64 sum, so in practice they are equal).
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
from paper_2607_04857_gb300 import workloads as wl
from plan_checks import fp32_lanes_fit

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


def check_int(r, o, cap=None):
    assert r.min == o.min, (r.min, o.min)
    assert r.n_ties == o.n_ties, (r.n_ties, o.n_ties)
    assert np.array_equal(r.ties, o.ties), (r.ties[:8], o.ties[:8])
    assert np.array_equal(r.topk, o.topk), (r.topk, o.topk)
    assert np.array_equal(r.topk_E, o.topk_E), (r.topk_E, o.topk_E)


def check_float(r, o):
    assert abs(r.min - o.min) <= FLOAT_RTOL * max(1.0, abs(o.min)), (r.min, o.min)
    assert r.n_ties == o.n_ties
    assert np.array_equal(r.ties, o.ties)
    assert np.array_equal(r.topk, o.topk), (r.topk, o.topk)
    assert np.allclose(r.topk_E, o.topk_E, rtol=FLOAT_RTOL, atol=FLOAT_RTOL)


# --- integers -----------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 5, 9, 13])
def test_direct_path_small_n(q, n):
    for seed in range(3):
        Q = wl.upper_int(n, -9, 9, seed=seed)
        K = min(1 << n, 16)
        check_int(q.solve(Q, topk=K), oracle.solve(Q, method=oracle.DIRECT, topk=K))


# Integer kernels: packed 16-bit lanes (chosen first for these small entries), FP32 lanes, int32.
LANES = {"i16p": {"QUBO_NO_I32Z": "1"}, "i32f": {"QUBO_NO_I32Z": "1", "QUBO_NO_I16P": "1"},
         "i32": {"QUBO_NO_I32Z": "1", "QUBO_NO_I16P": "1", "QUBO_NO_I32F": "1"}}


@pytest.mark.parametrize("n", [14, 15, 16, 19, 22, 26])
@pytest.mark.parametrize("topk", [0, 1, 16])
@pytest.mark.parametrize("lanes", list(LANES))
def test_int_parity(q, n, topk, lanes, monkeypatch):
    for k, v in LANES[lanes].items():
        monkeypatch.setenv(k, v)
    for seed in range(2):
        Q = wl.upper_int(n, -30, 30, seed=1000 * n + seed)
        r = q.solve(Q, topk=topk)
        assert r.info["acc"] == lanes
        check_int(r, oracle.solve(Q, topk=topk))


def test_full_nonsymmetric_int_q(q):
    rng = np.random.default_rng(3)
    Q = rng.integers(-50, 50, size=(21, 21)).astype(np.int32)
    check_int(q.solve(Q, topk=8), oracle.solve(Q, topk=8))


def test_config1_n24(q):
    Q = wl.config1()
    r = q.solve(Q)
    check_int(r, oracle.solve(Q, method=oracle.DIRECT))
    assert r.info["states_scanned"] == 1 << 24 and r.info["acc"] in ("i32", "i32f", "i16p")


@pytest.mark.parametrize("walk_bits", [4, 5, 8, 11, 13])
def test_plan_shapes_agree(q, walk_bits):
    Q = wl.upper_int(27, -200, 200, seed=77)
    o = oracle.solve(Q, topk=16)
    r = q.solve(Q, topk=16, walk_bits=walk_bits)
    check_int(r, o)
    assert r.info["walk_bits"] == walk_bits


def test_int64_accumulator_for_wide_range(q):
    Q = wl.upper_int(20, -2**31, 2**31 - 1, seed=5)
    r = q.solve(Q, topk=4)
    assert r.info["acc"] == "i64"
    check_int(r, oracle.solve(Q, topk=4))


def test_plain_int64_scan_matches(q):
    Q = wl.upper_int(23, -1000, 1000, seed=6)
    r = q.solve(Q, topk=16, plain=True)
    assert r.info["acc"] == "i64"
    check_int(r, oracle.solve(Q, topk=16))


def test_int16_input(q):
    Q = wl.upper_int(20, -127, 127, seed=8, dtype=np.int16)
    check_int(q.solve(Q, topk=3), oracle.solve(Q.astype(np.int32), topk=3))


# --- special instances --------------------------------------------------------------------

def test_zero_matrix_truncation(q):
    n = 18
    Q = np.zeros((n, n), dtype=np.int32)
    r = q.solve(Q, topk=5, states_cap=1000)
    assert r.min == 0 and r.n_ties == 1 << n and r.truncated and r.status == q.QUBO_TRUNCATED
    assert np.array_equal(r.ties, np.arange(1000, dtype=np.uint64))
    assert np.array_equal(r.topk, np.arange(5, dtype=np.uint64))


def test_diagonal_tie_set(q):
    Q = wl.diagonal(24, seed=3, zeros=7)
    check_int(q.solve(Q, states_cap=1 << 10), oracle.solve(Q, cap=1 << 10))


def test_planted(q):
    Q, xs = wl.planted(30, seed=4)
    r = q.solve(Q)
    assert r.n_ties == 1 and int(r.ties[0]) == xs


def test_maxcut_complement_pairs(q):
    Q = wl.maxcut_qubo(24, 0.5, seed=9)
    r = q.solve(Q, topk=6)
    check_int(r, oracle.solve(Q, topk=6))
    full = (1 << 24) - 1
    ties = set(int(t) for t in r.ties)
    assert all((full ^ t) in ties for t in ties)


def test_relabelled_instance_same_minimum(q):
    Q = wl.upper_int(25, -100, 100, seed=10)
    perm = np.random.default_rng(2).permutation(25)
    a, b = q.solve(Q), q.solve(Q[np.ix_(perm, perm)])
    assert a.min == b.min and a.n_ties == b.n_ties


# --- sub-cubes, merge, device-resident problems ------------------------------------------

def test_subcubes_merge_to_whole(q):
    Q = wl.upper_int(28, -64, 64, seed=12)
    whole = q.solve(Q, topk=16)
    acc = None
    for v in range(8):
        part = q.solve(Q, topk=16, fix_bits=3, fix_value=v)
        assert part.info["states_scanned"] == 1 << 25
        acc = part if acc is None else q.merge(acc, part, 1 << 16, 16)
    check_int(acc, whole)
    check_int(whole, oracle.solve(Q, topk=16))


def test_problem_run_fetch(q):
    Q = wl.upper_int(26, -500, 500, seed=13)
    p = q.Problem(Q, topk=16)
    parts = []
    for v in range(4):
        p.run(2, v)
        parts.append(p.fetch())
    p.close()
    acc = parts[0]
    for r in parts[1:]:
        acc = q.merge(acc, r, 1 << 16, 16)
    check_int(acc, oracle.solve(Q, topk=16))


def test_overflow_splits_and_stays_exact(q):
    """A tiny candidate buffer forces the split-and-merge path; results stay exact."""
    code = (
        "import numpy as np, oracle, paper_2607_04857_gb300 as q;"
        "from paper_2607_04857_gb300 import workloads as wl;"
        "Q = wl.diagonal(20, seed=3, zeros=12);"
        "r = q.solve(Q, topk=4, states_cap=500); o = oracle.solve(Q, topk=4, cap=500);"
        "assert r.min == o.min and r.n_ties == o.n_ties == 4096, (r.n_ties, o.n_ties);"
        "assert np.array_equal(r.ties, o.ties) and np.array_equal(r.topk, o.topk);"
        "assert r.info['passes'] > 1, r.info; print('passes', r.info['passes'])"
    )
    env = dict(os.environ, QUBO_MAX_RECORDS="1000")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    res = subprocess.run([sys.executable, "-c", code], env=env, cwd=root, capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stdout + res.stderr


# --- floats ---------------------------------------------------------------------------------

@pytest.mark.parametrize("n", [6, 14, 18, 22, 25])
def test_float_parity(q, n):
    for seed in range(2):
        Q = wl.sk_float32(n, seed=500 + n + seed)
        r = q.solve(Q, topk=8)
        check_float(r, oracle.solve(Q, topk=8))
        assert r.info["acc"] == "f32" or n < 14


@pytest.mark.parametrize("n", [18, 21, 24])
@pytest.mark.parametrize("topk", [1, 16])
def test_float_ulp_near_ties(q, n, topk):
    """3^(n//2) exact-arithmetic minimisers split by FP64 rounding (FP64 input, weights 0.1, 0.2,
    0.3, 0.7): the FP32 scan must pass all of them to the FP64 rescoring, whose fixed-order sums
    (the oracle's) decide the tie set and the K lowest bit for bit; at n = 24 the 2^14-step
    walks are re-anchored inside."""
    Q = wl.decimal_pairs(n, seed=n)
    r = q.solve(Q, topk=topk, states_cap=1 << 16)
    o = oracle.solve(Q, topk=topk, cap=1 << 16)
    assert r.info["acc"] == "f32"
    assert 1 < o.n_ties < 3 ** (n // 2)
    assert r.min == o.min
    check_float(r, o)
    assert np.array_equal(r.topk_E, o.topk_E)


def test_float64_input_and_plain_fp64(q):
    Q = wl.sk_float32(21, seed=44).astype(np.float64)
    o = oracle.solve(Q, topk=8)
    check_float(q.solve(Q, topk=8), o)
    rp = q.solve(Q, topk=8, plain=True)
    assert rp.info["acc"] == "f64"
    check_float(rp, o)


def test_float_drift_within_margin(q):
    Q = wl.config3()[:30, :30].copy()
    r = q.solve(Q, topk=4)
    assert r.info["acc"] == "f32"
    assert 2 * r.info["fp32_max_drift"] < 1e-3
    assert r.info["fp32_max_abs_err"] < 1e-3
    check_float(r, oracle.solve(Q, topk=4))


def test_fp32_reanchoring_inside_long_walks(q):
    """Walks of 2^14 Gray steps re-anchored every 2^10.  On an instance whose FP32 sums are all
    exact (multiples of 2^-10 below 2^6) the rebuilt columns must equal the incrementally updated
    ones, so the measured drift is exactly 0 (a wrong row set or a missing coupling in the rebuild
    shows up here) and the results equal the oracle's; on an SK instance the drift is positive and
    within the margin."""
    Qd = (wl.upper_int(34, -60, 60, seed=7) / 1024.0).astype(np.float32)
    r = q.solve(Qd, topk=8, fix_bits=4, fix_value=5, walk_bits=14)
    i = r.info
    assert (i["acc"], i["walk_bits"], i["anchor_bits"]) == ("f32", 14, 10), i
    assert i["fp32_max_drift"] == 0.0
    check_float(r, oracle.solve(Qd, topk=8, fix_bits=4, fix_value=5))
    Q = wl.sk_float32(34, seed=34)
    r = q.solve(Q, topk=8, fix_bits=4, fix_value=9, walk_bits=14)
    i = r.info
    assert (i["acc"], i["walk_bits"], i["anchor_bits"]) == ("f32", 14, 10), i
    assert 0.0 < 2 * i["fp32_max_drift"] < 1e-3
    check_float(r, oracle.solve(Q, topk=8, fix_bits=4, fix_value=9))


def test_fp32_drift_guard_shortens_the_anchor_period(q):
    """A candidate margin just below what the measured drift needs at 2^10-step anchoring makes the
    host rescan with a shorter period (or, at the shortest, in FP64); the results stay exact."""
    Q = wl.sk_float32(34, seed=35)
    r0 = q.solve(Q, topk=4, fix_bits=4, walk_bits=14)
    d10 = r0.info["fp32_max_drift"]
    U = np.triu(Q.astype(np.float64)) + np.triu(Q.astype(np.float64).T, 1)
    slack = 8.0 * 2.0 ** -24 * (1.0 + np.abs(U).sum())
    margin = 0.999 * (2 * d10 + slack)
    r = q.solve(Q, topk=4, fix_bits=4, walk_bits=14, margin=margin)
    i = r.info
    assert i["acc"] == "f64" or (i["acc"] == "f32" and i["anchor_bits"] < 10), i
    assert i["passes"] >= 2
    check_float(r, oracle.solve(Q, topk=4, fix_bits=4))


def test_fp32_rigorous_mode(q):
    """QUBO_FLAG_RIGOROUS: the FP32 scan re-anchors at the period its rounding bound proves
    (n = 34 SK sub-cubes, 2^14-step walks), results equal the oracle's; the measured drift and
    the scan's energy errors stay within the reported bound; with a margin no period can meet
    the scan runs in FP64, still exact."""
    Q = wl.sk_float32(34, seed=36)
    o = oracle.solve(Q, topk=8, fix_bits=4, fix_value=6)
    r = q.solve(Q, topk=8, fix_bits=4, fix_value=6, walk_bits=14, rigorous=True)
    i = r.info
    assert i["acc"] == "f32" and i["walk_bits"] == 14
    assert i["anchor_bits"] == min(10, i["fp32_rigorous_anchor_bits"]) and i["anchor_bits"] >= 5
    assert 2 * i["fp32_err_bound"] <= 1e-3
    assert i["fp32_max_drift"] <= 2 * i["fp32_err_bound"]
    assert i["fp32_max_abs_err"] <= 2 * i["fp32_err_bound"]
    check_float(r, o)
    d = q.solve(Q, topk=8, fix_bits=4, fix_value=6, walk_bits=14)  # default: measured drift
    assert d.info["anchor_bits"] == 10 and d.info["fp32_max_drift"] <= 2 * d.info["fp32_err_bound"]
    check_float(d, o)
    f = q.solve(Q, topk=8, fix_bits=4, fix_value=6, margin=1e-6, rigorous=True)
    assert f.info["acc"] == "f64"
    check_float(f, o)


# --- batched ----------------------------------------------------------------------------------

def test_batched_matches_per_instance(q):
    insts = wl.config4(count=96, seed=4)
    insts = [Q for Q in insts if Q.shape[0] <= 24][:40]
    insts += [wl.upper_int(n, -127, 127, seed=n, dtype=np.int16) for n in (3, 8, 12, 13)]
    rs = q.solve_batched(insts, topk=4, states_cap=64)
    for Q, r in zip(insts, rs):
        o = oracle.solve(Q.astype(np.int32), topk=4, cap=64)
        check_int(r, o)
        assert r.info["states_scanned"] == 1 << Q.shape[0]


def test_batched_prepacked_input_equals_list(q):
    """A batch packed once (pack_batch) gives the same results as the list of matrices."""
    insts = wl.config4(count=40, seed=7)
    insts = [Q for Q in insts if Q.shape[0] <= 22]
    a = q.solve_batched(insts, topk=2, states_cap=16)
    b = q.solve_batched(q.pack_batch(insts), topk=2, states_cap=16)
    assert len(a) == len(b) == len(insts)
    for ra, rb in zip(a, b):
        assert ra.min == rb.min and ra.n_ties == rb.n_ties
        assert np.array_equal(ra.ties, rb.ties) and np.array_equal(ra.topk, rb.topk)


def test_batched_float(q):
    insts = [wl.sk_float32(n, seed=n) for n in (10, 15, 18, 20, 16)]
    rs = q.solve_batched(insts, topk=2)
    for Q, r in zip(insts, rs):
        check_float(r, oracle.solve(Q, topk=2))


# --- the n=50 configuration, sampled ---------------------------------------------------------

def test_n50_sampled_subcubes(q):
    """The n=50 instance with the plan the benchmark uses (the default variant, 14 walked bits):
    sub-cubes of 2^24 states at 64 sampled prefixes, each checked against the oracle."""
    Q = wl.config5()
    rng = np.random.default_rng(50)
    for v in rng.integers(0, 1 << 26, size=64):
        r = q.solve(Q, topk=16, fix_bits=26, fix_value=int(v), walk_bits=14)
        i = r.info
        # the benchmark's 2^43-state steps plan 14 walked bits with the default variant too
        assert i["acc"] == "i32f" and i["walk_bits"] == 14  # exact in FP32 lanes for this plan
        assert i["split_k"] + i["walk_bits"] + i["suffix_bits"] == 50
        check_int(r, oracle.solve(Q, topk=16, fix_bits=26, fix_value=int(v)))


# --- time limit ------------------------------------------------------------------------------

def test_time_limit_returns_timeout(q):
    Q = wl.upper_int(46, -1000, 1000, seed=1)
    with pytest.raises(q.QuboError) as e:
        q.solve(Q, time_limit=0.2)
    assert e.value.status == q.QUBO_ERR_TIMEOUT
    # the context stays usable
    Q2 = wl.upper_int(20, -10, 10, seed=2)
    check_int(q.solve(Q2), oracle.solve(Q2))


# --- compiled kernel variants and the n=44 FP32 configuration ---------------------------------

@pytest.mark.parametrize("variant", range(24))
def test_scan_variants_agree(q, variant, monkeypatch):
    monkeypatch.setenv("QUBO_SCAN_VARIANT", str(variant))
    Q = wl.upper_int(27, -300, 300, seed=90)
    Qk1 = wl.upper_int(26, -300, 300, seed=91)
    for lanes in ("i32f", "i32"):
        for k, v in LANES[lanes].items():
            monkeypatch.setenv(k, v)
        r = q.solve(Q, topk=16)
        assert r.info["acc"] == lanes
        check_int(r, oracle.solve(Q, topk=16))
        check_int(q.solve(Qk1), oracle.solve(Qk1))
    Qf = wl.sk_float32(25, seed=92)
    r = q.solve(Qf, topk=8)
    assert r.info["acc"] == "f32"
    check_float(r, oracle.solve(Qf, topk=8))


@pytest.mark.parametrize("lim", [3, 300, 60000, 350000])
def test_grouped_form_parity(q, lim, monkeypatch):
    """The grouped step form (the default in FP32 lanes): groups of 16 Gray steps skip the min
    over the columns while a lower bound proves they hold no candidate.  Entries from tie-heavy
    (+-3, most groups reach the threshold, many ties) to the FP32-lane limit (the bound's sum
    rounded down near 2^24; the largest entries leave the FP32 lanes for the int32 kernel, which
    has no grouped form); top-16, K = 1 and the tie set against the oracle."""
    for k, v in LANES["i32f"].items():
        monkeypatch.setenv(k, v)
    for n, seed in ((27, 120 + lim % 7), (29, 121)):
        Q = wl.upper_int(n, -lim, lim, seed=seed)
        # an 8-bit walk: small instances otherwise take a short-body variant
        r = q.solve(Q, topk=16, states_cap=4096, walk_bits=8)
        assert r.info["grouped"] == (r.info["acc"] == "i32f"), r.info
        assert r.info["variant"] == (20 if r.info["acc"] == "i32f" else 16), r.info
        check_int(r, oracle.solve(Q, topk=16, cap=4096))
        r1 = q.solve(Q, states_cap=4096, walk_bits=8)
        check_int(r1, oracle.solve(Q, cap=4096))


def test_grouped_form_fires_on_every_group(q, monkeypatch):
    """All-zero couplings but the diagonal: every state's column part is equal, so every group's
    bound reaches the threshold and the min tree runs everywhere; the 2^k tie set is exact."""
    monkeypatch.setenv("QUBO_NO_I32Z", "1")
    monkeypatch.setenv("QUBO_NO_I16P", "1")
    Q = np.zeros((26, 26), dtype=np.int32)
    Q[np.arange(10), np.arange(10)] = -1  # 2^16 ties: the first 10 variables set, the rest free
    r = q.solve(Q, states_cap=1 << 16, walk_bits=8)
    assert r.info["grouped"] == 1
    check_int(r, oracle.solve(Q, cap=1 << 16))


def test_config3_subcube_stays_fp32(q):
    """The n=44 SK instance: an FP32 scan (no FP64 fallback) on sampled sub-cubes of 2^24
    states, checked against the FP64 oracle."""
    Q = wl.config3()
    for v in (0, 777, 1 << 19):
        r = q.solve(Q, topk=16, fix_bits=20, fix_value=v)
        assert r.info["acc"] == "f32", r.info
        assert 2 * r.info["fp32_max_drift"] < 1e-3 and r.info["fp32_max_abs_err"] < 5e-4
        check_float(r, oracle.solve(Q, topk=16, fix_bits=20, fix_value=v))


# --- device-resident batch replayed as a CUDA graph -------------------------------------------

def test_batch_graph_replays_match_oracle(q):
    insts = wl.config4(count=64, seed=44)
    insts = [Q for Q in insts if Q.shape[0] <= 24][:30] + [wl.upper_int(9, -50, 50, seed=9, dtype=np.int16)]
    b = q.Batch(insts, topk=3, states_cap=32)
    for rep in range(3):  # replays reuse the graph; thresholds and counters are reset each time
        b.run()
        rs = b.fetch()
        for Q, r in zip(insts, rs):
            check_int(r, oracle.solve(Q.astype(np.int32), topk=3, cap=32))
    b.close()


def test_batch_graph_float(q):
    insts = [wl.sk_float32(n, seed=100 + n) for n in (12, 16, 19, 21)]
    b = q.Batch(insts, topk=2)
    b.run()
    for Q, r in zip(insts, b.fetch()):
        check_float(r, oracle.solve(Q, topk=2))
    b.close()


# --- stored oracle results and the autotuner --------------------------------------------------

GOLDEN_DIR = os.path.join(os.path.dirname(__file__), "golden")


def test_config2_matches_golden(q):
    import json

    g = json.load(open(os.path.join(GOLDEN_DIR, "cfg2_n36_top16.json")))
    r = q.solve(wl.config2(), topk=16)
    assert r.min == g["min"] and r.n_ties == g["n_ties"]
    assert [int(c) for c in r.ties] == g["ties"]
    assert [int(c) for c in r.topk] == g["topk"] and [int(e) for e in r.topk_E] == g["topk_E"]


def test_config4_matches_golden(q):
    import json

    path = os.path.join(GOLDEN_DIR, "cfg4_batched.json")
    if not os.path.exists(path):
        pytest.skip("cfg4 golden not generated")
    g = json.load(open(path))
    insts = wl.config4()
    b = q.Batch(insts, topk=0, states_cap=g["cap"])
    b.run()
    rs = b.fetch()
    b.close()
    for row, r in zip(g["instances"], rs):
        assert r.min == row["min"] and r.n_ties == row["n_ties"], row["i"]
        assert [int(c) for c in r.ties] == row["ties"], row["i"]


def test_autotune_installs_a_working_plan(q):
    Q = wl.upper_int(34, -500, 500, seed=55)
    p = q.autotune(Q, fix_bits=8)
    try:
        assert p["trials"] >= 2 and p["states_per_s"] > 0
        r = q.solve(Q, topk=8, fix_bits=6, fix_value=3)
        assert r.info["walk_bits"] == p["walk_bits"]
        check_int(r, oracle.solve(Q, topk=8, fix_bits=6, fix_value=3))
    finally:
        q.autotune_clear()


def test_autotune_plans_persist(q, tmp_path):
    """Tuned plans saved to a file and loaded into a cleared process state are used again; a file
    from another device model installs nothing, and a malformed file is an argument error."""
    Q = wl.upper_int(34, -500, 500, seed=56)
    p = q.autotune(Q, fix_bits=8)
    path = str(tmp_path / "plans.txt")
    try:
        assert q.autotune_save(path) >= 1
        q.autotune_clear()
        assert q.autotune_load(path) >= 1
        r = q.solve(Q, topk=4, fix_bits=6, fix_value=1)
        assert r.info["walk_bits"] == p["walk_bits"]
        check_int(r, oracle.solve(Q, topk=4, fix_bits=6, fix_value=1))
        other = tmp_path / "other.txt"
        other.write_text("qubo-autotune 1\nSome Other GPU\t80\t1\t34\t0\t9\n")
        q.autotune_clear()
        assert q.autotune_load(str(other)) == 0
        bad = tmp_path / "bad.txt"
        bad.write_text("not a plan file\n")
        with pytest.raises(q.QuboError) as e:
            q.autotune_load(str(bad))
        assert e.value.status == q.QUBO_ERR_ARG
    finally:
        q.autotune_clear()


def test_autotune_batched(q):
    insts = [wl.upper_int(n, -100, 100, seed=n, dtype=np.int16) for n in (14, 17, 20, 22, 23)]
    p = q.autotune_batched(insts)
    try:
        assert p["trials"] >= 1
        for Q, r in zip(insts, q.solve_batched(insts, topk=2)):
            check_int(r, oracle.solve(Q.astype(np.int32), topk=2, cap=64))
    finally:
        q.autotune_clear()


def test_autotune_batched_float_and_wide_accumulator(q):
    """The batch autotuner on an FP32 batch (SK instances, n = 18..24) and on an int64 batch
    (entries too wide for int32 energies): the tuned plans run and the results equal the
    oracle's."""
    fl = [wl.sk_float32(n, seed=600 + n) for n in (18, 19, 21, 22, 24)]
    wide = [wl.upper_int(n, -(1 << 26), 1 << 26, seed=700 + n) for n in (17, 20, 23)]
    try:
        for insts, is_float in ((fl, True), (wide, False)):
            q.autotune_clear()
            p = q.autotune_batched(insts)
            assert p["trials"] >= 1
            for Q, r in zip(insts, q.solve_batched(insts, topk=3)):
                o = oracle.solve(Q, topk=3, cap=64)
                if is_float:
                    check_float(r, o)
                else:
                    assert r.info["acc"] == "i64"
                    check_int(r, o)
    finally:
        q.autotune_clear()


def test_autotune_batched_per_size_plans_on_config4(q, tmp_path):
    """The batch autotuner on the 4096-instance configuration: one variant for the launch, a walk
    per instance size; the tuned plans are what the next batch runs (every instance's walk is its
    size's tuned walk), they survive a save / clear / load, and the results equal the oracle's
    stored ones."""
    import json

    path = os.path.join(GOLDEN_DIR, "cfg4_batched.json")
    if not os.path.exists(path):
        pytest.skip("cfg4 golden not generated")
    g = json.load(open(path))
    insts = wl.config4()
    try:
        p = q.autotune_batched(insts)
        walks = p["walk_bits_per_n"]
        assert set(walks) == {int(Q.shape[0]) for Q in insts}, walks
        assert p["trials"] > len(walks) and p["states_per_s"] > 0
        saved = str(tmp_path / "plans.txt")
        assert q.autotune_save(saved) >= 1 + len(walks)
        q.autotune_clear()
        assert q.autotune_load(saved) >= 1 + len(walks)
        b = q.Batch(insts, topk=0, states_cap=g["cap"])
        b.run()
        rs = b.fetch()
        b.close()
        for Q, row, r in zip(insts, g["instances"], rs):
            assert r.info["walk_bits"] == walks[int(Q.shape[0])], (row["i"], r.info["walk_bits"])
            assert r.min == row["min"] and r.n_ties == row["n_ties"], row["i"]
            assert [int(c) for c in r.ties] == row["ties"], row["i"]
    finally:
        q.autotune_clear()


# --- low-energy window (every state within a band above the minimum) --------------------------

def oracle_window(Q, window):
    o = oracle.solve(Q, topk=4096, cap=1)
    sel = o.topk_E <= o.min + window
    assert not sel.all() or len(sel) < 4096, "window too wide for the oracle check"
    return int(sel.sum()), o.topk[sel], o.topk_E[sel]


@pytest.mark.parametrize("n,window", [(12, 40), (16, 150), (21, 60), (24, 0)])
def test_window_matches_oracle(q, n, window):
    Q = wl.upper_int(n, -50, 50, seed=400 + n)
    cnt, codes, E, info = q.solve_window(Q, window)
    ocnt, ocodes, oE = oracle_window(Q, window)
    assert cnt == ocnt and np.array_equal(codes, ocodes) and np.array_equal(E, oE)


@pytest.mark.parametrize("fix_value", [0, 12345, (1 << 22) - 1])
def test_window_n50_subcubes(q, fix_value):
    """The benchmark's window (20000 above the minimum) on the n = 50 instance, on 2^28-state
    sub-cubes: the states in the window are the oracle's, in (E, code) order."""
    Q = wl.config5()
    cnt, codes, E, info = q.solve_window(Q, 20000, fix_bits=22, fix_value=fix_value)
    o = oracle.solve(Q, topk=4096, cap=1, fix_bits=22, fix_value=fix_value)
    sel = o.topk_E <= o.min + 20000
    assert not sel.all()
    assert cnt == int(sel.sum()) and np.array_equal(codes, o.topk[sel]) and np.array_equal(E, o.topk_E[sel])
    assert info["states_scanned"] == 1 << 28


def test_window_float(q):
    Q = wl.sk_float32(20, seed=41)
    cnt, codes, E, info = q.solve_window(Q, 0.5)
    ocnt, ocodes, oE = oracle_window(Q, 0.5)
    assert cnt == ocnt and np.array_equal(codes, ocodes)
    assert np.allclose(E, oE, rtol=FLOAT_RTOL, atol=FLOAT_RTOL)


def test_window_through_overflow_split(q):
    """175 states in the window and room for 128 candidates: the sub-cube splits and merges."""
    code = (
        "import numpy as np, oracle, paper_2607_04857_gb300 as q;"
        "from paper_2607_04857_gb300 import workloads as wl;"
        "Q = wl.upper_int(18, -20, 20, seed=5);"
        "cnt, codes, E, info = q.solve_window(Q, 80, cap=5000);"
        "o = oracle.solve(Q, topk=4096, cap=1); sel = o.topk_E <= o.min + 80;"
        "assert sel.sum() < 4096 and cnt == sel.sum(), (cnt, sel.sum());"
        "assert np.array_equal(codes, o.topk[sel]) and np.array_equal(E, o.topk_E[sel]);"
        "assert info['passes'] > 1, info"
    )
    env = dict(os.environ, QUBO_MAX_RECORDS="128")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    res = subprocess.run([sys.executable, "-c", code], env=env, cwd=root, capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stdout + res.stderr


# --- integer energies in FP32 lanes versus the int32 kernel -----------------------------------

def test_int32_kernel_when_fp32_lanes_disabled(q, monkeypatch):
    monkeypatch.setenv("QUBO_NO_I16P", "1")
    monkeypatch.setenv("QUBO_NO_I32F", "1")
    for n, seed in ((22, 1), (26, 2), (27, 3)):
        Q = wl.upper_int(n, -1000, 1000, seed=seed)
        r = q.solve(Q, topk=16)
        assert r.info["acc"] == "i32"
        check_int(r, oracle.solve(Q, topk=16))


def test_fp32_lanes_rejected_when_out_of_range(q):
    """Entries of +-2^22: column values exceed 2^24, so the int32 kernel must run."""
    Q = wl.upper_int(21, -(1 << 22), 1 << 22, seed=8)
    r = q.solve(Q, topk=8)
    assert not fp32_lanes_fit(Q, r.info["suffix_bits"], r.info["walk_bits"], r.info["reg_rows"])
    assert r.info["acc"] == "i32"
    check_int(r, oracle.solve(Q, topk=8))


@pytest.mark.parametrize("lim", [60000, 120000, 350000, 400000, 1000000])
def test_fp32_lanes_chosen_exactly_when_bounded(q, lim, monkeypatch):
    """Entries sized across the 2^24 bound (the crude S_nf + 2 S_ww bound alone for the
    smallest, the exact range beyond it): the FP32-lane scan is used exactly when the run's plan
    keeps every value it forms below 2^24, and the results are bit-exact either way."""
    monkeypatch.setenv("QUBO_NO_I16P", "1")
    Q = wl.upper_int(27, -lim, lim, seed=9)
    r = q.solve(Q, topk=8, walk_bits=5)  # the same plan for either kernel (both 9 suffix bits)
    check_int(r, oracle.solve(Q, topk=8))
    i = r.info
    assert (i["suffix_bits"], i["walk_bits"], i["reg_rows"]) == (9, 5, 4)  # a 4-register-row variant
    expect = "i32f" if fp32_lanes_fit(Q, 9, 5, 4) else "i32"
    assert i["acc"] == expect
