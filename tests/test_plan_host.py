"""The host's planning (qubo_plan_query), which needs no GPU: the accumulator and kernel shape
each benchmark instance gets, and the admission of the packed 16-bit and FP32-lane scans checked
against numpy restatements of their exactness conditions."""
import numpy as np
import pytest

from paper_2607_04857_gb300 import workloads as wl
from plan_checks import column_range, fp32_lanes_fit


@pytest.fixture(scope="module")
def q():
    from paper_2607_04857_gb300 import build as qbuild

    qbuild.build()
    import paper_2607_04857_gb300 as q

    q.load_library()
    return q


def shape(p):
    return p["acc"], p["walk_bits"], p["suffix_bits"]


def test_benchmark_plans(q, monkeypatch):
    monkeypatch.delenv("QUBO_SCAN_VARIANT", raising=False)
    q.autotune_clear()
    # n = 50 int32 (2^43-state steps): integers in FP32 lanes, 2^14-step walks, 16 columns
    p = q.plan_query(wl.config5(), topk=16, fix_bits=7)
    assert shape(p) == ("i32f", 14, 9) and p["split_k"] == 27
    # n = 44 FP32 (2^42): FP32, 2^14-step walks re-anchored every 2^10 steps
    p = q.plan_query(wl.config3(), fix_bits=2)
    assert shape(p) == ("f32", 14, 9) and p["anchor_bits"] == 10
    # Max-Cut n = 48 (2^42): factored scan, 3 factored rows, 64 columns
    p = q.plan_query(wl.maxcut_qubo(48, 0.5, seed=48), topk=16, fix_bits=6)
    assert shape(p) == ("i32z", 12, 11) and p["zero_rows"] == 3
    # sparse n = 56 (2^46): every walked row factored (one block per unit)
    for Q, acc in ((wl.sparse_int(56, 0.05, -1000, 1000, seed=56), "i32z"), (wl.sparse_float32(56, 0.05, seed=56), "f32z")):
        p = q.plan_query(Q, topk=16, fix_bits=10)
        assert shape(p) == (acc, 14, 11) and p["zero_rows"] == 14
    # the plain form runs in the plain accumulators
    assert q.plan_query(wl.config5(), fix_bits=7, plain=True)["acc"] == "i64"
    assert q.plan_query(wl.config3(), fix_bits=2, plain=True)["acc"] == "f64"


@pytest.mark.parametrize("lim", [60000, 120000, 350000, 400000, 1000000])
def test_fp32_lane_admission(q, lim, monkeypatch):
    """The FP32-lane scan is planned exactly when every value its plan forms stays below 2^24."""
    monkeypatch.setenv("QUBO_NO_I16P", "1")
    monkeypatch.setenv("QUBO_NO_I32Z", "1")
    Q = wl.upper_int(27, -lim, lim, seed=9)
    p = q.plan_query(Q, topk=8, walk_bits=5)
    # a 5-bit walk is shorter than the default variant takes: the 4-register-row variant runs
    assert (p["suffix_bits"], p["walk_bits"], p["reg_rows"]) == (9, 5, 4)
    assert p["acc"] == ("i32f" if fp32_lanes_fit(Q, 9, 5, 4) else "i32")


@pytest.mark.parametrize("lim", [300, 900, 1400, 2000, 3000])
def test_packed_admission(q, lim, monkeypatch):
    """The packed 16-bit scan is planned exactly when the plan's column range fits 16 bits."""
    monkeypatch.setenv("QUBO_NO_I32Z", "1")
    Q = wl.upper_int(24, -lim, lim, seed=11)
    p = q.plan_query(Q, topk=8, walk_bits=6)
    lo, hi = column_range(Q, 10, 6, 5)  # default packed variant: 10 suffix bits, 5 register rows
    assert (p["acc"] == "i16p") == (lo >= -32768 and hi <= 32767), (lo, hi, p)


def test_fp32_lanes_fall_back_to_shorter_walks(q, monkeypatch):
    """Large couplings among variables 13..22 only: with 2^14-step walks variables 21 and 22 are
    walked and E_L leaves the FP32 lanes' exact range, with 2^12-step walks they are fixed and
    those couplings go to the int32 prefix part.  The planner takes the shorter walk rather than
    the int32 kernel; with moderate couplings it keeps the longer one."""
    monkeypatch.setenv("QUBO_NO_I16P", "1")
    monkeypatch.setenv("QUBO_NO_I32Z", "1")
    for big, expect in ((400000, 14), (600000, 12), (800000, 12)):
        Q = wl.upper_int(40, -1000, 1000, seed=40)
        Q[13:21, 21:23] = big
        Q[21, 22] = big
        p = q.plan_query(Q, fix_bits=2)
        rc = p["reg_rows"]
        assert fp32_lanes_fit(Q, 9, 14, rc) == (expect == 14) and fp32_lanes_fit(Q, 9, 12, rc)
        assert (p["acc"], p["walk_bits"]) == ("i32f", expect), (big, p)


def test_factored_rows_of_a_diagonal_instance(q):
    """A diagonal instance has no couplings at all: every walked row is factored out."""
    Q = np.diag(np.arange(-15, 15, dtype=np.int32))
    p = q.plan_query(Q)
    assert p["acc"] == "i32z" and p["zero_rows"] == p["walk_bits"]


def test_plan_query_rejects_bad_arguments(q):
    Q = wl.upper_int(20, -5, 5, seed=1)
    for kw in (dict(fix_bits=21), dict(topk=q.QUBO_MAX_TOPK + 1)):
        with pytest.raises(q.QuboError) as e:
            q.plan_query(Q, **kw)
        assert e.value.status == q.QUBO_ERR_ARG


@pytest.mark.parametrize("seed", range(6))
def test_plan_shapes_are_consistent(q, seed):
    """For random instances and sub-cubes: n = split_k + walk_bits + suffix_bits whenever the scan
    is split (else the sub-cube is evaluated directly), a dense walk covers at least one unrolled
    body (a factored one at least its 3 factored rows), and the fixed bits of a unit include the
    sub-cube's."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(12, 64))
    kind = seed % 3
    Q = (wl.upper_int(n, -300, 300, seed=seed) if kind == 0 else
         wl.sparse_int(n, 0.1, -300, 300, seed=seed) if kind == 1 else wl.sk_float32(n, seed=seed))
    for fb in sorted({0, n // 4, n // 2, max(0, n - 30)}):
        if n - fb > 63:
            continue
        p = q.plan_query(Q, fix_bits=fb)
        if p["suffix_bits"] == 0:  # evaluated directly
            assert p["walk_bits"] == 0
            continue
        assert p["split_k"] + p["walk_bits"] + p["suffix_bits"] == n, p
        factored = p["acc"] in ("i32z", "f32z")
        assert p["split_k"] >= fb and p["walk_bits"] >= (3 if factored else p["reg_rows"] + 1), p
        assert factored or p["reg_rows"] >= 2, p
        if factored:
            assert 3 <= p["zero_rows"] <= p["walk_bits"], p


@pytest.mark.parametrize("case", ["n44_step", "n44_subcube", "sk30", "n26_walk8"])
def test_fp32_rounding_bound_matches_its_definition(q, case):
    """The FP32 scan's worst-case rounding bound the host reports (qubo_result.fp32_err_bound)
    equals the bound recomputed in numpy from the folded matrix and the plan (tests/plan_checks.py
    states it term by term), at the run's period and, through the margin, at the longest period
    the bound admits; the rigorous option anchors there, or scans in FP64 when no period does."""
    from plan_checks import fp32_bound

    Q, kw = {"n44_step": (wl.config3(), dict(fix_bits=2)),
             "n44_subcube": (wl.config3(), dict(fix_bits=6, fix_value=37)),
             "sk30": (wl.sk_float32(30, seed=3), {}),
             "n26_walk8": (wl.sk_float32(26, seed=4), dict(walk_bits=8))}[case]
    p = q.plan_query(Q, **kw)
    B, L, RC = p["suffix_bits"], p["walk_bits"], p["reg_rows"]
    assert p["acc"] == "f32" and p["anchor_bits"] == min(10, L) and RC >= 2
    ref = fp32_bound(Q, B, L, RC, p["anchor_bits"])
    assert p["fp32_err_bound"] == pytest.approx(ref, rel=1e-9)
    bounds = [fp32_bound(Q, B, L, RC, a) for a in range(RC + 1, L + 1)]
    assert all(x < y for x, y in zip(bounds, bounds[1:]))  # longer periods, larger bound
    for margin in (1e-4, 1e-3, 3e-3, 1e-2):
        pm = q.plan_query(Q, margin=margin, **kw)
        a = pm["fp32_rigorous_anchor_bits"]
        fits = [RC + 1 + i for i, b in enumerate(bounds) if 2 * b <= margin]
        assert a == (max(fits) if fits else -1), (margin, a, fits)
        pr = q.plan_query(Q, margin=margin, rigorous=True, **kw)
        if a < 0:
            assert pr["acc"] == "f64"
        else:
            assert pr["acc"] == "f32" and pr["anchor_bits"] == min(10, a)
            assert 2 * pr["fp32_err_bound"] <= margin


def test_fp32_rigorous_period_of_the_benchmark_instance(q):
    """n = 44 SK instance in the benchmark's plan (2^14-step walks): the bound at the default
    2^10-step period is above what the 1e-3 margin admits (there correctness rests on the drift
    measured at every re-anchoring); re-anchoring every 2^6 steps is proven."""
    p = q.plan_query(wl.config3(), fix_bits=2)
    assert p["walk_bits"] == 14 and p["anchor_bits"] == 10
    assert 2 * p["fp32_err_bound"] > 1e-3
    assert p["fp32_rigorous_anchor_bits"] == 6
