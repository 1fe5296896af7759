"""Packed 16-bit scan (two biased 16-bit columns per 32-bit word) against the CPU oracle.

Small-coefficient integer instances (Max-Cut, int16 entries in [-127, 127]) are scanned in
packed lanes when the run's plan provably keeps every column value in [-32768, 32767]; results
must be bit-exact: minimum, exact tie count, tie codes, K lowest states and energies.
"""
import numpy as np
import pytest

import oracle
from paper_2607_04857_gb300 import workloads as wl
from plan_checks import column_range

pytestmark = pytest.mark.gpu


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


@pytest.fixture(autouse=True)
def dense_kernels_only(monkeypatch):
    """These instances test the packed scan; keep the factored sparse scan out of the way."""
    monkeypatch.setenv("QUBO_NO_I32Z", "1")


def check_int(r, o):
    assert r.min == o.min, (r.min, o.min)
    assert r.n_ties == o.n_ties, (r.n_ties, o.n_ties)
    assert np.array_equal(r.ties, o.ties), (r.ties[:8], o.ties[:8])
    assert np.array_equal(r.topk, o.topk), (r.topk, o.topk)
    assert np.array_equal(r.topk_E, o.topk_E), (r.topk_E, o.topk_E)


@pytest.mark.parametrize("n", [15, 18, 24, 28, 31])
@pytest.mark.parametrize("topk", [0, 16])
def test_packed_maxcut(q, n, topk):
    for seed in range(2):
        Q = wl.maxcut_qubo(n, 0.5, seed=100 * n + seed)
        r = q.solve(Q, topk=topk)
        assert r.info["acc"] == "i16p", r.info
        check_int(r, oracle.solve(Q.astype(np.int32), topk=topk))


@pytest.mark.parametrize("n", [16, 21, 26, 30])
@pytest.mark.parametrize("topk", [0, 1, 7])
def test_packed_int16(q, n, topk):
    Q = wl.upper_int(n, -127, 127, seed=300 + n, dtype=np.int16)
    r = q.solve(Q, topk=topk)
    assert r.info["acc"] == "i16p", r.info
    assert r.info["cols_per_thread"] == 2 * 16  # default packed variant: 16 words per thread
    check_int(r, oracle.solve(Q.astype(np.int32), topk=topk))


def test_packed_dense_maxcut_ties(q):
    """Complete graph with unit weights: the cut is maximal for every balanced bipartition, so
    the tie set is large and has a closed-form size, C(n, n/2)."""
    from math import comb

    n = 20
    iu = np.triu_indices(n, 1)
    Q = np.zeros((n, n), dtype=np.int16)
    Q[iu] = 2
    Q[np.arange(n), np.arange(n)] = -(n - 1)
    r = q.solve(Q, states_cap=1 << 18)
    assert r.info["acc"] == "i16p"
    assert r.min == -(n // 2) ** 2 and r.n_ties == comb(n, n // 2)
    check_int(r, oracle.solve(Q.astype(np.int32), cap=1 << 18))


@pytest.mark.parametrize("lim", [300, 900, 1400, 2000, 3000])
def test_packed_chosen_exactly_when_bounded(q, lim):
    """Entries sized around the 16-bit bound: the packed scan runs exactly when the plan's
    column range fits 16 bits, and the results are bit-exact whichever kernel runs."""
    Q = wl.upper_int(24, -lim, lim, seed=11)
    r = q.solve(Q, topk=8, walk_bits=6)
    check_int(r, oracle.solve(Q, topk=8))
    i = r.info
    if i["acc"] == "i16p":
        assert (i["suffix_bits"], i["walk_bits"]) == (10, 6)
    lo, hi = column_range(Q, 10, 6, 5)  # default packed variant: 5 register rows
    assert (i["acc"] == "i16p") == (lo >= -32768 and hi <= 32767), (lo, hi, i["acc"])


@pytest.mark.parametrize("variant", range(24))
def test_packed_variants_agree(q, variant, monkeypatch):
    monkeypatch.setenv("QUBO_SCAN_VARIANT", str(variant))
    Q = wl.maxcut_qubo(29, 0.5, seed=91)
    r = q.solve(Q, topk=16)
    assert r.info["acc"] == "i16p"
    check_int(r, oracle.solve(Q.astype(np.int32), topk=16))
    Qk1 = wl.upper_int(27, -127, 127, seed=92, dtype=np.int16)
    r = q.solve(Qk1)
    assert r.info["acc"] == "i16p"
    check_int(r, oracle.solve(Qk1.astype(np.int32)))


@pytest.mark.parametrize("fused", [True, False])
def test_packed_fused_and_separate_el(q, fused, monkeypatch):
    """The packed scan adds E_L to a step's packed column minima as one 32-bit add when the host
    proves no half can carry (the default when it can), else combines the halves first; both
    give the oracle's results, on Max-Cut and int16-entry instances and a walk of 2^12 steps."""
    if not fused:
        monkeypatch.setenv("QUBO_NO_PACKED_FUSED", "1")
    for Q, kw in ((wl.maxcut_qubo(30, 0.5, seed=77), {}), (wl.upper_int(29, -127, 127, seed=78, dtype=np.int16), {}),
                  (wl.upper_int(31, -127, 127, seed=79, dtype=np.int16), {"walk_bits": 12})):
        r = q.solve(Q, topk=16, **kw)
        assert r.info["acc"] == "i16p"
        check_int(r, oracle.solve(Q.astype(np.int32), topk=16))


@pytest.mark.parametrize("walk_bits", [4, 5, 7, 10, 13])
def test_packed_plan_shapes(q, walk_bits):
    Q = wl.upper_int(28, -60, 60, seed=12, dtype=np.int16)
    r = q.solve(Q, topk=16, walk_bits=walk_bits)
    assert r.info["acc"] == "i16p" and r.info["walk_bits"] == walk_bits
    check_int(r, oracle.solve(Q.astype(np.int32), topk=16))


def test_packed_subcubes(q):
    """n=38 Max-Cut: sampled sub-cubes of 2^26 states, each against the oracle."""
    Q = wl.maxcut_qubo(38, 0.5, seed=38)
    for v in (0, 5, 200, 4095):
        r = q.solve(Q, topk=4, fix_bits=12, fix_value=v)
        assert r.info["acc"] == "i16p"
        check_int(r, oracle.solve(Q.astype(np.int32), topk=4, fix_bits=12, fix_value=v))


def test_packed_window(q):
    Q = wl.maxcut_qubo(22, 0.4, seed=7)
    o = oracle.solve(Q.astype(np.int32), topk=4096, cap=1)
    sel = o.topk_E <= o.min + 3
    assert not sel.all()
    cnt, codes, E, info = q.solve_window(Q, 3)
    assert info["acc"] == "i16p"
    assert cnt == int(sel.sum())
    assert np.array_equal(codes, o.topk[sel]) and np.array_equal(E, o.topk_E[sel])


def test_packed_overflow_split(q, monkeypatch):
    """A candidate buffer far too small: the run splits its sub-cube and stays exact."""
    monkeypatch.setenv("QUBO_MAX_RECORDS", "200")
    Q = wl.maxcut_qubo(24, 0.3, seed=5)
    r = q.solve(Q, topk=32, states_cap=4096)
    assert r.info["acc"] == "i16p"
    check_int(r, oracle.solve(Q.astype(np.int32), topk=32, cap=4096))


def test_packed_batch(q):
    insts = [Q for Q in wl.config4(count=80, seed=45) if Q.shape[0] <= 25][:40]
    rs = q.solve_batched(insts, topk=2, states_cap=32)
    assert rs[0].info["acc"] == "i16p"
    for Q, r in zip(insts, rs):
        check_int(r, oracle.solve(Q.astype(np.int32), topk=2, cap=32))
    b = q.Batch(insts, topk=2, states_cap=32)
    for _ in range(2):
        b.run()
        for Q, r in zip(insts, b.fetch()):
            assert r.info["acc"] == "i16p"
            check_int(r, oracle.solve(Q.astype(np.int32), topk=2, cap=32))
    b.close()


def test_packed_disabled_falls_back(q, monkeypatch):
    monkeypatch.setenv("QUBO_NO_I16P", "1")
    Q = wl.maxcut_qubo(25, 0.5, seed=3)
    r = q.solve(Q, topk=5)
    assert r.info["acc"] == "i32f"
    check_int(r, oracle.solve(Q.astype(np.int32), topk=5))
