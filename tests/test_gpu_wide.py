"""Instances wider than one scan (qubo_solve_wide) against the CPU oracle.

The oracle side reduces each outer value's sub-problem with its own code (oracle.reduce, pinned
against exact big-integer energies on the CPU) and solves it; the results are combined here by
energy, then 128-bit code.  Integer results must be bit-exact.
"""
import numpy as np
import pytest

import oracle
from paper_2607_04857_gb300 import workloads as wl

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


def oracle_wide(Q, m, outer_values, topk=0, cap=64):
    """min, tie count, smallest cap tie codes and topk (E, code) over the given outer values."""
    best, n_ties, ties, top = None, 0, [], []
    for v in outer_values:
        R, c = oracle.reduce(Q, m, v)
        r = oracle.solve(R, topk=topk, cap=cap)
        E = r.min + c
        codes = [int(t) | (int(v) << m) for t in r.ties]
        if best is None or E < best:
            best, n_ties, ties = E, 0, []
        if E == best:
            n_ties += r.n_ties
            ties += codes
        top += [(e + c, int(t) | (int(v) << m)) for e, t in zip(r.topk_E.tolist(), r.topk)]
    top.sort()
    return best, n_ties, sorted(ties)[:cap], top[:topk]


def check(r, o, topk):
    mn, n_ties, ties, top = o
    assert r.min == mn and r.n_ties == n_ties
    assert r.ties == ties
    assert r.topk == [c for _, c in top][:topk]
    assert r.topk_E.tolist() == [e for e, _ in top][:topk]


def test_wide_full_range_equals_whole_solve(q):
    """n=30 split 20 + 10: all 1024 outer values (batched sub-problems) equal the whole solve."""
    Q = wl.upper_int(30, -60, 60, seed=30)
    r = q.solve_wide(Q, 20, topk=8, states_cap=256)
    o = oracle.solve(Q, topk=8, cap=256)
    assert r.min == o.min and r.n_ties == o.n_ties
    assert r.ties == [int(t) for t in o.ties]
    assert r.topk == [int(t) for t in o.topk] and r.topk_E.tolist() == o.topk_E.tolist()
    assert r.info["states_scanned"] == 1 << 30


def test_wide_single_outer_value(q):
    """One outer value: the sub-problem path that runs sub-problems one at a time."""
    Q = wl.upper_int(30, -500, 500, seed=31)
    r = q.solve_wide(Q, 22, outer_begin=37, outer_count=1, topk=4)
    o = oracle.solve(Q, topk=4, fix_bits=8, fix_value=37)
    assert r.min == o.min and r.n_ties == o.n_ties
    assert r.ties == [int(t) for t in o.ties] and r.topk == [int(t) for t in o.topk]


@pytest.mark.parametrize("n,m,count", [(70, 24, 5), (75, 30, 1)])
def test_wide_beyond_64_bits(q, n, m, count):
    """Five outer values as one batch, and one outer value alone, of instances above 64 bits."""
    rng = np.random.default_rng(n)
    Q = rng.integers(-3000, 3000, size=(n, n)).astype(np.int32)
    base = int(rng.integers(0, 1 << min(n - m, 62))) & ((1 << (n - m)) - 1)
    base = min(base, (1 << (n - m)) - count)
    r = q.solve_wide(Q, m, outer_begin=base, outer_count=count, topk=6)
    check(r, oracle_wide(Q, m, range(base, base + count), topk=6), 6)
    assert r.info["states_scanned"] == count << m


def test_wide_top_outer_values_of_64_outer_bits(q):
    """n = 96 = 32 inner + 64 outer: the last two outer values (codes beyond bit 63)."""
    rng = np.random.default_rng(96)
    Q = rng.integers(-1000, 1000, size=(96, 96)).astype(np.int16)
    base = (1 << 64) - 2
    r = q.solve_wide(Q, 32, outer_begin=base, outer_count=2, topk=3)
    check(r, oracle_wide(Q.astype(np.int64), 32, [base, base + 1], topk=3), 3)
    assert all(c >> 95 == 1 for c in r.ties)


def test_wide_float(q):
    Q = wl.sk_float32(80, seed=8)
    r = q.solve_wide(Q, 20, outer_begin=1000, outer_count=3, topk=4)
    mn, n_ties, ties, top = oracle_wide(Q.astype(np.float64), 20, range(1000, 1003), topk=4)
    assert abs(r.min - mn) <= 1e-9 * max(1.0, abs(mn))
    assert r.n_ties == n_ties and r.ties == ties
    assert r.topk == [c for _, c in top]


def test_wide_maxcut_ties_and_truncation(q):
    """Max-Cut is symmetric under complementing every variable, so ties come in pairs across
    outer values; a small states_cap truncates with the exact count kept."""
    Q = wl.maxcut_qubo(32, 0.5, seed=34)
    r = q.solve_wide(Q, 20, topk=0, states_cap=1)
    o = oracle.solve(Q.astype(np.int32), cap=1)
    assert r.min == o.min and r.n_ties == o.n_ties and r.n_ties % 2 == 0
    assert r.ties == [int(o.ties[0])]
    assert r.truncated == (o.n_ties > 1)


def test_wide_rejects_bad_ranges(q):
    Q = wl.upper_int(70, -10, 10, seed=1)
    for kw in (dict(n_inner=65), dict(n_inner=5), dict(n_inner=30, outer_begin=1 << 40, outer_count=1),
               dict(n_inner=30, outer_begin=(1 << 40) - 1, outer_count=2), dict(n_inner=30, outer_count=0)):
        with pytest.raises(q.QuboError) as e:
            q.solve_wide(Q, **kw)
        assert e.value.status == q.QUBO_ERR_ARG


def test_wide_benchmark_shape_closed_form(q, monkeypatch):
    """The benchmark's launch shape (n = 80, 40 inner variables, 64 outer values in one batched
    launch, top 16) on an instance whose inner variables couple only to outer ones: each
    sub-problem's minimum is c + sum_i min(0, R_ii) (R, c from oracle.reduce) and its tie count
    2^(number of zero R_ii).  The FP32-lane kernel is forced (the factored and packed scans would
    take such sub-problems)."""
    monkeypatch.setenv("QUBO_NO_I32Z", "1")
    monkeypatch.setenv("QUBO_NO_I16P", "1")
    rng = np.random.default_rng(81)
    n, m, base = 80, 40, 1000
    Q = np.triu(rng.integers(-1000, 1000, size=(n, n))).astype(np.int32)
    Q[:m, :m] = np.diag(np.diag(Q)[:m])
    r = q.solve_wide(Q, m, outer_begin=base, outer_count=64, topk=16, states_cap=64)
    best, ties = None, 0
    for v in range(base, base + 64):
        R, c = oracle.reduce(Q, m, v)
        d = np.diag(R).astype(np.int64)
        e = c + int(np.minimum(d, 0).sum())
        if best is None or e < best:
            best, ties = e, 0
        if e == best:
            ties += 1 << int((d == 0).sum())
    assert r.min == best and r.n_ties == ties
    assert r.info["acc"] == "i32f" and r.info["states_scanned"] == 64 << 40


def test_wide_benchmark_instance_codes(q):
    """The benchmark instance and launch shape: each of the 16 returned states has the reported
    energy (its outer value's sub-problem from oracle.reduce, direct energy), they come in (E, code)
    order, and the sub-problem holding the minimum, solved alone (the unbatched path), agrees."""
    Q = wl.upper_int(80, -1000, 1000, seed=80)
    r = q.solve_wide(Q, 40, outer_begin=0, outer_count=64, topk=16)
    E = r.topk_E.tolist()
    for code, e in zip(r.topk, E):
        R, c = oracle.reduce(Q, 40, code >> 40)
        assert oracle.energy(R, code & ((1 << 40) - 1)) + c == e
    assert list(zip(E, r.topk)) == sorted(zip(E, r.topk)) and E[0] == r.min
    v = r.topk[0] >> 40
    r1 = q.solve_wide(Q, 40, outer_begin=v, outer_count=1, topk=1)
    assert r1.min == r.min and r1.topk[0] == r.topk[0]
