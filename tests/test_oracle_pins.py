"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Every check here compares the oracle with something other than itself: the Gray sequence the
paper prints, closed forms, the matrix form E = diag(X Q X^T) of Sec. 2.1 evaluated by numpy
on every state, invariants (relabelling, Max-Cut complement symmetry, the QUBO/Ising change of
variables), and the direct evaluator against the Gray walk.
"""
import itertools
import os

import numpy as np
import pytest

import oracle
from paper_2607_04857_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def all_states(n):
    codes = np.arange(1 << n, dtype=np.int64)
    X = ((codes[:, None] >> np.arange(n)[None, :]) & 1).astype(np.float64)
    return codes, X


def matrix_form_energies(Q):
    """E = diag(X Q X^T) over all 2^n states (Sec. 2.1, eq. total energy), by numpy."""
    n = Q.shape[0]
    codes, X = all_states(n)
    Qf = np.asarray(Q, dtype=np.float64)
    E = np.einsum("si,ij,sj->s", X, Qf, X)
    if np.asarray(Q).dtype.kind != "f":
        E = np.rint(E).astype(np.int64)
    return codes, E


def brute_reference(Q, K, cap):
    codes, E = matrix_form_energies(Q)
    order = np.lexsort((codes, E))
    emin = E[order[0]]
    ties = np.sort(codes[E == emin])
    return emin, len(ties), ties[:cap], codes[order[:K]], E[order[:K]]


# --- Gray order --------------------------------------------------------------------------

def test_gray_sequence_matches_paper_figure():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "gray3.txt")) if not l.startswith("#")]
    assert len(rows) == 8
    for dec, word in rows:
        assert format(oracle.gray_code(int(dec)), "03b") == word


def test_gray_consecutive_states_differ_in_one_bit():
    for i in range(1, 1 << 12):
        d = oracle.gray_code(i) ^ oracle.gray_code(i - 1)
        assert d & (d - 1) == 0 and d == 1 << ((i & -i).bit_length() - 1)


# --- energies ----------------------------------------------------------------------------

def test_closed_forms():
    rng = np.random.default_rng(7)
    Q = rng.integers(-50, 50, size=(10, 10))
    assert oracle.energy(Q, 0) == 0
    for i in range(10):
        assert oracle.energy(Q, 1 << i) == Q[i, i]
        for j in range(i + 1, 10):
            assert oracle.energy(Q, (1 << i) | (1 << j)) == Q[i, i] + Q[j, j] + Q[i, j] + Q[j, i]


@pytest.mark.parametrize("kind", ["full", "upper", "symmetric"])
def test_direct_energy_equals_matrix_form(kind):
    rng = np.random.default_rng({"full": 1, "upper": 2, "symmetric": 3}[kind])
    n = 9
    Q = rng.integers(-30, 30, size=(n, n))
    if kind == "upper":
        Q = np.triu(Q)
    if kind == "symmetric":
        Q = Q + Q.T
    codes, E = matrix_form_energies(Q)
    for c in codes:
        assert oracle.energy(Q, int(c)) == E[c]
    # the folded upper-triangular matrix has the same energy everywhere
    U = oracle.fold(Q)
    assert np.all(np.tril(U, -1) == 0)
    _, EU = matrix_form_energies(U)
    assert np.array_equal(E, EU)


def test_float_direct_energy_close_to_matrix_form():
    Q = wl.sk_float32(10, seed=11)
    codes, E = matrix_form_energies(Q)
    for c in codes[::7]:
        assert abs(oracle.energy(Q, int(c)) - E[c]) <= 1e-12 * max(1.0, abs(E[c]))


def test_gray_walk_matches_direct():
    Q = wl.upper_int(14, -100, 100, seed=5)
    walk = oracle.gray_walk(Q)
    codes, E = matrix_form_energies(Q)
    g = codes ^ (codes >> 1)
    assert np.array_equal(walk, E[g])


# --- whole solves against brute force ------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 12])
@pytest.mark.parametrize("method", [oracle.DIRECT, oracle.GRAY])
def test_int_solve_matches_bruteforce(n, method):
    rng = np.random.default_rng(100 + n)
    for trial in range(3):
        Q = rng.integers(-8, 8, size=(n, n))  # small range: many ties
        K = min(1 << n, 16)
        emin, nt, ties, tk, tkE = brute_reference(Q, K, cap=1 << n)
        r = oracle.solve(Q, method=method, topk=K, cap=1 << n)
        assert r.min == emin and r.n_ties == nt
        assert np.array_equal(r.ties, ties)
        assert np.array_equal(r.topk, tk) and np.array_equal(r.topk_E, tkE)


@pytest.mark.parametrize("method", [oracle.DIRECT, oracle.GRAY])
def test_float_solve_matches_bruteforce(method):
    for seed in range(4):
        Q = wl.sk_float32(11, seed=seed)
        emin, nt, ties, tk, tkE = brute_reference(Q, 8, cap=16)
        r = oracle.solve(Q, method=method, topk=8, cap=16)
        assert abs(r.min - emin) <= 1e-12 * max(1.0, abs(emin))
        assert np.array_equal(r.ties, ties) and r.n_ties == nt == 1
        assert np.array_equal(r.topk, tk)
        assert np.allclose(r.topk_E, tkE, rtol=1e-12, atol=1e-12)


def test_gray_equals_direct_n20():
    for seed in range(3):
        Q = wl.upper_int(20, -30, 30, seed=seed)
        a = oracle.solve(Q, method=oracle.DIRECT, topk=16)
        b = oracle.solve(Q, method=oracle.GRAY, topk=16)
        assert a.min == b.min and a.n_ties == b.n_ties
        assert np.array_equal(a.ties, b.ties)
        assert np.array_equal(a.topk, b.topk) and np.array_equal(a.topk_E, b.topk_E)


def test_float_gray_equals_direct_n18():
    Q = wl.sk_float32(18, seed=9)
    a = oracle.solve(Q, method=oracle.DIRECT, topk=16)
    b = oracle.solve(Q, method=oracle.GRAY, topk=16)
    assert a.min == b.min  # both decided by the direct FP64 evaluator
    assert np.array_equal(a.ties, b.ties)
    assert np.array_equal(a.topk, b.topk) and np.array_equal(a.topk_E, b.topk_E)
    assert b.n_candidates < (1 << 18) // 8  # the walk really pre-selects


def fixed_order_energies(Q):
    """FP64 energies of every state summed in the direct evaluator's defining order (i
    ascending, then j ascending over the folded upper triangle), by numpy over all states at
    once.  A term of an unset variable adds nothing (adding 0.0 leaves every FP64 value
    unchanged), so this is the same rounding sequence, written independently."""
    Q = np.asarray(Q, dtype=np.float64)
    n = Q.shape[0]
    U = np.triu(Q + Q.T, 1) + np.diag(np.diag(Q))
    codes = np.arange(1 << n, dtype=np.int64)
    X = ((codes[:, None] >> np.arange(n)[None, :]) & 1).astype(bool)
    acc = np.zeros(1 << n)
    for i in range(n):
        acc = np.where(X[:, i], acc + U[i, i], acc)
        for j in range(i + 1, n):
            acc = np.where(X[:, i] & X[:, j], acc + U[i, j], acc)
    return codes, acc


@pytest.mark.parametrize("n,seed", [(16, 0), (17, 1), (18, 0), (18, 1), (18, 2)])
@pytest.mark.parametrize("K", [1, 16])
def test_float_gray_preselection_keeps_ulp_near_ties(n, seed, K):
    """Brute force defines the answer (Sec. 1.4): with the FP64 energy fixed by the direct
    order, the Gray walk's candidate pre-selection must keep every state of the tie set and
    of the K lowest although its own running energies round differently.  The instances have
    3^(n//2) exact-arithmetic minimisers split by one or two roundings, and 2^16-step walks
    cross the re-anchoring period many times.  A pre-selection without its rounding
    tolerance drops many of them."""
    Q = wl.decimal_pairs(n, seed=seed)
    codes, E = fixed_order_energies(Q)
    emin = E.min()
    ties = codes[E == emin]
    near = np.count_nonzero(np.abs(E - emin) <= 1e-12)
    assert near == 3 ** (n // 2) and len(ties) < near  # rounding really splits the real ties
    order = np.lexsort((codes, E))
    for method in (oracle.GRAY, oracle.DIRECT):
        r = oracle.solve(Q, method=method, topk=K, cap=1 << 16)
        assert r.min == emin and r.n_ties == len(ties)
        assert np.array_equal(r.ties, ties)
        assert np.array_equal(r.topk, codes[order[:K]])
        assert np.array_equal(r.topk_E, E[order[:K]])


@pytest.mark.parametrize("method", [oracle.DIRECT, oracle.GRAY])
def test_float_zero_matrix_every_state_ties(method):
    """Float Q = 0: every state has energy exactly 0 and ties with the minimum; the Gray
    pre-selection's tolerance is then 0 and only a non-strict comparison keeps the states."""
    n = 16
    Q = np.zeros((n, n), dtype=np.float32)
    r = oracle.solve(Q, method=method, topk=5, cap=100)
    assert r.min == 0.0 and r.n_ties == 1 << n and r.truncated
    assert np.array_equal(r.ties, np.arange(100, dtype=np.uint64))
    assert np.array_equal(r.topk, np.arange(5, dtype=np.uint64))


# --- special cases with known answers -------------------------------------------------------

@pytest.mark.parametrize("method", [oracle.DIRECT, oracle.GRAY])
def test_diagonal_closed_form(method):
    n, z = 14, 5
    Q = wl.diagonal(n, seed=3, zeros=z)
    d = np.diag(Q).astype(np.int64)
    r = oracle.solve(Q, method=method, cap=1 << n)
    assert r.min == int(np.minimum(d, 0).sum())
    assert r.n_ties == 1 << z
    neg = sum(1 << i for i in range(n) if d[i] < 0)
    zero_bits = [i for i in range(n) if d[i] == 0]
    expect = sorted(neg | sum(1 << zero_bits[b] for b in range(z) if (m >> b) & 1) for m in range(1 << z))
    assert np.array_equal(r.ties, np.array(expect, dtype=np.uint64))


@pytest.mark.parametrize("method", [oracle.DIRECT, oracle.GRAY])
def test_zero_matrix_truncation(method):
    n = 16
    Q = np.zeros((n, n), dtype=np.int32)
    r = oracle.solve(Q, method=method, topk=5, cap=100)
    assert r.min == 0 and r.n_ties == 1 << n and r.truncated
    assert np.array_equal(r.ties, np.arange(100, dtype=np.uint64))
    assert np.array_equal(r.topk, np.arange(5, dtype=np.uint64))


def test_planted_unique_argmin():
    for seed in range(3):
        Q, xs = wl.planted(22, seed=seed)
        r = oracle.solve(Q)
        assert r.n_ties == 1 and int(r.ties[0]) == xs
        assert r.min == int(np.minimum(np.diag(Q), 0).sum())


def test_maxcut_energy_is_minus_cut_and_complement_symmetric():
    n = 12
    Q = wl.maxcut_qubo(n, 0.5, seed=21)
    # rebuild the graph from the same draw and count cut weights directly
    rng = np.random.Generator(np.random.PCG64(21))
    iu = np.triu_indices(n, k=1)
    edge = rng.random(len(iu[0])) < 0.5
    w = np.where(rng.random(len(iu[0])) < 0.5, -1, 1) * edge
    full = (1 << n) - 1
    for x in range(0, 1 << n, 37):
        bits = [(x >> i) & 1 for i in range(n)]
        cut = sum(int(w[e]) for e in range(len(w)) if bits[iu[0][e]] != bits[iu[1][e]])
        assert oracle.energy(Q, x) == -cut
        assert oracle.energy(Q, x) == oracle.energy(Q, full ^ x)
    r = oracle.solve(Q, cap=1 << n)
    ties = set(int(t) for t in r.ties)
    assert r.n_ties % 2 == 0 and all((full ^ t) in ties for t in ties)


def test_relabelling_invariance():
    n = 15
    Q = wl.upper_int(n, -20, 20, seed=8)
    perm = np.random.default_rng(1).permutation(n)  # new variable a is old variable perm[a]
    Qp = Q[np.ix_(perm, perm)]
    a = oracle.solve(Q, cap=1 << n)
    b = oracle.solve(Qp, cap=1 << n)
    assert a.min == b.min and a.n_ties == b.n_ties

    def to_old(code):
        return sum(1 << int(perm[i]) for i in range(n) if (code >> i) & 1)

    assert sorted(to_old(int(c)) for c in b.ties) == [int(c) for c in a.ties]


def test_qubo_ising_correspondence():
    """x = (1 + s)/2 maps E(x) to H(s) + const with J_ij = U_ij/4 (i < j),
    h_i = U_ii/2 + sum_{j != i} U_ij/4 and const = sum_i U_ii/2 + sum_{i<j} U_ij/4."""
    n = 12
    Q = wl.upper_int(n, -40, 40, seed=4)
    U = oracle.fold(Q).astype(np.float64)
    J = np.triu(U, 1) / 4.0
    Us = np.triu(U, 1) + np.triu(U, 1).T
    h = np.diag(U) / 2.0 + Us.sum(1) / 4.0
    const = np.diag(U).sum() / 2.0 + np.triu(U, 1).sum() / 4.0
    codes, X = all_states(n)
    S = 2 * X - 1
    H = np.einsum("si,ij,sj->s", S, J, S) + S @ h
    _, E = matrix_form_energies(Q)
    assert np.allclose(E, H + const, atol=1e-9)
    r = oracle.solve(Q)
    assert r.min == pytest.approx(H.min() + const, abs=1e-9)


def test_subcube_results_merge_to_full():
    n, f = 18, 2
    Q = wl.upper_int(n, -25, 25, seed=12)
    full = oracle.solve(Q, topk=8, cap=1 << n)
    parts = [oracle.solve(Q, topk=8, cap=1 << n, fix_bits=f, fix_value=v) for v in range(1 << f)]
    mn = min(p.min for p in parts)
    assert mn == full.min
    assert sum(p.n_ties for p in parts if p.min == mn) == full.n_ties
    ties = np.sort(np.concatenate([p.ties for p in parts if p.min == mn]))
    assert np.array_equal(ties, full.ties)
    allk = sorted((int(e), int(c)) for p in parts for e, c in zip(p.topk_E, p.topk))[:8]
    assert [c for _, c in allk] == [int(c) for c in full.topk]
    for v, p in enumerate(parts):
        assert all(int(c) >> (n - f) == v for c in p.topk)


def test_rate_convention_from_paper_tables():
    """states/s = 2^N / total time: the H100 row of the raw-time table (N=50, 151.2 s) and the
    state-rate table (7.47e12) agree under this reading (Sec. 5.3, Tables 1 and 3)."""
    assert 2**50 / 151.2 == pytest.approx(7.45e12, rel=2e-3)
    assert 2**46 / 13690 == pytest.approx(5.1e9, rel=1e-2)


# --- sub-problems with fixed variables (Sec. 3.3.1; Sec. 4.3 for instances wider than a scan) ---

def bigint_energy(Q, x: int) -> int:
    """E(x) = sum_ij Q_ij x_i x_j over the unfolded matrix in exact Python integers (any n)."""
    on = [i for i in range(Q.shape[0]) if (x >> i) & 1]
    return sum(int(Q[i, j]) for i in on for j in on)


@pytest.mark.parametrize("n,m", [(70, 30), (100, 64), (9, 4), (20, 20)])
def test_reduce_matches_exact_energy_beyond_64_bits(n, m):
    rng = np.random.default_rng(n + m)
    Q = rng.integers(-5000, 5000, size=(n, n))  # full, non-symmetric: the fold is exercised
    for _ in range(25):
        x = int.from_bytes(rng.bytes(16), "little") & ((1 << n) - 1)
        R, c = oracle.reduce(Q, m, x >> m)
        assert R.shape == (m, m) and np.all(np.tril(R, -1) == 0)
        assert oracle.energy(R, x & ((1 << m) - 1)) + c == bigint_energy(Q, x)


def test_reduce_float_matches_exact_energy():
    import math

    n, m = 90, 25
    Q = wl.sk_float32(n, seed=7).astype(np.float64)
    rng = np.random.default_rng(1)
    for _ in range(20):
        x = int.from_bytes(rng.bytes(12), "little") & ((1 << n) - 1)
        on = [i for i in range(n) if (x >> i) & 1]
        exact = math.fsum(float(Q[i, j]) for i in on for j in on)
        R, c = oracle.reduce(Q, m, x >> m)
        got = oracle.energy(R, x & ((1 << m) - 1)) + c
        assert got == pytest.approx(exact, rel=1e-12, abs=1e-12)


def test_reduced_subproblems_equal_subcube_solves():
    """For n <= 64 the sub-problem of outer value v is the sub-cube whose top bits are v: its
    minimum plus c, and its tie codes with v above them, equal the sub-cube solve."""
    n, m = 22, 15
    Q = wl.upper_int(n, -40, 40, seed=21)
    for v in (0, 1, 77, (1 << (n - m)) - 1):
        R, c = oracle.reduce(Q, m, v)
        r = oracle.solve(R, topk=5)
        s = oracle.solve(Q, topk=5, fix_bits=n - m, fix_value=v)
        assert r.min + c == s.min and r.n_ties == s.n_ties
        assert [int(t) | (v << m) for t in r.ties] == [int(t) for t in s.ties]
        assert [int(t) | (v << m) for t in r.topk] == [int(t) for t in s.topk]
        assert [int(e) + c for e in r.topk_E] == [int(e) for e in s.topk_E]
