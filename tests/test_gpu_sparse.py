"""Factored scan of sparse integer instances against the CPU oracle.

Instances whose variables can be ordered so that at least three walked prefix variables have no
coupling to any suffix variable run the factored scan (accumulator "i32z"): the minimum over
those variables' patterns separates from the minimum over the columns.  Results must be
bit-exact with the oracle in the caller's variable order: minimum, exact tie count, tie codes,
K lowest states and energies.
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


def check_int(r, o):
    assert r.min == o.min, (r.min, o.min)
    assert r.n_ties == o.n_ties, (r.n_ties, o.n_ties)
    assert np.array_equal(r.ties, o.ties), (r.ties[:8], o.ties[:8])
    assert np.array_equal(r.topk, o.topk), (r.topk, o.topk)
    assert np.array_equal(r.topk_E, o.topk_E), (r.topk_E, o.topk_E)


@pytest.mark.parametrize("n", [16, 20, 25, 30])
@pytest.mark.parametrize("topk", [0, 1, 16])
def test_sparse_parity(q, n, topk):
    for seed in range(2):
        Q = wl.sparse_int(n, 0.1, -500, 500, seed=100 * n + seed)
        r = q.solve(Q, topk=topk)
        assert r.info["acc"] == "i32z", r.info
        check_int(r, oracle.solve(Q, topk=topk))


def test_sparse_maxcut_tie_pairs(q):
    """Sparse Max-Cut: complementing every variable keeps the cut, so ties come in pairs."""
    Q = wl.maxcut_qubo(30, 0.1, seed=3, dtype=np.int32)
    r = q.solve(Q, topk=8, states_cap=4096)
    assert r.info["acc"] == "i32z"
    o = oracle.solve(Q, topk=8, cap=4096)
    check_int(r, o)
    assert r.n_ties % 2 == 0


@pytest.mark.parametrize("walk_bits", [3, 5, 8, 12])
def test_sparse_plan_shapes(q, walk_bits):
    Q = wl.sparse_int(28, 0.08, -100, 100, seed=7)
    r = q.solve(Q, topk=12, walk_bits=walk_bits)
    assert r.info["acc"] == "i32z" and r.info["walk_bits"] == walk_bits
    check_int(r, oracle.solve(Q, topk=12))


@pytest.mark.parametrize("n,units", [(25, 1), (26, 2), (28, 8), (29, 16)])
def test_one_block_kernel_unit_pairing(q, n, units):
    """The one-block kernel scans the units of a claim two at a time (one E_L pass for both); a
    claim with a single unit left is scanned alone.  Diagonal-dominated instances factor every
    walked row, so the kernel runs with 1, 2, 8 and 16 units of 2^25 states."""
    Q = wl.sparse_int(n, 0.02, -100, 100, seed=n)
    Q[np.arange(n), np.arange(n)] = np.random.default_rng(n).integers(-400, 400, size=n)
    r = q.solve(Q, topk=12, walk_bits=14)
    i = r.info
    assert (i["acc"], i["zero_rows"], 1 << i["split_k"]) == ("i32z", 14, units), i
    check_int(r, oracle.solve(Q, topk=12))


def test_sparse_subcubes(q):
    Q = wl.sparse_int(40, 0.06, -1000, 1000, seed=40)
    for v in (0, 3, 1000, (1 << 14) - 1):
        r = q.solve(Q, topk=4, fix_bits=14, fix_value=v)
        assert r.info["acc"] == "i32z"
        check_int(r, oracle.solve(Q, topk=4, fix_bits=14, fix_value=v))


def test_sparse_window(q):
    Q = wl.sparse_int(22, 0.1, -20, 20, seed=5)
    o = oracle.solve(Q, topk=4096, cap=1)
    sel = o.topk_E <= o.min + 12
    assert not sel.all()
    cnt, codes, E, info = q.solve_window(Q, 12)
    assert info["acc"] == "i32z"
    assert cnt == int(sel.sum())
    assert np.array_equal(codes, o.topk[sel]) and np.array_equal(E, o.topk_E[sel])


def test_sparse_overflow_split(q, monkeypatch):
    """Nine free variables (no diagonal, no coupling) give 2^9 minimisers, more than a
    300-record buffer holds: the run splits along the top code bit (free, so each half holds
    256) and merges; the results stay exact."""
    Q = wl.sparse_int(24, 0.1, -50, 50, seed=9)
    Q[15:, :] = 0
    Q[:, 15:] = 0
    assert q.solve(Q).info["acc"] == "i32z"
    monkeypatch.setenv("QUBO_MAX_RECORDS", "300")
    r = q.solve(Q, states_cap=4096)
    assert r.info["passes"] > 1 and r.n_ties % 512 == 0
    check_int(r, oracle.solve(Q, cap=4096))


def test_diagonal_instance_uses_every_walked_row(q):
    """No couplings at all: every walked row is factored out; ties have the closed form."""
    Q = wl.diagonal(26, seed=4, zeros=5)
    r = q.solve(Q, states_cap=64)
    assert r.info["acc"] == "i32z" and r.n_ties == 1 << 5
    check_int(r, oracle.solve(Q, cap=64))


def test_sparse_disabled_falls_back(q, monkeypatch):
    Q = wl.sparse_int(26, 0.1, -500, 500, seed=11)
    o = oracle.solve(Q, topk=8)
    monkeypatch.setenv("QUBO_NO_I32Z", "1")
    r = q.solve(Q, topk=8)
    assert r.info["acc"] in ("i16p", "i32f", "i32")
    check_int(r, o)


def test_sparse_relabelled_instance(q):
    """Relabelling the variables (Sec. 2.4) changes the scan order the host picks; the minimum and
    tie count stay, and the codes map through the relabelling."""
    n = 28
    Q = wl.sparse_int(n, 0.08, -300, 300, seed=21)
    perm = np.random.default_rng(5).permutation(n)
    Qp = Q[np.ix_(perm, perm)]  # variable a of Qp is variable perm[a] of Q
    r, rp = q.solve(Q, topk=6), q.solve(Qp, topk=6)
    assert r.info["acc"] == rp.info["acc"] == "i32z"
    assert r.min == rp.min and r.n_ties == rp.n_ties

    def to_q(c):
        return sum(1 << int(perm[a]) for a in range(n) if (int(c) >> a) & 1)

    assert sorted(to_q(c) for c in rp.ties) == [int(c) for c in r.ties]
    check_int(rp, oracle.solve(Qp, topk=6))


def test_sparse_large_k_and_subcube_with_fixed_top_bits(q):
    Q = wl.sparse_int(36, 0.07, -50, 50, seed=36)
    r = q.solve(Q, topk=1024, fix_bits=6, fix_value=37, states_cap=4096)
    assert r.info["acc"] == "i32z"
    check_int(r, oracle.solve(Q, topk=1024, fix_bits=6, fix_value=37, cap=4096))


def test_sparse_problem_api_and_merge(q):
    """Device-resident problem, two halves of the cube, merged on the host."""
    Q = wl.sparse_int(30, 0.08, -200, 200, seed=30)
    p = q.Problem(Q, topk=8)
    parts = []
    for v in (0, 1):
        p.run(1, v)
        parts.append(p.fetch(states_cap=1024))
    p.close()
    assert parts[0].info["acc"] == "i32z"
    m = q.merge_all(parts, 1024, 8)
    check_int(m, oracle.solve(Q, topk=8, cap=1024))


def test_sparse_wide_subproblem(q):
    """A 70-variable sparse instance: one outer value's 28-variable sub-problem (solved alone,
    in the factored scan), against the oracle's reduction."""
    Q = wl.sparse_int(70, 0.05, -500, 500, seed=70)
    v = 123456789
    r = q.solve_wide(Q, 28, outer_begin=v, outer_count=1, topk=4)
    assert r.info["acc"] == "i32z" and r.info["states_scanned"] == 1 << 28
    R, c = oracle.reduce(Q, 28, v)
    o = oracle.solve(R, topk=4)
    assert r.min == o.min + c and r.n_ties == o.n_ties
    assert r.ties == [int(t) | (v << 28) for t in o.ties]
    assert r.topk == [int(t) | (v << 28) for t in o.topk]
    assert r.topk_E.tolist() == [int(e) + c for e in o.topk_E]


# --- sparse float instances: the factored scan in FP32 with FP64 rescoring ---------------------

FLOAT_RTOL = 1e-9


def check_float(r, o):
    assert abs(r.min - o.min) <= FLOAT_RTOL * max(1.0, abs(o.min)), (r.min, o.min)
    assert r.n_ties == o.n_ties
    assert np.array_equal(r.ties, o.ties)
    assert np.array_equal(r.topk, o.topk), (r.topk, o.topk)
    assert np.allclose(r.topk_E, o.topk_E, rtol=FLOAT_RTOL, atol=FLOAT_RTOL)


@pytest.mark.parametrize("n", [18, 24, 29])
@pytest.mark.parametrize("topk", [0, 8])
def test_sparse_float_parity(q, n, topk):
    Q = wl.sparse_float32(n, 0.1, seed=500 + n)
    r = q.solve(Q, topk=topk)
    assert r.info["acc"] == "f32z", r.info
    check_float(r, oracle.solve(Q, topk=topk))


def test_sparse_float_several_blocks_drift(q):
    """A walk longer than the factored rows: the columns change between blocks and the FP32
    drift is measured at the end of every unit."""
    Q = wl.sparse_float32(30, 0.25, seed=31)
    r = q.solve(Q, topk=6, walk_bits=10)
    assert r.info["acc"] == "f32z" and r.info["walk_bits"] == 10
    assert 0 < r.info["zero_rows"] < 10
    assert 2 * r.info["fp32_max_drift"] < 1e-3
    check_float(r, oracle.solve(Q, topk=6))


def test_sparse_float_window_and_subcube(q):
    Q = wl.sparse_float32(26, 0.1, seed=7)
    cnt, codes, E, info = q.solve_window(Q, 0.5)  # splits its cube (the window holds many states)
    o = oracle.solve(Q, topk=4096, cap=1)
    sel = o.topk_E <= o.min + 0.5
    assert cnt == int(sel.sum()) and np.array_equal(codes, o.topk[sel])
    assert np.allclose(E, o.topk_E[sel], rtol=FLOAT_RTOL, atol=FLOAT_RTOL)
    r = q.solve(Q, topk=4, fix_bits=2, fix_value=1)  # planned in whichever FP32 scan fits
    check_float(r, oracle.solve(Q, topk=4, fix_bits=2, fix_value=1))


def test_sparse_float_disabled_falls_back(q, monkeypatch):
    Q = wl.sparse_float32(24, 0.1, seed=8)
    o = oracle.solve(Q, topk=4)
    monkeypatch.setenv("QUBO_NO_I32Z", "1")
    r = q.solve(Q, topk=4)
    assert r.info["acc"] == "f32"
    check_float(r, o)
