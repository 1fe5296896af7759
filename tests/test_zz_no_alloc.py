"""qubo_solve_noalloc: the solve whose device scratch is a fixed array inside the library.

It serves callers that must not allocate device memory during a solve (a pool allocator owns
all of it, or the synchronisation a cudaMalloc may cost is not acceptable).  This file checks,
through the C ABI, its results against the CPU oracle and against the allocating entry point, on
calls made back to back (the array is shared and keeps the previous call's contents), up to its
largest admitted size.  Collected last so that a failure here stops a first-failure run only
after every other test has run.
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


def same(r, ref, cap):
    assert r.min == ref.min
    assert r.n_ties == ref.n_ties
    assert np.array_equal(np.asarray(r.ties, dtype=np.uint64), np.asarray(ref.ties, dtype=np.uint64)[:cap])


def test_noalloc_matches_oracle_on_consecutive_calls(q):
    cap = 64
    a = wl.upper_int(31, -500, 500, seed=301)
    b = wl.diagonal(26, seed=302, zeros=5)        # 32 minimisers
    c = wl.upper_int(12, -9, 9, seed=303)          # small enough for direct evaluation
    refs = [oracle.solve(M, method=oracle.GRAY, cap=cap) for M in (a, b, c)]
    assert refs[1].n_ties == 32
    for M, ref in zip((a, b, c, a, b), refs + refs[:2]):
        same(q.solve_noalloc(M, states_cap=cap), ref, cap)


@pytest.mark.parametrize("n", [37, 40])
def test_noalloc_at_its_largest_sizes(q, n):
    """n = 37..40 use the clamped 2^12-step walk and the largest header; the results equal the
    allocating entry point's, and the oracle's direct evaluator gives every returned tie the
    returned minimum."""
    cap = q.NOALLOC_MAX_TIES
    for seed in (401, 402):
        M = wl.upper_int(n, -1000, 1000, seed=seed + n)
        r = q.solve_noalloc(M, states_cap=cap)
        ref = q.solve(M, states_cap=cap)
        same(r, ref, cap)
        assert all(oracle.energy(M, int(x)) == r.min for x in r.ties)
    # many minimisers: the diagonal closed form (2^zeros ties), truncated to states_cap
    D = wl.diagonal(n, seed=n, zeros=13)
    d = np.diag(D).astype(np.int64)
    r = q.solve_noalloc(D, states_cap=cap)
    assert r.min == int(np.minimum(d, 0).sum()) and r.n_ties == 1 << 13
    assert r.status == q.QUBO_TRUNCATED and len(r.ties) == cap
    neg = sum(1 << i for i in range(n) if d[i] < 0)
    zb = [i for i in range(n) if d[i] == 0]
    expect = sorted(neg | sum(1 << zb[b] for b in range(13) if (m >> b) & 1) for m in range(1 << 13))[:cap]
    assert np.array_equal(r.ties, np.array(expect, dtype=np.uint64))


def test_noalloc_honours_abort_between_kernels(q):
    M = wl.upper_int(20, -50, 50, seed=7)
    q.abort()
    try:
        with pytest.raises(q.QuboError) as e:
            q.solve_noalloc(M)
        assert e.value.status == q.QUBO_ERR_TIMEOUT
    finally:
        q.abort_clear()
    same(q.solve_noalloc(M), oracle.solve(M, method=oracle.GRAY, cap=64), 64)


def test_noalloc_rejects_sizes_beyond_its_limits(q):
    with pytest.raises(q.QuboError) as e:
        q.solve_noalloc(wl.upper_int(q.NOALLOC_MAX_N + 1, -5, 5, seed=1))
    assert e.value.status == q.QUBO_ERR_ARG
    with pytest.raises(q.QuboError) as e:
        q.solve_noalloc(wl.upper_int(20, -5, 5, seed=1), states_cap=q.NOALLOC_MAX_TIES + 1)
    assert e.value.status == q.QUBO_ERR_ARG
