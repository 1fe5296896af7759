"""qubo_solve_noalloc: the solve whose device scratch is a fixed array inside the library.

It serves callers that must not allocate device memory during a solve (a pool allocator owns
all of it, or the synchronisation a cudaMalloc may cost is not acceptable).  This file checks,
through the C ABI, that its results equal those of the allocating entry point, on calls made
back to back (the array is shared and keeps the previous call's contents).  Collected last so
that a failure here stops a first-failure run only after every other test has run.
"""
import numpy as np
import pytest

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
    assert np.array_equal(r.ties, ref.ties[:cap])


def test_noalloc_matches_allocating_entry_point_on_consecutive_calls(q):
    cap = 64
    a = wl.upper_int(31, -500, 500, seed=301)
    b = wl.diagonal(26, seed=302, zeros=5)        # 32 minimisers
    c = wl.upper_int(12, -9, 9, seed=303)          # small enough for direct evaluation
    refs = [q.solve(M, states_cap=cap) for M in (a, b, c)]
    for M, ref in zip((a, b, c, a), refs + refs[:1]):
        same(q.solve_noalloc(M, states_cap=cap), ref, cap)


def test_noalloc_rejects_sizes_beyond_its_limits(q):
    with pytest.raises(q.QuboError) as e:
        q.solve_noalloc(wl.upper_int(q.NOALLOC_MAX_N + 1, -5, 5, seed=1))
    assert e.value.status == q.QUBO_ERR_ARG
    with pytest.raises(q.QuboError) as e:
        q.solve_noalloc(wl.upper_int(20, -5, 5, seed=1), states_cap=q.NOALLOC_MAX_TIES + 1)
    assert e.value.status == q.QUBO_ERR_ARG
