"""Edge cases of the C ABI on the GPU: full-width codes, the largest K, stopping a running call
from another thread, and the time limit of a wide solve."""
import threading
import time

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


@pytest.mark.parametrize("v", [(1 << 40) - 1, 1 << 39, 12345])
def test_n64_subcubes_with_the_top_code_bit(q, v):
    """n = 64: codes use all 64 bits; sub-cubes of 2^24 states with the top bits fixed."""
    Q = wl.upper_int(64, -200, 200, seed=64)
    r = q.solve(Q, topk=8, fix_bits=40, fix_value=v)
    check_int(r, oracle.solve(Q, topk=8, fix_bits=40, fix_value=v))
    assert all(int(c) >> 24 == v for c in r.topk)


def test_largest_topk(q):
    Q = wl.upper_int(20, -50, 50, seed=20)
    r = q.solve(Q, topk=q.QUBO_MAX_TOPK)
    check_int(r, oracle.solve(Q, topk=q.QUBO_MAX_TOPK))


def test_abort_from_another_thread(q):
    """qubo_abort from a second thread stops a running whole-cube scan (about a minute of work)
    at its next work unit; the call returns QUBO_ERR_TIMEOUT and the context stays usable."""
    Q = wl.upper_int(50, -1000, 1000, seed=1)
    out = {}

    def run():
        try:
            q.solve(Q)
            out["status"] = 0
        except q.QuboError as e:
            out["status"] = e.status

    t0 = time.time()
    th = threading.Thread(target=run)
    th.start()
    time.sleep(0.5)
    q.abort()
    th.join(60)
    q.abort_clear()
    assert not th.is_alive()
    assert out.get("status") == q.QUBO_ERR_TIMEOUT and time.time() - t0 < 20
    Q2 = wl.upper_int(20, -10, 10, seed=2)
    check_int(q.solve(Q2), oracle.solve(Q2))


def test_wide_time_limit(q):
    """Four sub-problems of 2^42 states (about 1 s in all) under a 0.3 s limit."""
    Q = wl.upper_int(70, -100, 100, seed=3)
    with pytest.raises(q.QuboError) as e:
        q.solve_wide(Q, 42, outer_begin=0, outer_count=4, time_limit=0.3)
    assert e.value.status == q.QUBO_ERR_TIMEOUT
    Q2 = wl.upper_int(20, -10, 10, seed=4)
    check_int(q.solve(Q2), oracle.solve(Q2))


def test_allocation_failure_is_reported_and_recovers(q, monkeypatch):
    """An injected allocation failure (QUBO_FAIL_ALLOC=1) returns QUBO_ERR_NOMEM from every entry
    point that needs its workspace; once lifted, the next call succeeds."""
    Q = wl.upper_int(22, -20, 20, seed=6)
    monkeypatch.setenv("QUBO_FAIL_ALLOC", "1")
    for call in (lambda: q.solve(Q, topk=4), lambda: q.solve_batched([Q[:18, :18], Q[:20, :20]]),
                 lambda: q.solve_window(Q, 5)):
        with pytest.raises(q.QuboError) as e:
            call()
        assert e.value.status == q.QUBO_ERR_NOMEM
    monkeypatch.delenv("QUBO_FAIL_ALLOC")
    check_int(q.solve(Q, topk=4), oracle.solve(Q, topk=4))


def test_plain_c_client(q, tmp_path):
    """tests/c_abi_client.c, a C program linked to libqubo.so: a dense planted n = 34 instance
    (unique minimiser, closed-form minimum) and the all-zero n = 20 instance (truncated tie set,
    exact count) through qubo_solve."""
    import subprocess

    from test_abi_host import build_c_client

    exe = build_c_client(q, tmp_path)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "c_abi_client ok" in r.stdout
