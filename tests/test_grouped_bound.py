"""The lower bound behind the grouped step form, restated in numpy and checked by brute force (no
GPU).  A unit's columns are walked in reflected Gray order; at each group's first state the
thread's exact column minimum m is taken, and over the group's next 15 steps (register rows 0-3)
the minimum must never fall below m + D, where D is the smallest running sum of each step's
smallest column move.  E_L's group minimum completes the test.  A wrong sign pattern, a dropped
coupling to the fixed bits or a running sum taken over the wrong steps fails these checks."""
import numpy as np
import pytest

from paper_2607_04857_gb300 import workloads as wl


def columns_over_walk(U, B, L, fixed):
    """Column values col[i, j] (suffix pattern j, walk step i) and E_L(i) of one unit: the state's
    energy is col + E_L + const, col holding every term with a suffix variable."""
    n = U.shape[0]
    S = U + U.T - np.diag(np.diag(U))
    steps = 1 << L
    col = np.zeros((steps, 1 << B), dtype=np.int64)
    el = np.zeros(steps, dtype=np.int64)
    for i in range(steps):
        g = i ^ (i >> 1)
        x = np.zeros(n, dtype=np.int64)
        for r in range(L):
            x[B + r] = (g >> r) & 1
        x[B + L:] = fixed
        base = x @ U @ x
        for j in range(1 << B):
            y = x.copy()
            y[:B] = [(j >> b) & 1 for b in range(B)]
            col[i, j] = y @ U @ y - base
        walked = np.zeros(n, dtype=np.int64)
        walked[B:B + L] = x[B:B + L]
        el[i] = walked @ U @ walked
    return col, el, S


def group_bound(M, w, par):
    """D for one thread's columns: register rows r = 0..3 move column j by +-(M[r, j] + w[r])."""
    lo = (M + w[:, None]).min(axis=1)
    hi = (M + w[:, None]).max(axis=1)
    cum, best = 0, 0
    for t in range(1, 16):
        kk = (t & -t).bit_length() - 1
        neg = bool(par) if kk == 3 else bool((t >> (kk + 1)) & 1)
        cum += -hi[kk] if neg else lo[kk]
        best = min(best, cum)
    return best


@pytest.mark.parametrize("seed", range(4))
def test_group_bound_holds_by_brute_force(seed):
    n, B, L = 12, 3, 6  # 8 columns, 64 walk steps = 4 groups of 16, 3 fixed bits
    U = np.triu(wl.upper_int(n, -50, 50, seed=seed).astype(np.int64))
    rng = np.random.default_rng(seed)
    fixed = rng.integers(0, 2, n - B - L)
    col, el, S = columns_over_walk(U, B, L, fixed)
    # register row r: M[r, j] = sum of U over the suffix bits set in j, w[r] = coupling to the set
    # fixed bits (the kernel folds it into the row)
    M = np.array([[sum(S[b, B + r] for b in range(B) if (j >> b) & 1) for j in range(1 << B)] for r in range(4)])
    w = np.array([S[B + r, B + L:] @ fixed for r in range(4)])
    # the kernel's columns carry the fixed-bit couplings of the set register rows (the rest of the
    # prefix energy, constant within a group, sits in the threshold)
    steps = np.arange(1 << L)
    gray = steps ^ (steps >> 1)
    col = col + sum(((gray >> r) & 1) * w[r] for r in range(4))[:, None]
    # the row moves every column exactly as the walk does
    for i in range(1, 1 << L):
        kk = (i & -i).bit_length() - 1
        if kk < 4:
            sign = -1 if (i >> (kk + 1)) & 1 else 1
            assert np.array_equal(col[i] - col[i - 1], sign * (M[kk] + w[kk]))
    for g in range(col.shape[0] // 16):
        m = col[16 * g].min()
        D = group_bound(M, w, g & 1)
        assert m + D <= col[16 * g:16 * g + 16].min()
        # the test: no state of the group is at or below u when m + D > u - min E_L
        emin = (col[16 * g:16 * g + 16] + el[16 * g:16 * g + 16, None]).min()
        assert m + D + el[16 * g:16 * g + 16].min() <= emin


def test_group_bound_is_tight_for_one_column():
    """With a single column every step's smallest move is the move itself, so m + D is the
    column's exact minimum over the group."""
    M = np.array([[5], [-7], [3], [-2]])
    w = np.array([1, 2, -4, 0])
    walk = [0]
    for t in range(1, 16):
        kk = (t & -t).bit_length() - 1
        neg = (t >> (kk + 1)) & 1  # group 0: the sign of row 3 follows bit 4 of the position (0)
        walk.append(walk[-1] + (-1 if neg else 1) * (M[kk, 0] + w[kk]))
    assert group_bound(M, w, 0) == min(walk)
