"""Restatements, in numpy, of the host's admission checks for the packed 16-bit and FP32-lane
scans, written from their definitions (not from the library's code); shared by the CPU plan tests
and the GPU parity tests."""
import numpy as np

import oracle


def column_range(Q, B, L, RC):
    """Range of the column values a packed scan with B suffix bits, L walked bits and RC
    register rows can hold: for every suffix pattern j, E_s(j) plus each outside coupling sum
    c_i(j) and each register-row/fixed coupling at its sign's extreme."""
    U = oracle.fold(np.asarray(Q).astype(np.int64)).astype(np.int64)
    n = U.shape[0]
    W = np.triu(U, 1) + np.triu(U, 1).T
    j = np.arange(1 << B, dtype=np.int64)
    J = (j[:, None] >> np.arange(B)) & 1
    Es = J @ np.diag(U)[:B] + ((J @ W[:B, :B]) * J).sum(1) // 2
    c = J @ W[:B, B:]
    hi = Es + np.clip(c, 0, None).sum(1)
    lo = Es + np.clip(c, None, 0).sum(1)
    wr = W[B:B + RC, B + L:]
    return int(lo.min() + np.clip(wr, None, 0).sum()), int(hi.max() + np.clip(wr, 0, None).sum())


def plan_bound(Q, suffix_bits, walk_bits):
    """S_nf + 2 S_ww of a plan: the crude bound on the magnitudes the FP32-lane scan forms."""
    U = np.abs(oracle.fold(Q)).astype(np.float64)
    nf = suffix_bits + walk_bits
    return U[:nf, :].sum() + 2 * U[suffix_bits:nf, suffix_bits:nf].sum()


def fp32_lanes_fit(Q, B, L, RC):
    """Whether every value an FP32-lane scan with B suffix bits, L walked bits and RC register
    rows holds stays below 2^24: the crude bound, else the exact column range (every outside
    coupling sum at its sign's extreme, per suffix pattern), the walked energies E_L by brute
    force, and each table row's sum of |U|."""
    if plan_bound(Q, B, L) + 2 < 2**24:
        return True
    U = oracle.fold(np.asarray(Q).astype(np.int64)).astype(np.int64)
    nf = B + L
    W = np.triu(U, 1) + np.triu(U, 1).T
    for r in range(B, nf):
        row = np.abs(W[r, :B]).sum() + (np.abs(W[r, nf:]).sum() if r < B + RC else 0)
        if row >= 2**24:
            return False
    j = np.arange(1 << B, dtype=np.int64)
    J = (j[:, None] >> np.arange(B)) & 1
    Es = J @ np.diag(U)[:B] + ((J @ W[:B, :B]) * J).sum(1) // 2
    c = J @ W[:B, B:]
    wr = W[B:B + RC, nf:]
    hi = int((Es + np.clip(c, 0, None).sum(1)).max() + np.clip(wr, 0, None).sum())
    lo = int((Es + np.clip(c, None, 0).sum(1)).min() + np.clip(wr, None, 0).sum())
    g = np.arange(1 << L, dtype=np.int64)
    G = (g[:, None] >> np.arange(L)) & 1
    Uw = U[B:nf, B:nf]
    EL = G @ np.diag(Uw) + ((G @ np.triu(Uw, 1)) * G).sum(1)
    el = int(np.abs(EL).max())
    C = max(-lo, hi, 0) + el + 1
    return C + el + 1 < 2**24


def fp32_bound(Q, B, L, RC, anchor_bits, margin=1e-3):
    """Worst-case rounding error of the dense FP32 scan's decision value for a plan with B suffix
    bits, L walked bits (suffix = variables 0..B-1, walked = B..B+L-1, fixed = the rest), RC
    register rows, re-anchored every 2^anchor_bits walk steps: every FP32 operation rounds to
    nearest (error <= u |result|, u = 2^-24), the tables are FP64 sums rounded once, and each
    quantity's magnitude is bounded from |U| over the variables it involves (column values Cc,
    walked energies CL, prefix energy CP, thresholds CT); the per-unit fields and c(x_f) are
    FP64 sums rounded to FP32 once, the column fields lin(j) FP32 sums of them."""
    U = oracle.fold(np.asarray(Q, dtype=np.float64))
    n = U.shape[0]
    nf = B + L
    k = n - nf
    u = 2.0 ** -24
    A = np.abs(U)
    S = A + np.triu(A, 1).T  # |W|, symmetric, diagonal |U_ii|
    beta = A.sum()
    bF = np.triu(A)[nf:, nf:].sum()
    rF = np.array([S[v, nf:].sum() for v in range(nf)])
    rS = np.array([S[v, :B].sum() - (S[v, v] if v < B else 0.0) for v in range(nf)])
    CabsF = rF[:B].sum()
    CP = bF + rF[B + RC:nf].sum()
    W = np.triu(U, 1) + np.triu(U, 1).T
    j = np.arange(1 << B, dtype=np.int64)
    J = ((j[:, None] >> np.arange(B)) & 1).astype(np.float64)
    Es = J @ np.diag(U)[:B] + ((J @ W[:B, :B]) * J).sum(1) / 2
    c = J @ W[:B, B:]
    Cc = (np.abs(Es) + np.abs(c).sum(1)).max() + rF[B:B + RC].sum()
    g = np.arange(1 << L, dtype=np.int64)
    G = ((g[:, None] >> np.arange(L)) & 1).astype(np.float64)
    Uw = U[B:nf, B:nf]
    CL = np.abs(G @ np.diag(Uw) + ((G @ np.triu(Uw, 1)) * G).sum(1)).max() * (1 + 2.0 ** -30)
    CT = beta * (1 + 2.0 ** -20) + margin
    e64 = n * n * 2.0 ** -52 * beta
    u64 = 2.0 ** -52
    Ecol0 = 2 * u * Cc + e64 + (B + 3) * u * CabsF + k * u64 * CabsF + (L - RC) * u * Cc
    for r in range(L):
        if r < RC:
            Ecol0 += 2 * u * (rS[B + r] + rF[B + r]) + (u + k * u64) * rF[B + r] + e64
        else:
            Ecol0 += u * rS[B + r] + e64
    a = min(max(anchor_bits, RC + 1), L)
    Ecol = Ecol0 + np.expm1(2.0 ** a * np.log1p(u)) * (Cc + Ecol0)
    EP0 = (u + (k + 8) * u64) * bF + (L - RC) * u * CP + (u + k * u64) * rF[B + RC:nf].sum()
    tP = 2.0 ** max(0, a - RC - 1) + 1
    EP = EP0 + np.expm1(tP * np.log1p(u)) * (CP + EP0)
    return (Ecol + (RC + 1) * u * (Cc + Ecol) + EP + (u * CL + e64) + u * (Cc + CL) + u * CT + u * (CT + CP)
            + u * (CT + CP + CL))
