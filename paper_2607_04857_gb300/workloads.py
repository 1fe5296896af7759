"""Seeded synthetic QUBO instances.

This module only draws input matrices; it evaluates no energies.  Both the CUDA path and the
CPU oracle are fed from it, so it is the one piece of code the two sides share.

The paper benchmarks on uniformly random dense matrices and notes that an exhaustive scan's
execution trace does not depend on the instance (Sec. 5.3), so random matrices of the stated
shapes are the whole workload; no public dataset is involved.

Conventions: numpy ``Generator(PCG64(seed))``; an upper-triangular matrix is filled row-major
over i <= j from one draw of n(n+1)/2 values; integer uniforms include both end points.
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def upper_int(n: int, lo: int, hi: int, seed: int, dtype=np.int32) -> np.ndarray:
    """Upper-triangular integer Q with entries i.i.d. uniform in [lo, hi]."""
    rng = _rng(seed)
    iu = np.triu_indices(n)
    vals = rng.integers(lo, hi, size=len(iu[0]), endpoint=True, dtype=np.int64)
    Q = np.zeros((n, n), dtype=dtype)
    Q[iu] = vals.astype(dtype)
    return Q


def sk_float32(n: int, seed: int) -> np.ndarray:
    """Symmetric FP32 Q, Sherrington-Kirkpatrick-like: Q_ij = Q_ji ~ N(0,1)/sqrt(n) off the
    diagonal, Q_ii ~ N(0,1).  Values are rounded to FP32 once and stored."""
    rng = _rng(seed)
    iu = np.triu_indices(n, k=1)
    off = (rng.standard_normal(len(iu[0])) / np.sqrt(n)).astype(np.float32)
    diag = rng.standard_normal(n).astype(np.float32)
    Q = np.zeros((n, n), dtype=np.float32)
    Q[iu] = off
    Q[(iu[1], iu[0])] = off
    Q[np.arange(n), np.arange(n)] = diag
    return Q


def maxcut_qubo(n: int, p: float, seed: int, dtype=np.int16) -> np.ndarray:
    """Max-Cut of a G(n, p) graph with edge weights +-1, as the upper-triangular QUBO whose
    energy is minus the cut weight: E(x) = sum_{(i,j) in E} w_ij (2 x_i x_j - x_i - x_j),
    i.e. U_ij = 2 w_ij for each edge and U_ii = -sum_j w_ij."""
    rng = _rng(seed)
    iu = np.triu_indices(n, k=1)
    edge = rng.random(len(iu[0])) < p
    w = np.where(rng.random(len(iu[0])) < 0.5, -1, 1) * edge
    Q = np.zeros((n, n), dtype=np.int64)
    Q[iu] = 2 * w
    deg = np.zeros(n, dtype=np.int64)
    np.add.at(deg, iu[0], w)
    np.add.at(deg, iu[1], w)
    Q[np.arange(n), np.arange(n)] = -deg
    return Q.astype(dtype)


def sparse_int(n: int, density: float, lo: int, hi: int, seed: int, dtype=np.int32) -> np.ndarray:
    """Upper-triangular integer Q: diagonal entries uniform in [lo, hi] (a drawn 0 becomes lo),
    each off-diagonal entry present with probability `density`, its value uniform in [lo, hi]
    (a drawn 0 becomes hi)."""
    rng = _rng(seed)
    iu = np.triu_indices(n, k=1)
    present = rng.random(len(iu[0])) < density
    vals = rng.integers(lo, hi, size=len(iu[0]), endpoint=True, dtype=np.int64)
    vals = np.where(vals == 0, hi, vals) * present
    Q = np.zeros((n, n), dtype=np.int64)
    Q[iu] = vals
    d = rng.integers(lo, hi, size=n, endpoint=True, dtype=np.int64)
    Q[np.arange(n), np.arange(n)] = np.where(d == 0, lo, d)
    return Q.astype(dtype)


def sparse_float32(n: int, density: float, seed: int) -> np.ndarray:
    """Symmetric FP32 Q: diagonal N(0,1), each off-diagonal pair present with probability
    `density` with value N(0,1)/sqrt(n * density) (a sparse SK-like spin glass); stored FP32."""
    rng = _rng(seed)
    iu = np.triu_indices(n, k=1)
    present = rng.random(len(iu[0])) < density
    off = (rng.standard_normal(len(iu[0])) / np.sqrt(max(1.0, n * density))).astype(np.float32) * present
    Q = np.zeros((n, n), dtype=np.float32)
    Q[iu] = off
    Q[(iu[1], iu[0])] = off
    Q[np.arange(n), np.arange(n)] = rng.standard_normal(n).astype(np.float32)
    return Q


def planted(n: int, seed: int, x_star: int | None = None, dtype=np.int32):
    """Diagonal Q = diag(w * (1 - 2 x*)) with w > 0, whose unique minimiser is x*.
    Returns (Q, x*)."""
    rng = _rng(seed)
    if x_star is None:
        x_star = int(rng.integers(0, 1 << min(n, 62))) & ((1 << n) - 1)
    w = rng.integers(1, 100, size=n, endpoint=True)
    bits = np.array([(x_star >> i) & 1 for i in range(n)], dtype=np.int64)
    Q = np.diag(w * (1 - 2 * bits)).astype(dtype)
    return Q, x_star


def decimal_pairs(n: int, seed: int, dtype=np.float64) -> np.ndarray:
    """Float Q made of n//2 uncoupled variable pairs {a, b} on shuffled positions, each with
    Q_aa = Q_bb = -v and Q_ab = v for v drawn from {0.1, 0.2, 0.3, 0.7}; an odd n leaves one
    variable with Q_ii = -v alone.  In exact arithmetic every pair has the three minimisers 01,
    10 and 11, so the real minimum is taken by 3^(n//2) states; in floating point their sums,
    formed in different orders, differ in the last bits (near-ties one rounding apart)."""
    rng = _rng(seed)
    perm = rng.permutation(n)
    vals = rng.choice(np.array([0.1, 0.2, 0.3, 0.7]), size=(n + 1) // 2)
    Q = np.zeros((n, n), dtype=dtype)
    for p in range(n // 2):
        a, b = sorted((int(perm[2 * p]), int(perm[2 * p + 1])))
        Q[a, a] = Q[b, b] = -vals[p]
        Q[a, b] = vals[p]
    if n % 2:
        Q[perm[-1], perm[-1]] = -vals[-1]
    return Q


def diagonal(n: int, seed: int, zeros: int, dtype=np.int32) -> np.ndarray:
    """Diagonal Q with `zeros` zero entries (at random positions) and the rest nonzero."""
    rng = _rng(seed)
    d = rng.integers(1, 50, size=n, endpoint=True) * np.where(rng.random(n) < 0.5, -1, 1)
    pos = rng.permutation(n)[:zeros]
    d[pos] = 0
    return np.diag(d).astype(dtype)


# ---- the five benchmark configurations --------------------------------------------------

CONFIGS = {
    1: dict(name="n24_int32", n=24, seed=1, outputs="min + tie set"),
    2: dict(name="n36_int32_top16", n=36, seed=2, outputs="min + tie set + top-16"),
    3: dict(name="n44_fp32_sk", n=44, seed=3, outputs="FP32 scan + FP64 rescore"),
    4: dict(name="batched_4096_n16_32", n=None, seed=4, outputs="min + tie set per instance"),
    5: dict(name="n50_int32_top16", n=50, seed=5, outputs="min + tie set + top-16"),
}


def config1() -> np.ndarray:
    """n=24, upper-triangular int32, entries uniform in [-100, 100]."""
    return upper_int(24, -100, 100, seed=1)


def config2() -> np.ndarray:
    """n=36, upper-triangular int32, entries uniform in [-1000, 1000]."""
    return upper_int(36, -1000, 1000, seed=2)


def config3() -> np.ndarray:
    """n=44 symmetric FP32, SK-like."""
    return sk_float32(44, seed=3)


def config5() -> np.ndarray:
    """n=50, upper-triangular int32, entries uniform in [-32768, 32767]."""
    return upper_int(50, -32768, 32767, seed=5)


def config4(count: int = 4096, seed: int = 4):
    """`count` instances with n uniform in {16..32}: even index -> int16 upper-triangular Q
    uniform in [-127, 127]; odd index -> Max-Cut QUBO of G(n, 0.5) with weights +-1.
    Returns a list of int16 matrices."""
    rng = _rng(seed)
    ns = rng.integers(16, 32, size=count, endpoint=True)
    sub = rng.integers(0, 2**31 - 1, size=count)
    out = []
    for i in range(count):
        n = int(ns[i])
        if i % 2 == 0:
            out.append(upper_int(n, -127, 127, seed=int(sub[i]), dtype=np.int16))
        else:
            out.append(maxcut_qubo(n, 0.5, seed=int(sub[i]), dtype=np.int16))
    return out
