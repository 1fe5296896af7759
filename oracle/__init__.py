"""CPU oracle for exhaustive dense-QUBO minimisation (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package.  It shares no code with the CUDA library it checks.

The C source (``oracle.c``) states what is computed and which passage of the paper each part
follows: the objective of Sec. 1, the reflected Gray order of Sec. 3.2, and the naive
O(n^2)-per-state and O(n)-per-state brute-force methods of Sec. 1.4.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

DIRECT = 0
GRAY = 1


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` with gcc and OpenMP (plain C, portable flags)."""
    stale = (not os.path.exists(_LIB_PATH)) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(
            ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"],
            check=True,
        )
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB_PATH)
    P = ctypes.c_void_p
    i32, u64, i64 = ctypes.c_int, ctypes.c_uint64, ctypes.c_int64
    lib.oracle_energy_i64.restype = i64
    lib.oracle_energy_i64.argtypes = [P, i32, u64]
    lib.oracle_energy_f64.restype = ctypes.c_double
    lib.oracle_energy_f64.argtypes = [P, i32, u64]
    lib.oracle_fold_i64.argtypes = [P, i32, P]
    lib.oracle_fold_f64.argtypes = [P, i32, P]
    lib.oracle_gray_code.restype = u64
    lib.oracle_gray_code.argtypes = [u64]
    lib.oracle_gray_walk_i64.argtypes = [P, i32, P]
    lib.oracle_solve_i64.restype = i32
    lib.oracle_solve_i64.argtypes = [P, i32, i32, i32, u64, i32, u64, i32, P, P, P, P, P, P, P]
    lib.oracle_solve_f64.restype = i32
    lib.oracle_solve_f64.argtypes = [P, i32, i32, i32, u64, i32, u64, i32, P, P, P, P, P, P, P, P]
    lib.oracle_max_threads.restype = i32
    lib.oracle_reduce_i64.argtypes = [P, i32, i32, P, P, P]
    lib.oracle_reduce_f64.argtypes = [P, i32, i32, P, P, P]
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def is_float(Q) -> bool:
    return np.asarray(Q).dtype.kind == "f"


def _as_matrix(Q):
    Q = np.asarray(Q)
    if Q.ndim != 2 or Q.shape[0] != Q.shape[1]:
        raise ValueError("Q must be a square matrix")
    if Q.dtype.kind == "f":
        return np.ascontiguousarray(Q, dtype=np.float64)  # FP32 widens exactly
    return np.ascontiguousarray(Q, dtype=np.int64)


def fold(Q) -> np.ndarray:
    """Upper-triangular U with U_ii = Q_ii, U_ij = Q_ij + Q_ji (i < j)."""
    Q = _as_matrix(Q)
    n = Q.shape[0]
    U = np.zeros_like(Q)
    lib = _load()
    (lib.oracle_fold_f64 if Q.dtype == np.float64 else lib.oracle_fold_i64)(_ptr(Q), n, _ptr(U))
    return U


def energy(Q, x: int):
    """Direct energy of state code x (bit i = variable i), canonical summation order."""
    U = fold(Q)
    n = U.shape[0]
    lib = _load()
    if U.dtype == np.float64:
        return float(lib.oracle_energy_f64(_ptr(U), n, int(x)))
    return int(lib.oracle_energy_i64(_ptr(U), n, int(x)))


def gray_code(i: int) -> int:
    return int(_load().oracle_gray_code(int(i)))


def gray_walk(Q) -> np.ndarray:
    """Energies along the Gray walk of all 2^n states (integer Q, n <= 24)."""
    U = fold(Q)
    n = U.shape[0]
    if U.dtype != np.int64 or n > 24:
        raise ValueError("gray_walk takes an integer Q with n <= 24")
    out = np.zeros(1 << n, dtype=np.int64)
    _load().oracle_gray_walk_i64(_ptr(U), n, _ptr(out))
    return out


@dataclass
class OracleResult:
    min: object          # int for integer Q, float for float Q
    n_ties: int          # exact size of the tie set
    ties: np.ndarray     # smallest tie codes ascending (at most cap), uint64
    topk: np.ndarray     # K lowest codes by (E, code), uint64
    topk_E: np.ndarray   # their energies
    n_candidates: int = 0

    @property
    def truncated(self) -> bool:
        return self.n_ties > len(self.ties)


def solve(Q, method: int = GRAY, topk: int = 0, cap: int = 1 << 16, fix_bits: int = 0,
          fix_value: int = 0, nthreads: int = 0) -> OracleResult:
    """Exact minimum, tie set and K lowest states of E over the (sub)cube."""
    Q = _as_matrix(Q)
    n = Q.shape[0]
    lib = _load()
    ties = np.zeros(max(cap, 1), dtype=np.uint64)
    tk = np.zeros(max(topk, 1), dtype=np.uint64)
    nties = np.zeros(1, dtype=np.uint64)
    nw = np.zeros(1, dtype=np.uint64)
    nk = np.zeros(1, dtype=np.int32)
    if Q.dtype == np.float64:
        mn = np.zeros(1, dtype=np.float64)
        tkE = np.zeros(max(topk, 1), dtype=np.float64)
        ncand = np.zeros(1, dtype=np.uint64)
        rc = lib.oracle_solve_f64(_ptr(Q), n, method, fix_bits, fix_value, topk, cap, nthreads,
                                  _ptr(mn), _ptr(nties), _ptr(ties), _ptr(nw), _ptr(tk), _ptr(tkE),
                                  _ptr(nk), _ptr(ncand))
        mval, nc = float(mn[0]), int(ncand[0])
    else:
        mn = np.zeros(1, dtype=np.int64)
        tkE = np.zeros(max(topk, 1), dtype=np.int64)
        rc = lib.oracle_solve_i64(_ptr(Q), n, method, fix_bits, fix_value, topk, cap, nthreads,
                                  _ptr(mn), _ptr(nties), _ptr(ties), _ptr(nw), _ptr(tk), _ptr(tkE),
                                  _ptr(nk))
        mval, nc = int(mn[0]), 0
    if rc != 0:
        raise RuntimeError(f"oracle solve failed with status {rc}")
    k = int(nk[0])
    return OracleResult(mval, int(nties[0]), ties[: int(nw[0])].copy(), tk[:k].copy(), tkE[:k].copy(), nc)


def reduce(Q, m: int, fixed):
    """Sub-problem over variables 0..m-1 with variables m..n-1 fixed (``fixed``: an int whose
    bit f is variable m + f, or a sequence of 0/1).  Returns (R, c): R is an m x m
    upper-triangular matrix and E_Q(x) = E_R(x_0..x_{m-1}) + c for every x with that fixed part
    (oracle.c states the split)."""
    U = fold(Q)
    n = U.shape[0]
    if isinstance(fixed, (int, np.integer)):
        xf = np.array([(int(fixed) >> f) & 1 for f in range(n - m)], dtype=np.uint8)
    else:
        xf = np.ascontiguousarray(fixed, dtype=np.uint8)
    if xf.shape != (n - m,):
        raise ValueError("fixed must give the n - m fixed variables")
    R = np.zeros((m, m), dtype=U.dtype)
    lib = _load()
    if U.dtype == np.float64:
        c = ctypes.c_double()
        lib.oracle_reduce_f64(_ptr(U), n, m, _ptr(xf), _ptr(R), ctypes.byref(c))
        return R, float(c.value)
    c = ctypes.c_int64()
    lib.oracle_reduce_i64(_ptr(U), n, m, _ptr(xf), _ptr(R), ctypes.byref(c))
    return R, int(c.value)


def max_threads() -> int:
    return int(_load().oracle_max_threads())
