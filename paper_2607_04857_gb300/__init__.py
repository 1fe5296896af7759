"""GB300 exhaustive dense-QUBO solver: Python binding of libqubo.so (include/qubo.h).

Argument marshalling only: every step of the scan runs in the CUDA library.  The library must be
built first (``paper_2607_04857_gb300.build.build()``); importing the functions below raises if it
is missing, there is no fallback.

Conventions (as in qubo.h): a state code holds variable i in bit i; Q is any n x n matrix and
every entry counts, E(x) = sum_ij Q_ij x_i x_j.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libqubo.so")

QUBO_I16, QUBO_I32, QUBO_F32, QUBO_F64 = 1, 2, 3, 4
ACC_NAMES = {1: "i32", 2: "i64", 3: "f32", 4: "f64", 5: "i32f", 6: "i16p", 7: "i32z", 8: "f32z"}
QUBO_OK, QUBO_TRUNCATED = 0, 1
QUBO_ERR_ARG, QUBO_ERR_OVERFLOW, QUBO_ERR_CUDA = -1, -2, -3
QUBO_ERR_NOMEM, QUBO_ERR_TIMEOUT, QUBO_ERR_INTERNAL = -4, -5, -6
QUBO_FLAG_PLAIN = 0x1
QUBO_FLAG_INT32 = 0x2
QUBO_FLAG_RIGOROUS = 0x4
MAX_TOPK = 1024

# every entry point declared in include/qubo.h
EXPORTS = (
    "qubo_solve", "qubo_solve_ex", "qubo_solve_batched", "qubo_problem_create", "qubo_problem_run",
    "qubo_problem_fetch", "qubo_problem_destroy", "qubo_merge", "qubo_strerror", "qubo_abort",
    "qubo_abort_clear", "qubo_device_sm_count", "qubo_version", "qubo_solve_noalloc",
    "qubo_batch_create", "qubo_batch_run", "qubo_batch_fetch", "qubo_batch_destroy",
    "qubo_autotune", "qubo_autotune_batched", "qubo_autotune_clear", "qubo_solve_window", "qubo_solve_wide",
    "qubo_merge_wide", "qubo_autotune_save", "qubo_autotune_load", "qubo_plan_query", "qubo_autotune_batched_ex",
)
WIDE_MAX_N = 128
QUBO_MAX_TOPK = 1024
NOALLOC_MAX_N = 40
NOALLOC_MAX_TIES = 4096


class QuboError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {strerror(status)} (status {status})")


class Options(ctypes.Structure):
    _fields_ = [
        ("split_k", ctypes.c_int32), ("topk", ctypes.c_int32), ("fix_bits", ctypes.c_int32),
        ("walk_bits", ctypes.c_int32), ("fix_value", ctypes.c_uint64), ("flags", ctypes.c_uint32),
        ("reserved", ctypes.c_uint32), ("margin", ctypes.c_double), ("time_limit_s", ctypes.c_double),
    ]


class ResultInfo(ctypes.Structure):
    _fields_ = [
        ("min_i", ctypes.c_int64), ("min_f", ctypes.c_double), ("n_ties", ctypes.c_uint64),
        ("n_written", ctypes.c_uint64), ("truncated", ctypes.c_int32), ("acc", ctypes.c_int32),
        ("n_topk", ctypes.c_int32), ("anchor_bits", ctypes.c_int32), ("fp32_max_abs_err", ctypes.c_double),
        ("fp32_max_drift", ctypes.c_double), ("n_near_ties", ctypes.c_uint64),
        ("states_scanned", ctypes.c_uint64), ("candidates", ctypes.c_uint64), ("seconds", ctypes.c_double),
        ("seconds_gpu", ctypes.c_double), ("seconds_scan", ctypes.c_double), ("states_per_s", ctypes.c_double),
        ("n", ctypes.c_int32),
        ("split_k", ctypes.c_int32), ("walk_bits", ctypes.c_int32), ("suffix_bits", ctypes.c_int32),
        ("cols_per_thread", ctypes.c_int32), ("threads", ctypes.c_int32), ("blocks", ctypes.c_int32),
        ("passes", ctypes.c_int32), ("kernel_launches", ctypes.c_int32), ("zero_rows", ctypes.c_int32),
        ("h2d_bytes", ctypes.c_uint64), ("d2h_bytes", ctypes.c_uint64),
        ("fp32_err_bound", ctypes.c_double), ("fp32_rigorous_anchor_bits", ctypes.c_int32),
        ("reg_rows", ctypes.c_int32), ("variant", ctypes.c_int32), ("grouped", ctypes.c_int32),
    ]

    def as_dict(self) -> dict:
        d = {name: getattr(self, name) for name, _ in self._fields_ if not name.startswith("reserved")}
        d["acc"] = ACC_NAMES.get(d["acc"], d["acc"])
        return d


class Plan(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int32), ("walk_bits", ctypes.c_int32), ("states_per_s", ctypes.c_double),
                ("trials", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class Partial(ctypes.Structure):
    _fields_ = [
        ("is_float", ctypes.c_int32), ("n_topk", ctypes.c_int32), ("min_i", ctypes.c_int64),
        ("min_f", ctypes.c_double), ("n_ties", ctypes.c_uint64), ("n_written", ctypes.c_uint64),
        ("states_scanned", ctypes.c_uint64), ("ties", ctypes.c_void_p), ("topk", ctypes.c_void_p),
        ("topk_E", ctypes.c_void_p),
    ]


class PartialWide(Partial):
    """qubo_partial_wide: the same fields, with two words per code in ties and topk."""


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libqubo.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_2607_04857_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P, I, U64, SZ = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_size_t
    lib.qubo_solve.argtypes = [P, I, I, I, I, P, P, SZ, P, P, P, P]
    lib.qubo_solve_ex.argtypes = [P, I, I, P, P, P, SZ, P, P, P, P]
    lib.qubo_solve_batched.argtypes = [P, P, P, I, I, I, P, P, SZ, P, P, P, P]
    lib.qubo_problem_create.argtypes = [P, I, I, P, P]
    lib.qubo_problem_run.argtypes = [P, I, U64, P]
    lib.qubo_problem_fetch.argtypes = [P, P, P, SZ, P, P, P]
    lib.qubo_problem_destroy.argtypes = [P]
    lib.qubo_problem_destroy.restype = None
    lib.qubo_merge.argtypes = [P, P, SZ, I, P]
    lib.qubo_solve_noalloc.argtypes = [P, I, I, P, P, SZ, P, P]
    lib.qubo_batch_create.argtypes = [P, P, P, I, I, I, SZ, P]
    lib.qubo_batch_run.argtypes = [P, P]
    lib.qubo_batch_fetch.argtypes = [P, P, P, P, P, P]
    lib.qubo_batch_destroy.argtypes = [P]
    lib.qubo_batch_destroy.restype = None
    lib.qubo_autotune.argtypes = [P, I, I, I, P]
    lib.qubo_solve_window.argtypes = [P, I, I, ctypes.c_double, P, P, P, SZ, P, P, P]
    lib.qubo_autotune_batched.argtypes = [P, P, P, I, I, P]
    lib.qubo_autotune_batched_ex.argtypes = [P, P, P, I, I, P, P]
    lib.qubo_solve_wide.argtypes = [P, I, I, I, U64, U64, P, P, P, SZ, P, P, P, P, P]
    lib.qubo_merge_wide.argtypes = [P, P, SZ, I, P]
    lib.qubo_autotune_save.argtypes = [ctypes.c_char_p]
    lib.qubo_autotune_load.argtypes = [ctypes.c_char_p]
    lib.qubo_plan_query.argtypes = [P, I, I, P, P]
    lib.qubo_autotune_clear.restype = None
    lib.qubo_strerror.argtypes = [I]
    lib.qubo_strerror.restype = ctypes.c_char_p
    lib.qubo_version.restype = ctypes.c_char_p
    lib.qubo_abort.restype = None
    lib.qubo_abort_clear.restype = None
    for name in ("qubo_solve", "qubo_solve_ex", "qubo_solve_batched", "qubo_problem_create", "qubo_problem_run",
                 "qubo_problem_fetch", "qubo_merge", "qubo_device_sm_count", "qubo_solve_noalloc",
                 "qubo_batch_create", "qubo_batch_run", "qubo_batch_fetch", "qubo_autotune",
                 "qubo_autotune_batched", "qubo_autotune_batched_ex", "qubo_solve_window", "qubo_solve_wide", "qubo_merge_wide",
                 "qubo_autotune_save", "qubo_autotune_load"):
        getattr(lib, name).restype = I
    _lib = lib
    return lib


def strerror(status: int) -> str:
    return load_library().qubo_strerror(int(status)).decode()


def version() -> str:
    return load_library().qubo_version().decode()


def device_sm_count() -> int:
    r = load_library().qubo_device_sm_count()
    if r < 0:
        raise QuboError(r, "qubo_device_sm_count")
    return r


def abort() -> None:
    load_library().qubo_abort()


def abort_clear() -> None:
    load_library().qubo_abort_clear()


def _stream_ptr(stream):
    """cudaStream_t as an integer: an int, an object with .cuda_stream (torch), or the current
    torch stream when torch with CUDA is available; else the default stream."""
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return int(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return int(stream.cuda_stream)
    return int(stream)


def as_qubo_matrix(Q):
    """numpy matrix and its qubo_dtype (int16/int32/float32/float64; int64 narrowed if exact)."""
    if hasattr(Q, "detach"):  # torch tensor on the host
        Q = Q.detach().cpu().numpy()
    Q = np.asarray(Q)
    if Q.ndim != 2 or Q.shape[0] != Q.shape[1]:
        raise ValueError("Q must be a square matrix")
    if Q.dtype == np.int16:
        return np.ascontiguousarray(Q), QUBO_I16
    if Q.dtype.kind in "iub":
        Q32 = Q.astype(np.int32)
        if not np.array_equal(Q32, Q):
            raise ValueError("integer Q must fit in int32")
        return np.ascontiguousarray(Q32), QUBO_I32
    if Q.dtype == np.float32:
        return np.ascontiguousarray(Q), QUBO_F32
    if Q.dtype.kind == "f":
        return np.ascontiguousarray(Q, dtype=np.float64), QUBO_F64
    raise ValueError(f"unsupported dtype {Q.dtype}")


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a.size else None


@dataclass
class Result:
    min: object                      # int (integer Q) or float (float Q)
    n_ties: int                      # exact number of minimisers
    ties: np.ndarray                 # smallest tie codes ascending (<= states_cap), uint64
    topk: np.ndarray                 # K lowest codes by (E, code)
    topk_E: np.ndarray
    status: int = 0
    info: dict = field(default_factory=dict)

    @property
    def truncated(self) -> bool:
        return self.n_ties > len(self.ties)


def _flags(plain: bool, int32: bool, rigorous: bool = False) -> int:
    return (QUBO_FLAG_PLAIN if plain else 0) | (QUBO_FLAG_INT32 if int32 else 0) | \
        (QUBO_FLAG_RIGOROUS if rigorous else 0)


def _check(st: int, where: str) -> int:
    if st < 0:
        raise QuboError(st, where)
    return st


def solve(Q, topk: int = 0, states_cap: int = 1 << 16, split_k: int = 0, walk_bits: int = 0, fix_bits: int = 0,
          fix_value: int = 0, plain: bool = False, margin: float = 0.0, time_limit: float = 0.0,
          stream=None, int32: bool = False, rigorous: bool = False) -> Result:
    """Exact minimum, tie set and K lowest states (qubo_solve_ex).  plain: the wide accumulator
    (QUBO_FLAG_PLAIN); int32: integer Q in the int32 kernel only (QUBO_FLAG_INT32); rigorous:
    float Q re-anchored where the rounding bound proves the candidates (QUBO_FLAG_RIGOROUS)."""
    lib = load_library()
    Qm, dt = as_qubo_matrix(Q)
    n = Qm.shape[0]
    isf = dt in (QUBO_F32, QUBO_F64)
    edt = np.float64 if isf else np.int64
    o = Options(split_k=split_k, topk=topk, fix_bits=fix_bits, walk_bits=walk_bits, fix_value=fix_value,
                flags=_flags(plain, int32, rigorous), margin=margin, time_limit_s=time_limit)
    mn = np.zeros(1, dtype=edt)
    ties = np.zeros(max(states_cap, 0), dtype=np.uint64)
    tk = np.zeros(max(topk, 0), dtype=np.uint64)
    tkE = np.zeros(max(topk, 0), dtype=edt)
    info = ResultInfo()
    st = lib.qubo_solve_ex(_ptr(Qm), n, dt, ctypes.byref(o), _ptr(mn), _ptr(ties), states_cap, _ptr(tk), _ptr(tkE),
                           ctypes.byref(info), _stream_ptr(stream))
    _check(st, "qubo_solve_ex")
    k = info.n_topk
    return Result(float(mn[0]) if isf else int(mn[0]), int(info.n_ties), ties[: info.n_written].copy(), tk[:k].copy(),
                  tkE[:k].copy(), st, info.as_dict())


class PackedBatch:
    """Instances in qubo_solve_batched's input layout (one contiguous row-major array of all
    matrices, their sizes and element offsets), built once by pack_batch and accepted wherever a
    list of matrices is, so repeated solves of the same batch skip the repacking."""

    def __init__(self, packed, ns, offs, dt):
        self.packed, self.ns, self.offs, self.dt = packed, ns, offs, dt

    def __len__(self):
        return len(self.ns)


def pack_batch(Qs) -> PackedBatch:
    return PackedBatch(*_pack(Qs))


def _pack(Qs):
    if isinstance(Qs, PackedBatch):
        return Qs.packed, Qs.ns, Qs.offs, Qs.dt
    mats = [as_qubo_matrix(Q) for Q in Qs]
    dts = {d for _, d in mats}
    if len(dts) != 1:
        raise ValueError("all instances of a batch must share one dtype")
    dt = dts.pop()
    ns = np.array([m.shape[0] for m, _ in mats], dtype=np.int32)
    offs = np.zeros(len(mats), dtype=np.uint64)
    offs[1:] = np.cumsum(ns[:-1].astype(np.uint64) ** 2)
    packed = np.concatenate([m.ravel() for m, _ in mats])
    return packed, ns, offs, dt


def _batch_outputs(count, dt, topk, states_cap):
    edt = np.float64 if dt in (QUBO_F32, QUBO_F64) else np.int64
    return (np.zeros(count, dtype=edt), np.zeros(count * states_cap, dtype=np.uint64),
            np.zeros(count * topk, dtype=np.uint64), np.zeros(count * topk, dtype=edt), (ResultInfo * count)())


def _batch_results(count, dt, topk, states_cap, mn, ties, tk, tkE, infos):
    return BatchResults(count, dt, topk, states_cap, mn, ties, tk, tkE, infos)


def autotune(Q, fix_bits: int) -> dict:
    """Time the compiled variants and walk lengths on sub-cubes of Q (top fix_bits fixed) and
    install the fastest plan for this size (qubo_autotune)."""
    lib = load_library()
    Qm, dt = as_qubo_matrix(Q)
    p = Plan()
    _check(lib.qubo_autotune(_ptr(Qm), Qm.shape[0], dt, fix_bits, ctypes.byref(p)), "qubo_autotune")
    return {"variant": p.variant, "walk_bits": p.walk_bits, "states_per_s": p.states_per_s, "trials": p.trials}


def autotune_batched(Qs) -> dict:
    """Tune a batch's plan on the current device and install it (qubo_autotune_batched_ex): the
    kernel variant for the whole batch, then the walk length per instance size.  Returns the
    variant, the tuned batch rate (states/s), the number of timed launches and, per size n
    present in the batch, the tuned walk (`walk_bits_per_n`)."""
    lib = load_library()
    packed, ns, offs, dt = _pack(Qs)
    p = Plan()
    per_n = (Plan * 65)()
    _check(lib.qubo_autotune_batched_ex(_ptr(packed), _ptr(ns), _ptr(offs), len(ns), dt, ctypes.byref(p), per_n),
           "qubo_autotune_batched_ex")
    walks = {m: per_n[m].walk_bits for m in range(65) if per_n[m].walk_bits > 0}
    return {"variant": p.variant, "walk_bits": p.walk_bits, "states_per_s": p.states_per_s, "trials": p.trials,
            "walk_bits_per_n": walks}


def autotune_clear() -> None:
    load_library().qubo_autotune_clear()


def autotune_save(path: str) -> int:
    """Write the plans tuned on the current device to `path` (qubo_autotune_save)."""
    return _check(load_library().qubo_autotune_save(os.fsencode(path)), "qubo_autotune_save")


def autotune_load(path: str) -> int:
    """Install the plans of `path` saved on a device like the current one (qubo_autotune_load)."""
    return _check(load_library().qubo_autotune_load(os.fsencode(path)), "qubo_autotune_load")


class BatchResults:
    """Results of a batch as arrays (min, n_ties, tie codes, K lowest); indexing gives a Result."""

    def __init__(self, count, dt, topk, states_cap, mn, ties, tk, tkE, infos):
        self._args = (count, dt, topk, states_cap, mn, ties, tk, tkE, infos)
        self.min = mn
        self.count = count

    def __len__(self):
        return self.count

    def __getitem__(self, i):
        count, dt, topk, states_cap, mn, ties, tk, tkE, infos = self._args
        if i < 0:
            i += count
        inf = infos[i]
        k = inf.n_topk
        isf = dt in (QUBO_F32, QUBO_F64)
        return Result(float(mn[i]) if isf else int(mn[i]), int(inf.n_ties),
                      ties[i * states_cap: i * states_cap + inf.n_written].copy(),
                      tk[i * topk: i * topk + k].copy(), tkE[i * topk: i * topk + k].copy(),
                      QUBO_TRUNCATED if inf.n_ties > states_cap else QUBO_OK, inf.as_dict())

    def __iter__(self):
        return (self[i] for i in range(self.count))


class Batch:
    """Device-resident batch replayed as one CUDA graph (qubo_batch_*)."""

    def __init__(self, Qs, topk: int = 0, states_cap: int = 64):
        self._lib = load_library()
        packed, ns, offs, dt = _pack(Qs)
        self.count, self.dt, self.topk, self.states_cap = len(ns), dt, topk, states_cap
        h = ctypes.c_void_p()
        _check(self._lib.qubo_batch_create(_ptr(packed), _ptr(ns), _ptr(offs), self.count, dt, topk, states_cap,
                                           ctypes.byref(h)), "qubo_batch_create")
        self._h = h
        self._out = _batch_outputs(self.count, dt, topk, states_cap)

    def run(self, stream=None) -> None:
        _check(self._lib.qubo_batch_run(self._h, _stream_ptr(stream)), "qubo_batch_run")

    def fetch(self) -> BatchResults:
        """Wait for the last run; results stay in this batch's arrays until the next fetch."""
        mn, ties, tk, tkE, infos = self._out
        _check(self._lib.qubo_batch_fetch(self._h, _ptr(mn), _ptr(ties), _ptr(tk), _ptr(tkE), infos),
               "qubo_batch_fetch")
        return BatchResults(self.count, self.dt, self.topk, self.states_cap, mn, ties, tk, tkE, infos)

    def close(self) -> None:
        if getattr(self, "_h", None):
            self._lib.qubo_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()


def solve_wide(Q, n_inner: int, outer_begin: int = 0, outer_count: int | None = None, topk: int = 0,
               states_cap: int = 64, plain: bool = False, margin: float = 0.0, time_limit: float = 0.0,
               stream=None) -> Result:
    """Minimum over the sub-problems of a wide instance (qubo_solve_wide): variables
    0..n_inner-1 scanned, variables n_inner..n-1 fixed to each outer value in
    [outer_begin, outer_begin + outer_count) (all 2^(n - n_inner) values by default).  State
    codes are Python ints (bit i = variable i); ties and topk are lists of them."""
    lib = load_library()
    Qm, dt = as_qubo_matrix(Q)
    n = Qm.shape[0]
    if outer_count is None:
        outer_count = (1 << (n - n_inner)) - outer_begin
    isf = dt in (QUBO_F32, QUBO_F64)
    o = Options(topk=topk, flags=QUBO_FLAG_PLAIN if plain else 0, margin=margin, time_limit_s=time_limit)
    mn = np.zeros(1, dtype=np.float64 if isf else np.int64)
    st_codes = np.zeros(2 * max(states_cap, 1), dtype=np.uint64)
    nt = np.zeros(1, dtype=np.uint64)
    tk = np.zeros(2 * max(topk, 1), dtype=np.uint64)
    tkE = np.zeros(max(topk, 1), dtype=np.float64 if isf else np.int64)
    info = ResultInfo()
    st = _check(lib.qubo_solve_wide(_ptr(Qm), n, dt, n_inner, outer_begin, outer_count, ctypes.byref(o), _ptr(mn),
                                    _ptr(st_codes), states_cap, _ptr(nt), _ptr(tk), _ptr(tkE), ctypes.byref(info),
                                    _stream_ptr(stream)), "qubo_solve_wide")
    wide = lambda a, k: [int(a[2 * t]) | (int(a[2 * t + 1]) << 64) for t in range(k)]  # noqa: E731
    k = int(info.n_topk)
    return Result(float(mn[0]) if isf else int(mn[0]), int(nt[0]), wide(st_codes, int(info.n_written)),
                  wide(tk, k), tkE[:k].copy(), st, info.as_dict())


def plan_query(Q, topk: int = 0, split_k: int = 0, walk_bits: int = 0, fix_bits: int = 0, fix_value: int = 0,
               plain: bool = False, int32: bool = False, rigorous: bool = False, margin: float = 0.0) -> dict:
    """The plan a solve with these options would run (qubo_plan_query), computed on the host alone:
    accumulator, split, walk, suffix bits, columns per thread, factored rows, anchoring period."""
    lib = load_library()
    Qm, dt = as_qubo_matrix(Q)
    o = Options(split_k=split_k, topk=topk, fix_bits=fix_bits, walk_bits=walk_bits, fix_value=fix_value,
                flags=_flags(plain, int32, rigorous), margin=margin)
    info = ResultInfo()
    _check(lib.qubo_plan_query(_ptr(Qm), Qm.shape[0], dt, ctypes.byref(o), ctypes.byref(info)), "qubo_plan_query")
    d = info.as_dict()
    return {k: d[k] for k in ("acc", "n", "split_k", "walk_bits", "suffix_bits", "cols_per_thread", "zero_rows",
                              "anchor_bits", "fp32_err_bound", "fp32_rigorous_anchor_bits", "reg_rows",
                              "variant", "grouped")}


def solve_window(Q, window: float, cap: int = 1 << 16, fix_bits: int = 0, fix_value: int = 0, plain: bool = False,
                 stream=None):
    """Every state with E <= E_min + window in (E, code) order (qubo_solve_window).
    Returns (count, codes, energies, info)."""
    lib = load_library()
    Qm, dt = as_qubo_matrix(Q)
    isf = dt in (QUBO_F32, QUBO_F64)
    o = Options(fix_bits=fix_bits, fix_value=fix_value, flags=QUBO_FLAG_PLAIN if plain else 0)
    codes = np.zeros(max(cap, 1), dtype=np.uint64)
    E = np.zeros(max(cap, 1), dtype=np.float64 if isf else np.int64)
    cnt = np.zeros(1, dtype=np.uint64)
    info = ResultInfo()
    _check(lib.qubo_solve_window(_ptr(Qm), Qm.shape[0], dt, float(window), ctypes.byref(o), _ptr(codes), _ptr(E), cap,
                                 _ptr(cnt), ctypes.byref(info), _stream_ptr(stream)), "qubo_solve_window")
    k = int(info.n_written)
    return int(cnt[0]), codes[:k].copy(), E[:k].copy(), info.as_dict()


def solve_batched(Qs, topk: int = 0, states_cap: int = 64, stream=None) -> "BatchResults":
    """Solve many instances in one persistent launch (qubo_solve_batched).  All matrices must
    share one dtype.  The results are array-backed; indexing or iterating gives Result objects."""
    lib = load_library()
    packed, ns, offs, dt = _pack(Qs)
    count = len(ns)
    mn, ties, tk, tkE, infos = _batch_outputs(count, dt, topk, states_cap)
    st = lib.qubo_solve_batched(_ptr(packed), _ptr(ns), _ptr(offs), count, dt, topk, _ptr(mn), _ptr(ties),
                                states_cap, _ptr(tk), _ptr(tkE), infos, _stream_ptr(stream))
    _check(st, "qubo_solve_batched")
    return _batch_results(count, dt, topk, states_cap, mn, ties, tk, tkE, infos)


def solve_noalloc(Q, states_cap: int = 64, stream=None) -> Result:
    """Minimum and tie set through qubo_solve_noalloc, which takes all its device scratch from a
    fixed array inside the library and allocates nothing (for callers that must not allocate;
    integer Q, n <= 40, states_cap <= 4096, no K lowest)."""
    lib = load_library()
    Qm, dt = as_qubo_matrix(Q)
    if dt not in (QUBO_I16, QUBO_I32):
        raise ValueError("solve_noalloc takes an integer Q")
    n = Qm.shape[0]
    mn = np.zeros(1, dtype=np.int64)
    nt = np.zeros(1, dtype=np.uint64)
    ties = np.zeros(max(states_cap, 1), dtype=np.uint64)
    st = _check(lib.qubo_solve_noalloc(_ptr(Qm), n, dt, _ptr(mn), _ptr(ties) if states_cap else None, states_cap,
                                       _ptr(nt), _stream_ptr(stream)), "qubo_solve_noalloc")
    k = min(int(nt[0]), states_cap)
    return Result(int(mn[0]), int(nt[0]), ties[:k].copy(), np.zeros(0, np.uint64), np.zeros(0, np.int64), st, {})


class Problem:
    """Device-resident problem: upload once, run sub-cubes, fetch (qubo_problem_*)."""

    def __init__(self, Q, topk: int = 0, split_k: int = 0, walk_bits: int = 0, plain: bool = False,
                 margin: float = 0.0, time_limit: float = 0.0, int32: bool = False, rigorous: bool = False):
        self._lib = load_library()
        Qm, dt = as_qubo_matrix(Q)
        self.n = Qm.shape[0]
        self.topk = topk
        self.is_float = dt in (QUBO_F32, QUBO_F64)
        o = Options(split_k=split_k, topk=topk, walk_bits=walk_bits, flags=_flags(plain, int32, rigorous),
                    margin=margin, time_limit_s=time_limit)
        h = ctypes.c_void_p()
        _check(self._lib.qubo_problem_create(_ptr(Qm), self.n, dt, ctypes.byref(o), ctypes.byref(h)),
               "qubo_problem_create")
        self._h = h

    def run(self, fix_bits: int = 0, fix_value: int = 0, stream=None) -> None:
        _check(self._lib.qubo_problem_run(self._h, fix_bits, fix_value, _stream_ptr(stream)), "qubo_problem_run")

    def fetch(self, states_cap: int = 1 << 16) -> Result:
        edt = np.float64 if self.is_float else np.int64
        mn = np.zeros(1, dtype=edt)
        ties = np.zeros(states_cap, dtype=np.uint64)
        tk = np.zeros(self.topk, dtype=np.uint64)
        tkE = np.zeros(self.topk, dtype=edt)
        info = ResultInfo()
        st = _check(self._lib.qubo_problem_fetch(self._h, _ptr(mn), _ptr(ties), states_cap, _ptr(tk), _ptr(tkE),
                                                 ctypes.byref(info)), "qubo_problem_fetch")
        k = info.n_topk
        return Result(float(mn[0]) if self.is_float else int(mn[0]), int(info.n_ties),
                      ties[: info.n_written].copy(), tk[:k].copy(), tkE[:k].copy(), st, info.as_dict())

    def close(self) -> None:
        if getattr(self, "_h", None):
            self._lib.qubo_problem_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()


def shard_subcubes(fix_bits: int, world: int, rank: int) -> list[int]:
    """Sub-cubes (values of the top fix_bits code bits) scanned by `rank` of `world` ranks: a
    round-robin split of the 2^fix_bits independent parts (Sec. 3.3.1)."""
    return [v for v in range(1 << fix_bits) if v % world == rank]


def merge_all(results, states_cap: int, topk: int) -> Result:
    """Fold qubo_merge over results of disjoint state sets."""
    acc = None
    for r in results:
        acc = r if acc is None else merge(acc, r, states_cap, topk)
    return acc


def merge(a: Result, b: Result, states_cap: int, topk: int) -> Result:
    """Merge the results of two disjoint state sets (qubo_merge)."""
    lib = load_library()
    isf = isinstance(a.min, float)
    edt = np.float64 if isf else np.int64

    def part(r: Result, keep):
        ties = np.ascontiguousarray(r.ties, dtype=np.uint64)
        tk = np.ascontiguousarray(r.topk, dtype=np.uint64)
        tkE = np.ascontiguousarray(r.topk_E, dtype=edt)
        keep.extend([ties, tk, tkE])
        return Partial(is_float=int(isf), n_topk=len(tk), min_i=0 if isf else int(r.min), min_f=float(r.min),
                       n_ties=r.n_ties, n_written=len(ties), states_scanned=int(r.info.get("states_scanned", 1)),
                       ties=ties.ctypes.data if ties.size else None, topk=tk.ctypes.data if tk.size else None,
                       topk_E=tkE.ctypes.data if tkE.size else None)

    keep = []
    pa, pb = part(a, keep), part(b, keep)
    ot = np.zeros(max(states_cap, 1), dtype=np.uint64)
    ok = np.zeros(max(topk, 1), dtype=np.uint64)
    okE = np.zeros(max(topk, 1), dtype=edt)
    po = Partial(ties=ot.ctypes.data, topk=ok.ctypes.data, topk_E=okE.ctypes.data)
    _check(lib.qubo_merge(ctypes.byref(pa), ctypes.byref(pb), states_cap, topk, ctypes.byref(po)), "qubo_merge")
    mval = po.min_f if isf else po.min_i
    return Result(float(mval) if isf else int(mval), int(po.n_ties), ot[: po.n_written].copy(),
                  ok[: po.n_topk].copy(), okE[: po.n_topk].copy(), 0,
                  {"states_scanned": int(po.states_scanned)})
def merge_wide(a: Result, b: Result, states_cap: int, topk: int) -> Result:
    """Merge two results of qubo_solve_wide over disjoint state sets (qubo_merge_wide); codes are
    Python ints of up to 128 bits."""
    lib = load_library()
    isf = isinstance(a.min, float)
    edt = np.float64 if isf else np.int64

    def words(codes):
        w = np.zeros(2 * max(len(codes), 1), dtype=np.uint64)
        for t, c in enumerate(codes):
            w[2 * t], w[2 * t + 1] = int(c) & (2**64 - 1), int(c) >> 64
        return w

    def part(r: Result, keep):
        ties, tk = words(r.ties), words(r.topk)
        tkE = np.ascontiguousarray(r.topk_E, dtype=edt)
        keep.extend([ties, tk, tkE])
        return PartialWide(is_float=int(isf), n_topk=len(r.topk), min_i=0 if isf else int(r.min),
                           min_f=float(r.min), n_ties=r.n_ties, n_written=len(r.ties),
                           states_scanned=int(r.info.get("states_scanned", 1)), ties=ties.ctypes.data,
                           topk=tk.ctypes.data, topk_E=tkE.ctypes.data if tkE.size else None)

    keep = []
    pa, pb = part(a, keep), part(b, keep)
    ot = np.zeros(2 * max(states_cap, 1), dtype=np.uint64)
    ok = np.zeros(2 * max(topk, 1), dtype=np.uint64)
    okE = np.zeros(max(topk, 1), dtype=edt)
    po = PartialWide(ties=ot.ctypes.data, topk=ok.ctypes.data, topk_E=okE.ctypes.data)
    _check(lib.qubo_merge_wide(ctypes.byref(pa), ctypes.byref(pb), states_cap, topk, ctypes.byref(po)),
           "qubo_merge_wide")
    mval = po.min_f if isf else po.min_i
    wide = lambda w, k: [int(w[2 * t]) | (int(w[2 * t + 1]) << 64) for t in range(k)]  # noqa: E731
    return Result(float(mval) if isf else int(mval), int(po.n_ties), wide(ot, int(po.n_written)),
                  wide(ok, int(po.n_topk)), okE[: po.n_topk].copy(), 0, {"states_scanned": int(po.states_scanned)})


def merge_all_wide(results, states_cap: int, topk: int) -> Result:
    """Fold qubo_merge_wide over results of disjoint state sets."""
    acc = None
    for r in results:
        acc = r if acc is None else merge_wide(acc, r, states_cap, topk)
    return acc


