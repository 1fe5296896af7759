"""C-ABI checks that need no GPU: the library builds and loads, exports every entry point that
include/qubo.h declares, and its host-only logic (status strings, result merge, argument
checks) behaves."""
import os
import re

import numpy as np
import pytest

import oracle
from paper_2607_04857_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def q():
    from paper_2607_04857_gb300 import build as qbuild

    qbuild.build()
    import paper_2607_04857_gb300 as q

    q.load_library()
    return q


def declared_functions():
    src = open(os.path.join(ROOT, "include", "qubo.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qubo_[a-z_]+)\s*\(", src)))


def test_header_declares_the_binding_list(q):
    assert declared_functions() == sorted(q.EXPORTS)


def test_every_declared_symbol_is_exported(q):
    import ctypes

    lib = ctypes.CDLL(q.LIB_PATH)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_library_is_the_in_tree_build(q):
    assert os.path.dirname(q.LIB_PATH) == os.path.join(ROOT, "paper_2607_04857_gb300")


def test_strerror_and_version(q):
    assert q.strerror(0) == "ok"
    assert "argument" in q.strerror(-1)
    assert "sm_103a" in q.version()


def test_bad_arguments_are_rejected_before_any_device_work(q):
    lib = q.load_library()
    Q = np.zeros((4, 4), dtype=np.int32)
    out = np.zeros(1, dtype=np.int64)
    # n out of range, bad dtype, null Q, topk beyond the cap
    assert lib.qubo_solve(Q.ctypes.data, 0, 2, 0, 0, out.ctypes.data, None, 0, None, None, None, None) == -1
    assert lib.qubo_solve(Q.ctypes.data, 65, 2, 0, 0, out.ctypes.data, None, 0, None, None, None, None) == -1
    assert lib.qubo_solve(Q.ctypes.data, 4, 9, 0, 0, out.ctypes.data, None, 0, None, None, None, None) == -1
    assert lib.qubo_solve(None, 4, 2, 0, 0, out.ctypes.data, None, 0, None, None, None, None) == -1
    assert lib.qubo_solve(Q.ctypes.data, 4, 2, 0, 5000, out.ctypes.data, None, 0, None, None, None, None) == -1


def test_every_entry_point_rejects_bad_arguments_on_the_host(q):
    """Argument errors are QUBO_ERR_ARG and are found before any device work (no GPU here)."""
    import ctypes

    lib = q.load_library()
    ARG = q.QUBO_ERR_ARG
    Q = np.zeros((4, 4), dtype=np.int32)
    Q70 = np.zeros((70, 70), dtype=np.int32)
    out = np.zeros(1, dtype=np.int64)
    codes, E, cnt = np.zeros(8, dtype=np.uint64), np.zeros(8, dtype=np.int64), np.zeros(1, dtype=np.uint64)
    o = q.Options(fix_bits=9)
    assert lib.qubo_solve_ex(Q.ctypes.data, 4, 2, ctypes.byref(o), out.ctypes.data, None, 0, None, None, None, None) == ARG
    assert lib.qubo_solve_ex(Q.ctypes.data, 4, 2, None, None, None, 0, None, None, None, None) == ARG
    for window in (-1.0, float("nan"), float("inf")):
        assert lib.qubo_solve_window(Q.ctypes.data, 4, 2, window, None, codes.ctypes.data, E.ctypes.data, 8,
                                     cnt.ctypes.data, None, None) == ARG
    assert lib.qubo_solve_window(Q.ctypes.data, 4, 2, 1.0, None, codes.ctypes.data, E.ctypes.data, 8, None, None,
                                 None) == ARG
    w = np.zeros(16, dtype=np.uint64)
    for n, inner, count in ((70, 65, 1), (70, 30, 0), (129, 30, 1), (70, 0, 1)):
        assert lib.qubo_solve_wide(Q70.ctypes.data, n, 2, inner, 0, count, None, out.ctypes.data, w.ctypes.data, 8,
                                   None, None, None, None, None) == ARG
    ns, offs, Qb = np.array([45], dtype=np.int32), np.zeros(1, dtype=np.uint64), np.zeros(45 * 45, dtype=np.int32)
    for count in (1, 0):  # n = 45 is beyond the batched limit; an empty batch
        assert lib.qubo_solve_batched(Qb.ctypes.data, ns.ctypes.data, offs.ctypes.data, count, 2, 0, out.ctypes.data,
                                      None, 0, None, None, None, None) == ARG
    assert lib.qubo_plan_query(Q.ctypes.data, 4, 2, None, None) == ARG
    assert lib.qubo_merge(None, None, 8, 0, None) == ARG


def _as_result(q, o, scanned):
    return q.Result(o.min, o.n_ties, o.ties, o.topk, o.topk_E, 0, {"states_scanned": scanned})


@pytest.mark.parametrize("kind", ["int", "float", "degenerate"])
def test_merge_of_subcube_results_equals_full_solve(q, kind):
    """qubo_merge (the reduce of Sec. 3.3) applied to oracle results of disjoint sub-cubes gives
    the oracle result of the whole cube."""
    n, f, K, cap = 16, 3, 8, 100
    if kind == "int":
        Q = wl.upper_int(n, -20, 20, seed=5)
    elif kind == "float":
        Q = wl.sk_float32(n, seed=6)
    else:
        Q = wl.diagonal(n, seed=7, zeros=9)
    full = oracle.solve(Q, topk=K, cap=cap)
    acc = None
    for v in range(1 << f):
        part = _as_result(q, oracle.solve(Q, topk=K, cap=cap, fix_bits=f, fix_value=v), 1 << (n - f))
        acc = part if acc is None else q.merge(acc, part, cap, K)
    assert acc.min == full.min and acc.n_ties == full.n_ties
    assert np.array_equal(acc.ties, full.ties)
    assert np.array_equal(acc.topk, full.topk) and np.array_equal(acc.topk_E, full.topk_E)
    assert acc.info["states_scanned"] == 1 << n


def test_ncu_summary_arithmetic(tmp_path):
    """The counters summary: instructions per state = warp instructions x 32 / states, and the
    issue roofline = SMs x 128 lanes x clock / instructions per state."""
    from paper_2607_04857_gb300 import ncu_summary

    rows = [
        '"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size",'
        '"Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"',
        '"0","1","python","h","scan_kernel","1","7","(128, 1, 1)","(456, 1, 1)","0","10.3","",'
        '"sm__inst_executed.sum","inst","2,147,483,648"',
        '"0","1","python","h","scan_kernel","1","7","(128, 1, 1)","(456, 1, 1)","0","10.3","",'
        '"dram__bytes_read.sum","byte","1,024"',
        '"0","1","python","h","scan_kernel","1","7","(128, 1, 1)","(456, 1, 1)","0","10.3","",'
        '"gpu__time_duration.sum","ns","1,000,000"',
    ]
    p = tmp_path / "x.csv"
    p.write_text("==PROF== noise\n" + "\n".join(rows) + "\n")
    s = ncu_summary.summarise(ncu_summary.read_metrics(str(p)), 1 << 36)
    assert s["inst_per_state"] == 2**31 * 32 / 2**36 == 1.0
    assert s["issue_roofline_states_per_s"] == 152 * 128 * 2070e6
    assert s["dram_bytes_per_state"] == 1024 / 2**36
    assert s["states_per_s_under_ncu"] == 2**36 / 1e-3


def build_c_client(q, out_dir):
    """Compile tests/c_abi_client.c with the system C compiler against include/qubo.h and link it
    to the in-tree libqubo.so (no Python between the client and the library)."""
    import shutil
    import subprocess

    cc = shutil.which("cc") or shutil.which("gcc")
    if cc is None:
        pytest.skip("no C compiler")
    libdir = os.path.dirname(q.LIB_PATH)
    exe = os.path.join(str(out_dir), "c_abi_client")
    r = subprocess.run([cc, "-std=c11", "-Wall", "-Wextra", "-Werror", "-O2", "-I", os.path.join(ROOT, "include"),
                        os.path.join(ROOT, "tests", "c_abi_client.c"), "-L", libdir, "-lqubo",
                        f"-Wl,-rpath,{libdir}", "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_c_client_compiles_and_links_against_the_header(q, tmp_path):
    assert os.path.exists(build_c_client(q, tmp_path))


def test_pack_batch_layout(q):
    """pack_batch lays the matrices out row-major one after another, with their sizes and element
    offsets, in one dtype; a packed batch passes through unchanged."""
    mats = [wl.upper_int(n, -9, 9, seed=n, dtype=np.int16) for n in (3, 5, 4)]
    p = q.pack_batch(mats)
    assert len(p) == 3 and p.ns.tolist() == [3, 5, 4] and p.offs.tolist() == [0, 9, 34]
    assert p.packed.dtype == np.int16 and p.packed.size == 9 + 25 + 16
    for M, o in zip(mats, p.offs.tolist()):
        n = M.shape[0]
        assert np.array_equal(p.packed[o:o + n * n].reshape(n, n), M)
    assert q.pack_batch(p).packed is p.packed
    with pytest.raises(ValueError):
        q.pack_batch([mats[0], mats[1].astype(np.int32)])


def test_merge_rejects_inputs_whose_counts_exceed_their_arrays(q):
    """qubo_merge / qubo_merge_wide check the inputs' counts against their arrays on the host."""
    import ctypes

    lib = q.load_library()
    ties = np.zeros(4, dtype=np.uint64)
    tk = np.zeros(4, dtype=np.uint64)
    tkE = np.zeros(4, dtype=np.int64)

    def part(cls=q.Partial, **kw):
        p = cls(is_float=0, n_topk=0, min_i=0, min_f=0.0, n_ties=1, n_written=1, states_scanned=8,
                ties=ties.ctypes.data, topk=tk.ctypes.data, topk_E=tkE.ctypes.data)
        for k, v in kw.items():
            setattr(p, k, v)
        return p

    for merge, cls in ((lib.qubo_merge, q.Partial), (lib.qubo_merge_wide, q.PartialWide)):
        out = part(cls)
        good = part(cls)
        assert merge(ctypes.byref(good), ctypes.byref(part(cls)), 4, 0, ctypes.byref(out)) == 0
        for bad in (dict(ties=None), dict(n_topk=2, topk=None), dict(n_topk=2, topk_E=None), dict(n_topk=-1),
                    dict(n_written=2, n_ties=1)):
            assert merge(ctypes.byref(good), ctypes.byref(part(cls, **bad)), 4, 0, ctypes.byref(out)) == \
                q.QUBO_ERR_ARG, bad
