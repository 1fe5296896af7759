"""Sharding across ranks (world_size 2, gloo on the CPU): every rank takes its own sub-cubes
(the round-robin split the benchmark uses under torchrun), the partial results are gathered, and
qubo_merge combines them into the result of the whole cube.  Partial results come from the CPU
oracle here, so the exchange and merge logic is tested without a GPU."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, kind, out_path):
    import sys

    sys.path.insert(0, ROOT)
    import oracle
    import paper_2607_04857_gb300 as q
    from paper_2607_04857_gb300 import build as qbuild
    from paper_2607_04857_gb300 import workloads as wl

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n, fb, K, cap = 20, 3, 8, 64
    Q = wl.upper_int(n, -40, 40, seed=77) if kind == "int" else wl.sk_float32(n, seed=78)
    mine = []
    for v in q.shard_subcubes(fb, world, rank):
        o = oracle.solve(Q, topk=K, cap=cap, fix_bits=fb, fix_value=v)
        mine.append((o.min, o.n_ties, o.ties.tolist(), o.topk.tolist(), o.topk_E.tolist()))
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    if rank == 0:
        qbuild.build()
        edt = np.float64 if kind == "float" else np.int64
        parts = [q.Result(m, nt, np.array(t, np.uint64), np.array(k, np.uint64), np.array(e, edt), 0,
                          {"states_scanned": 1 << (n - fb)}) for rk in gathered for (m, nt, t, k, e) in rk]
        merged = q.merge_all(parts, cap, K)
        full = oracle.solve(Q, topk=K, cap=cap)
        ok = (merged.min == full.min and merged.n_ties == full.n_ties and np.array_equal(merged.ties, full.ties)
              and np.array_equal(merged.topk, full.topk) and len(parts) == 1 << fb
              and merged.info["states_scanned"] == 1 << n)
        with open(out_path, "w") as fh:
            fh.write("ok" if ok else f"mismatch {merged.min} {full.min} {merged.n_ties} {full.n_ties}")
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("kind", ["int", "float"])
def test_two_rank_shards_merge_to_whole(tmp_path, kind):
    out = tmp_path / "result.txt"
    mp.start_processes(_rank_main, args=(2, _free_port(), kind, str(out)), nprocs=2, join=True,
                       start_method="spawn")
    assert out.read_text() == "ok"


def test_shards_partition_the_subcubes():
    import paper_2607_04857_gb300 as q

    for world in (1, 2, 3, 8):
        parts = [q.shard_subcubes(5, world, r) for r in range(world)]
        flat = sorted(v for p in parts for v in p)
        assert flat == list(range(32))


def _rank_main_wide(rank, world, port, kind, out_path):
    """Wide instance (n = 70): each rank takes its outer values (the top 50 variables fixed per
    value), solves their 20-variable sub-problems with the oracle, and rank 0 merges the gathered
    results with qubo_merge_wide (128-bit codes)."""
    import sys

    sys.path.insert(0, ROOT)
    import oracle
    import paper_2607_04857_gb300 as q
    from paper_2607_04857_gb300 import build as qbuild
    from paper_2607_04857_gb300 import workloads as wl

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n, m, K, cap = 70, 20, 6, 64
    Q = wl.upper_int(n, -40, 40, seed=70) if kind == "int" else wl.sk_float32(n, seed=71).astype(np.float64)
    base = (1 << 49) + 12345
    values = [base + i for i in range(8)]
    mine = []
    for v in values[rank::world]:
        R, c = oracle.reduce(Q, m, v)
        o = oracle.solve(R, topk=K, cap=cap)
        mine.append((o.min + c, o.n_ties, [int(t) | (v << m) for t in o.ties],
                     [int(t) | (v << m) for t in o.topk], [e + c for e in o.topk_E.tolist()]))
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    if rank == 0:
        qbuild.build()
        edt = np.float64 if kind == "float" else np.int64
        parts = [q.Result(mn, nt, t, k, np.array(e, edt), 0, {"states_scanned": 1 << m})
                 for rk in gathered for (mn, nt, t, k, e) in rk]
        merged = q.merge_all_wide(parts, cap, K)
        # reference: the plain definition over the gathered parts
        best = min(p.min for p in parts)
        ties = sorted(c for p in parts if p.min == best for c in p.ties)[:cap]
        n_ties = sum(p.n_ties for p in parts if p.min == best)
        top = sorted((e, c) for p in parts for e, c in zip(p.topk_E.tolist(), p.topk))[:K]
        ok = (merged.min == best and merged.n_ties == n_ties and merged.ties == ties
              and merged.topk == [c for _, c in top] and merged.topk_E.tolist() == [e for e, _ in top]
              and merged.info["states_scanned"] == len(values) << m and max(merged.ties) >= 1 << 64)
        with open(out_path, "w") as fh:
            fh.write("ok" if ok else f"mismatch {merged.min} {best} {merged.n_ties} {n_ties}")
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("kind", ["int", "float"])
def test_two_rank_wide_ranges_merge(tmp_path, kind):
    out = tmp_path / "result.txt"
    mp.start_processes(_rank_main_wide, args=(2, _free_port(), kind, str(out)), nprocs=2, join=True,
                       start_method="spawn")
    assert out.read_text() == "ok"
