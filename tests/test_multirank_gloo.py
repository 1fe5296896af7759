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
