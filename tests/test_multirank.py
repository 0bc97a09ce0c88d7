"""Multi-rank host logic of bench.py (replicas only): world_size-2 gloo ranks on CPU.

Each rank factors and solves its own system (distinct seeds), and the reported step time
is the maximum over ranks, which every rank must receive."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(0.25 * (rank + 1), dist, "cpu")
    dist.barrier()
    q.put((rank, t, bench.replica_seed(rank)))
    dist.destroy_process_group()


def test_replicas_report_max_over_ranks():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, _, _ in res] == [0, 1]
    assert all(abs(t - 0.5) < 1e-15 for _, t, _ in res)      # both ranks see the slowest rank's time
    assert res[0][2] != res[1][2]                              # each replica its own system


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(0.125, None, "cpu") == 0.125
