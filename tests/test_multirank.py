"""The N > 1 bench path runs independent replicas: the only cross-rank steps are
the timing reduction (max of times, sum of work) and rank-0-only printing.
Covered here with world_size 2 on the gloo backend (CPU)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    ms, count = bench.reduce_over_ranks(10.0 + rank, 1000 * (rank + 1))
    assert bench.dist_env() == (ws, rank, rank)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ms, count))


def test_replica_reduction_gloo_ws2():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, count in res:
        assert ms == 11.0          # slowest replica
        assert count == 3000.0     # work of both replicas


def test_single_process_reduction_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(5.0, 7) == (5.0, 7.0)


def test_reference_arm_nonzero_rank_prints_nothing(capsys, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        steps, warmup, gpus = 1, 0, 2
    assert bench.run_reference(A()) == 0
    assert capsys.readouterr().out == ""
