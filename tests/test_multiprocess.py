"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): every rank
runs an independent replica; the reported value is the checks of all ranks
divided by the slowest rank's time (weak scaling, no collective on the data
path)."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    checks = 1000.0 * (rank + 1)
    secs = 0.5 + rank
    total, tmax = bench.aggregate(checks, secs, world)
    q.put((rank, total, tmax))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, total, tmax in out:
        assert total == 3000.0 and tmax == 1.5


def test_reference_arm_rank_nonzero_exits_quietly(capsys):
    sys.path.insert(0, ROOT)
    import bench

    class A:
        steps, warmup, cpu_sample, seed = 1, 0, 8, 0
    bench.reference_arm(A, rank=1, world=2)
    assert capsys.readouterr().out == ""
