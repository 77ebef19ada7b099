"""The multi-rank bookkeeping of bench.py (replicas, one per GPU): the job's
time is the slowest rank's, its work the sum over ranks.  Exercised with two
gloo processes on the CPU (no GPU involved)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, flops = bench.aggregate(100.0 + 50.0 * rank, 1e9 * (rank + 1))
    dist.barrier()
    if rank == 0:
        out.put((ms, flops))
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_sum_work():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    ms, flops = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert ms == 150.0 and flops == 3e9


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(12.5, 7.0) == (12.5, 7.0)
