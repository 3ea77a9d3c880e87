"""The multi-rank host logic of bench.py (max-over-ranks time, whole-job rate) on two gloo
processes on the CPU (one GPU per rank is not available here; the data path has no collective)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    sec = bench.max_over_ranks(torch, 1.0 + rank, dist, "cpu")  # rank 1 is the slow one
    rate = bench.whole_job_rate(100.0, world, sec)
    q.put((rank, sec, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [2.0, 2.0]          # both ranks see the slowest time
    assert [o[2] for o in out] == [100.0, 100.0]      # 2 ranks x 100 units / 2 s
