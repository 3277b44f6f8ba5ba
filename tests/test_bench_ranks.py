"""Host logic of the multi-rank benchmark on CPU: two gloo ranks (127.0.0.1).  Each rank solves
its own replica, so the only exchange is the job time, taken as the slowest rank's; the
reference arm runs on rank 0 only."""
import multiprocessing as mp
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    slowest = bench._max_over_ranks(dist, 10.0 + 5.0 * rank, torch.device("cpu"))
    ranks = bench._dist()

    class A:
        warmup, steps = 3, 1
    ref = bench.run_reference(A) if rank != 0 else "skipped on rank 0"
    q.put((rank, slowest, ranks, ref))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [15.0, 15.0]          # every rank sees the slowest time
    assert [o[2] for o in out] == [(2, 0, 0), (2, 1, 1)]
    assert out[1][3] is None                              # the reference arm does no work off rank 0
