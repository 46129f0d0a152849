"""The N > 1 benchmark path on the CPU: two gloo ranks run independent
replicas (no data-path collective); only the timing maximum and a barrier
cross ranks, and the reported value counts the work of all ranks."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        # each rank "timed" its own replica; the job time is the slowest rank
        mine = 1.0 + 0.5 * rank
        t = bench.max_over_ranks(world, mine)
        units_per_rank = 1000.0
        out.put((rank, t, units_per_rank * world / t))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling_aggregation():
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
    res = sorted(q.get(timeout=5) for _ in range(2))
    assert [r[1] for r in res] == [1.5, 1.5]              # max over ranks on both
    assert all(abs(r[2] - 2000.0 / 1.5) < 1e-9 for r in res)
