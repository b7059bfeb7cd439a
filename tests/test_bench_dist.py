"""bench.py's multi-rank logic on CPU with two gloo ranks: every rank runs its
own replica ("replicas only", no data-path collective); the step time that is
reported is the maximum over ranks and the value sums the ranks' work."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, results):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench

    class A:
        pass

    w, r, local, pg = bench.dist_setup(A())
    assert (w, r) == (world, rank) and pg is not None
    bench.barrier(pg)
    t = bench.max_over_ranks(pg, 1.0 + rank)  # rank 1 is the slow one
    results[rank] = t
    dist.destroy_process_group()


@pytest.mark.skipif(torch.cuda.is_available(), reason="CPU gloo path (with a GPU, bench uses NCCL)")
def test_two_rank_max_time_gloo():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    results = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, results)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert dict(results) == {0: 2.0, 1: 2.0}
