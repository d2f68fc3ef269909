"""The benchmark's multi-rank harness on CPU (gloo, world size 2): each rank
times its own replica; the reported time is the max over ranks and the value
counts every rank's keys.  No GPU and no data-path collective: the sort runs
as independent replicas, one per GPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = bench.dist_env()
    assert (r, w, lr) == (rank, world, rank)
    bench.barrier(world)
    my_ms = 10.0 + 5.0 * rank          # rank 1 is the slow one
    t = bench.reduce_max(my_ms, world)
    n_per_rank = 1000
    value = world * n_per_rank / (t / 1e3)
    q.put((rank, t, value))
    bench.barrier(world)
    dist.destroy_process_group()


def test_two_rank_max_over_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get() for _ in range(world))
    assert [r[1] for r in res] == [15.0, 15.0]            # every rank sees the max
    assert res[0][2] == pytest.approx(2 * 1000 / 0.015)  # whole-job keys over the slowest rank's time


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_max(3.5, 1) == 3.5
