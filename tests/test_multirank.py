"""The benchmark's multi-GPU logic on CPU: two gloo ranks, each with its own frame
(weak scaling, no data-path collective); the job's time is the slowest rank's."""
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

    ms_local = [3.0, 5.0][rank]
    ms, value = bench.aggregate(ms_local, 683008, world)
    q.put((rank, ms, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get() for _ in range(2))
    for rank, ms, value in res:
        assert ms == pytest.approx(5.0)
        assert value == pytest.approx(2 * 683008 / 5e-3 / 1e6)


def test_single_rank_has_no_collective():
    import bench

    ms, value = bench.aggregate(2.0, 1000, 1)
    assert ms == 2.0 and value == pytest.approx(1000 / 2e-3 / 1e6)
    assert not dist.is_initialized()
