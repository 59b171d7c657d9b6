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


def _grad_worker(rank, world, port, q):
    """Each rank takes one of the differentiation workload's cameras and computes its
    partial gradient (the oracle's adjoint stands in for the GPU adjoint on CPU); the
    library's all-reduce sums them."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import numpy as np

    import oracle
    import synthetic
    from paper_2103_01954_gb300 import torch_ops as T

    sc, rays, _ = synthetic.make_config("diff_small_64x8^3_2x48x40", 2)
    g = np.random.default_rng(3).standard_normal((rays.n, 4))
    per = rays.n // world
    sl = slice(rank * per, (rank + 1) * per)
    shard = synthetic.Rays(o=rays.o[sl], d=rays.d[sl], t_near=rays.t_near, t_far=rays.t_far, dt=rays.dt)
    R = oracle.backward(sc, shard, g[sl], 3)
    grads = [torch.from_numpy(R[k]) for k in ("g_payload", "g_t", "g_q", "g_s")]
    T.allreduce_gradients(grads)
    q.put((rank, [x.numpy() for x in grads]))
    dist.barrier()
    dist.destroy_process_group()


def test_backward_exchange_sums_the_shards():
    """Two gloo ranks, each with half of the rays: after the exchange every rank holds
    the gradient of the whole batch."""
    import numpy as np

    import oracle
    import synthetic

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_grad_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=300) for _ in range(2))
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    sc, rays, _ = synthetic.make_config("diff_small_64x8^3_2x48x40", 2)
    g = np.random.default_rng(3).standard_normal((rays.n, 4))
    full = oracle.backward(sc, rays, g, 3)
    for rank in (0, 1):
        for k, v in zip(("g_payload", "g_t", "g_q", "g_s"), res[rank]):
            np.testing.assert_allclose(v, full[k], rtol=1e-10, atol=1e-12 * np.abs(full[k]).max())


def test_exchange_is_a_no_op_without_a_group():
    from paper_2103_01954_gb300 import torch_ops as T

    g = torch.ones(3)
    T.allreduce_gradients([g, None])
    assert torch.equal(g, torch.ones(3))
