"""bench.py's multi-rank logic on CPU: two gloo ranks run independent replicas,
time them, take the max over ranks and report the whole-job rate (no collective
on the data path: envs are independent, paper App. B)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    w, r, local = bench.dist_init()
    assert (w, r, local) == (world, rank, rank)
    bench.barrier(w)
    # each replica "takes" a different time; every rank must see the max
    t = 100.0 + 50.0 * rank
    m = bench.max_over_ranks(t, w)
    val = bench.job_throughput(1000, 4, w, m)
    q.put((rank, m, val))
    dist.destroy_process_group()


def test_two_rank_max_and_weak_scaling_rate():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get() for _ in range(world))
    assert [m for _, m, _ in res] == [150.0, 150.0]
    # 2 ranks x 4 steps x 1000 units in 0.15 s
    assert res[0][2] == pytest.approx(2 * 4 * 1000 / 0.15)


def test_single_rank_defaults():
    import bench
    assert bench.max_over_ranks(3.0, 1) == 3.0
    assert bench.job_throughput(10, 2, 1, 1000.0) == 20.0
