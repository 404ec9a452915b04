"""bench.py's multi-rank logic on CPU: two gloo ranks each hold one shard of the
workload (their own range of global env ids under the same parameters), time
them, take the max over ranks and report the whole-job rate (no collective on
the data path: envs are independent, paper App. B).  The shard arithmetic is
checked through the C ABI's host-side sizing: each rank's economy shard draws
the agent counts of its own global envs, and the shards' slots add up to those
of one context over all envs."""
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


def _shard_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    from paper_2408_00930_gb300 import warpsci as W
    w, r, _ = bench.dist_init()
    n = 37
    base, n_r = bench.shard_of(n, w, r)
    cfg, _ = W.make_config(W.WS_ENV_ECONOMY, W.WS_PATH_BATCHED_BF16, n_r, 10, 540, 128, 128,
                           param_seed=5, env_base=base)
    st, _, _, slots = W.ws_query_bytes(cfg)
    assert st == W.WS_OK
    got = [None] * w
    dist.all_gather_object(got, (base, n_r, slots))
    q.put((r, got))
    dist.destroy_process_group()


def test_two_rank_env_shards_partition_the_workload():
    import oracle
    from paper_2408_00930_gb300 import build
    from paper_2408_00930_gb300 import warpsci as W
    build.build()
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    procs = [ctx.Process(target=_shard_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = [q.get() for _ in range(world)]
    assert res[0][1] == res[1][1]                      # both ranks saw the same shards
    shards = res[0][1]
    ranges = [set(range(b, b + m)) for b, m, _ in shards]
    assert not (ranges[0] & ranges[1]) and ranges[0] | ranges[1] == set(range(74))
    # slots of the shards == slots of one context over all 74 envs == the
    # oracle's agent counts of the global env ids (+ one planner per env)
    cfg, _ = W.make_config(W.WS_ENV_ECONOMY, W.WS_PATH_BATCHED_BF16, 74, 10, 540, 128, 128,
                           param_seed=5)
    union = W.ws_query_bytes(cfg)[3]
    assert sum(sl for _, _, sl in shards) == union
    assert union == sum(oracle.econ_agent_count(5, e) for e in range(74)) + 74
    for b, m, sl in shards:
        assert sl == sum(oracle.econ_agent_count(5, e) for e in range(b, b + m)) + m
    # a range past the 32-bit env ids is rejected
    bad, _ = W.make_config(W.WS_ENV_CONTROL, W.WS_PATH_PLAIN_FP32, 10, 4, 200, 8, 8,
                           env_base=2**32 - 5)
    assert W.ws_query_bytes(bad)[0] == W.WS_ERR_INVALID
