"""Serving loop: continuous batching, admission by device bytes, per-request
results identical alone and in a concurrent mix, flow control and timeouts."""
import time

import numpy as np
import pytest

from paper_2408_00930_gb300 import warpsci as W
from tests.gpu_common import need_gpu

pytestmark = pytest.mark.gpu
GB = 1 << 30


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


def req(env, n, horizon, seed, path=None, flags=0, fused=False):
    """A request of the env's test shape; fused=True asks for the configured
    shape that the BF16 path runs on its fused persistent kernel (economy
    16-128-128-20 with drawn U{8..256} agents, landscape D=24, M=4,096,
    24-256-256-48)."""
    if fused and env == W.WS_ENV_ECONOMY:
        return W.make_request(env, W.WS_PATH_BATCHED_BF16, n, horizon, 50, 540, 128, 128,
                              seed=seed, flags=flags)
    if fused and env == W.WS_ENV_LANDSCAPE:
        return W.make_request(env, W.WS_PATH_BATCHED_BF16, n, horizon, 50, 1000, 256, 256,
                              dim=24, n_gauss=4096, seed=seed, flags=flags)
    if env == W.WS_ENV_CONTROL:
        return W.make_request(env, path if path is not None else W.WS_PATH_BATCHED_BF16, n, horizon,
                              50, 200, 256, 256, seed=seed, flags=flags)
    if env == W.WS_ENV_ECONOMY:
        return W.make_request(env, path if path is not None else W.WS_PATH_BATCHED_FP32, n, horizon,
                              50, 540, 128, 128, seed=seed, flags=flags)
    if env == W.WS_ENV_ACROBOT:
        return W.make_request(env, path if path is not None else W.WS_PATH_BATCHED_BF16, n, horizon,
                              50, 500, 64, 64, seed=seed, flags=flags)
    return W.make_request(env, path if path is not None else W.WS_PATH_BATCHED_FP32, n, horizon, 50,
                          1000, 64, 64, dim=24, n_gauss=512, seed=seed, flags=flags)


FIELDS = (W.WS_F_ACTION, W.WS_F_OBS, W.WS_F_REWARD, W.WS_F_DONE)


def collect(srv, rid, n_slots, obs_dim, act_dim, n_chunks):
    out = []
    for c in range(n_chunks):
        assert srv.wait_chunk(rid, c, 60000) == W.WS_OK
        per = {}
        for f in FIELDS:
            width = {W.WS_F_ACTION: act_dim * 4, W.WS_F_OBS: obs_dim * 4, W.WS_F_REWARD: 4,
                     W.WS_F_DONE: 1}[f]
            buf = np.empty(50 * n_slots * width, np.uint8)
            assert srv.fetch(rid, f, c, buf) == W.WS_OK
            per[f] = buf.tobytes()
        out.append(per)
        assert srv.ack(rid, c) == W.WS_OK
    return out


def slots_of(q):
    cfg, _ = W.make_config(q.env, q.path, q.n_envs, 100, q.episode_limit, q.hidden0, q.hidden1,
                           dim=q.dim, n_gauss=q.n_gauss, param_seed=q.seed)
    return W.ws_query_bytes(cfg)[3]


def test_results_identical_alone_and_in_mix(torch):
    """Every request's records are the same served alone and in a concurrent
    mix of all env types, the configured BF16 shapes on their fused kernels
    included (the economy's work queue with drawn agent counts, the landscape's
    CTA-pair clusters over 4,096 Gaussians, the control and acrobot kernels)."""
    specs = [(W.WS_ENV_CONTROL, 5000, 150, 11, False), (W.WS_ENV_ECONOMY, 40, 100, 12, False),
             (W.WS_ENV_LANDSCAPE, 700, 100, 13, False), (W.WS_ENV_CONTROL, 70000, 200, 14, False),
             (W.WS_ENV_ACROBOT, 3000, 100, 15, False), (W.WS_ENV_ECONOMY, 300, 150, 16, True),
             (W.WS_ENV_LANDSCAPE, 1000, 100, 17, True)]
    dims = {W.WS_ENV_CONTROL: (4, 1), W.WS_ENV_ECONOMY: (16, 1), W.WS_ENV_LANDSCAPE: (24, 24),
            W.WS_ENV_ACROBOT: (6, 1)}
    alone = []
    srv = W.Server(8 * GB)
    for env, n, h, seed, fz in specs:
        q, keep = req(env, n, h, seed, fused=fz)
        st, rid = srv.submit(q)
        assert st == W.WS_OK
        alone.append(collect(srv, rid, slots_of(q), *dims[env], h // 50))
        srv.release(rid)
    srv.close()
    # all at once: their chunks run concurrently on separate streams
    srv = W.Server(8 * GB)
    ids = []
    for env, n, h, seed, fz in specs:
        q, keep = req(env, n, h, seed, fused=fz)
        st, rid = srv.submit(q)
        assert st == W.WS_OK
        ids.append((rid, q))
    mixed = [collect(srv, rid, slots_of(q), *dims[q.env], q.horizon // 50) for rid, q in ids]
    stats = srv.stats()
    srv.close()
    for (env, n, h, seed, fz), a, b in zip(specs, alone, mixed):
        assert a == b, (env, n, fz)
    assert stats["completed"] == len(specs)
    assert stats["chunks"] == sum(h // 50 for _, _, h, _, _ in specs)
    assert stats["p99_ms"] >= stats["p50_ms"] > 0


def test_admission_never_exceeds_budget(torch):
    q, _ = req(W.WS_ENV_CONTROL, 20000, 100, 1)
    cfg, _ = W.make_config(q.env, q.path, q.n_envs, 100, 200, 256, 256, param_seed=1)
    _, sb, rb, _ = W.ws_query_bytes(cfg)
    one = ((sb + 255) // 256 + (rb + 255) // 256) * 256
    srv = W.Server(int(2.5 * one))                      # room for two at a time
    ids = []
    for i in range(6):
        q, _ = req(W.WS_ENV_CONTROL, 20000, 100, 100 + i, flags=W.WS_REQ_CONSUME_ON_READY)
        st, rid = srv.submit(q)
        assert st == W.WS_OK
        ids.append(rid)
        st2 = srv.stats()
        assert st2["used_bytes"] <= st2["budget_bytes"]
    t0 = time.time()
    while srv.stats()["completed"] < 6:
        assert time.time() - t0 < 60
        time.sleep(0.01)
    st = srv.stats()
    assert st["peak_bytes"] <= st["budget_bytes"] and st["peak_bytes"] >= 2 * one
    assert st["used_bytes"] == 0
    big, _ = req(W.WS_ENV_CONTROL, 2_000_000, 100, 9)
    assert srv.submit(big)[0] == W.WS_ERR_NOMEM          # can never fit: rejected
    srv.close()


def test_release_frees_the_slot_and_wait_times_out(torch):
    q, _ = req(W.WS_ENV_CONTROL, 30000, 400, 3)
    cfg, _ = W.make_config(q.env, q.path, q.n_envs, 100, 200, 256, 256, param_seed=3)
    _, sb, rb, _ = W.ws_query_bytes(cfg)
    srv = W.Server(((sb + 255) // 256 + (rb + 255) // 256) * 256 + 4096)   # one at a time
    st, a = srv.submit(q)
    assert st == W.WS_OK
    assert srv.wait_chunk(a, 1, 30000) == W.WS_OK
    q2, _ = req(W.WS_ENV_CONTROL, 30000, 100, 4)
    st, b = srv.submit(q2)
    assert st == W.WS_OK
    # a holds its bytes (two chunks ahead of no acknowledgement): b cannot start
    assert srv.wait_chunk(b, 0, 200) == W.WS_ERR_TIMEOUT
    assert srv.stats()["pending"] == 1
    assert srv.release(a) == W.WS_OK                    # client gone: slot freed
    assert srv.wait_chunk(b, 0, 30000) == W.WS_OK
    assert srv.stats()["admitted"] == 2
    srv.close()
