"""Expiry of the fused kernels' bounded device waits, made to happen without any
fault: the launch field wait_ns caps every device wait (an MMA's completion,
a block load, the cluster partner) at 1 ns, far below an MMA's completion
time, so the waits run out in the first step.  Each kernel must then drain its
own MMAs and copies, free its tensor memory and leave; ws_sync reports a sticky
WS_ERR_TIMEOUT naming the wait's site, and a fresh context on the same device
runs clean afterwards (its records equal those of a second fresh context)."""
import numpy as np
import pytest

from paper_2408_00930_gb300 import warpsci as W
from tests.gpu_common import need_gpu

pytestmark = pytest.mark.gpu
BF16 = W.WS_PATH_BATCHED_BF16

# name, env, n_envs, hidden, extra config, launch fields, error sites of the kernel
CASES = [
    ("control", W.WS_ENV_CONTROL, 300, 256, {}, {}, range(101, 110)),
    ("acrobot", W.WS_ENV_ACROBOT, 300, 64, {}, {}, range(101, 110)),
    ("economy", W.WS_ENV_ECONOMY, 24, 128, {}, {}, range(300, 310)),
    ("landscape-cta", W.WS_ENV_LANDSCAPE, 130, 256, dict(dim=24, n_gauss=1024),
     dict(tile_ctas=1), (500, 501)),
    ("landscape-pair", W.WS_ENV_LANDSCAPE, 130, 256, dict(dim=24, n_gauss=1024),
     dict(tile_ctas=2), (500, 501)),
]


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


def _ctx(env, n, h, kw, launch, wait_ns=0):
    r = W.Rollout(env, BF16, n, 40, 15, h, h, param_seed=3, chunk_steps=10, **kw)
    r.set_launch(wait_ns=wait_ns, **launch)
    r.reset(8)
    return r


@pytest.mark.parametrize("name,env,n,h,kw,launch,sites", CASES, ids=[c[0] for c in CASES])
def test_device_wait_expiry_is_reported_and_recovered(torch, name, env, n, h, kw, launch, sites):
    r = _ctx(env, n, h, kw, launch, wait_ns=1)
    assert W.ws_rollout(r.ctx, 20) == W.WS_OK              # enqueued; the waits run out on the GPU
    st = W.ws_sync(r.ctx, 120000)
    msg = W.ws_last_error(r.ctx)
    assert st == W.WS_ERR_TIMEOUT and "device wait ran out" in msg, (st, msg)
    site = int(msg.split("site")[1].strip(" )"))
    assert site in sites, msg
    assert W.ws_rollout(r.ctx, 1) == W.WS_ERR_TIMEOUT       # sticky
    r.close()
    # the device is usable: two fresh contexts (default limit) agree byte for byte
    outs = []
    for _ in range(2):
        c = _ctx(env, n, h, kw, launch)
        c.rollout(20)
        c.sync()
        outs.append([c.fetch(f, 0, 20).tobytes() for f in (W.WS_F_OBS, W.WS_F_ACTION,
                                                           W.WS_F_LOGP, W.WS_F_DONE)])
        assert c.fetch(W.WS_F_DONE, 0, 20).sum() > 0         # episodes end and reset
        c.close()
    assert outs[0] == outs[1]
    torch.cuda.synchronize()
