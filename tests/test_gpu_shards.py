"""Env sharding (paper Sec. 2: the workflow runs on one GPU or several): a
context over global env ids [b, b + n) (ws_config.env_base = b) records exactly
what one context over all envs records for those envs.  Two shard contexts over
[0, n) and [n, 2 n) against one context over [0, 2 n), on one GPU: every ring
field and the final state byte for byte, on the fused tensor-core kernels of
every env and on the per-step FP32 paths.  Several GPUs would each hold one such
shard; nothing on the data path is exchanged."""
import numpy as np
import pytest

from paper_2408_00930_gb300 import warpsci as W
from tests import ws_helpers as H
from tests.gpu_common import need_gpu

pytestmark = pytest.mark.gpu
F32, BF16 = W.WS_PATH_BATCHED_FP32, W.WS_PATH_BATCHED_BF16

CASES = [
    ("control-bf16", W.WS_ENV_CONTROL, BF16, 300, 256, {}),
    ("control-f32", W.WS_ENV_CONTROL, F32, 300, 64, {}),
    ("acrobot-bf16", W.WS_ENV_ACROBOT, BF16, 200, 64, {}),
    ("economy-bf16", W.WS_ENV_ECONOMY, BF16, 24, 128, {}),
    ("economy-f32", W.WS_ENV_ECONOMY, F32, 12, 128, {}),
    ("landscape-bf16", W.WS_ENV_LANDSCAPE, BF16, 130, 256, dict(dim=24, n_gauss=1024)),
    ("landscape-f32", W.WS_ENV_LANDSCAPE, F32, 70, 32, dict(dim=8, n_gauss=256)),
]


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


def _fields(env):
    f = [W.WS_F_OBS, W.WS_F_ACTION, W.WS_F_LOGP, W.WS_F_REWARD, W.WS_F_DONE, W.WS_F_POLICY_OUT]
    if env == W.WS_ENV_ECONOMY:
        f.append(W.WS_F_WEALTH)
    if env == W.WS_ENV_LANDSCAPE:
        f.append(W.WS_F_ENERGY)
    return f


def _run(env, path, n, base, h, kw, T, limit):
    r = W.Rollout(env, path, n, T, limit, h, h, param_seed=9, env_base=base, chunk_steps=20,
                  flags=W.WS_FLAG_DEBUG_LOGITS, **kw)
    if env == W.WS_ENV_LANDSCAPE and path == BF16:
        r.set_launch(tile_ctas=2)       # the same Gaussian split in every context
    r.reset(31)
    r.rollout(T)
    r.sync()
    rec = {f: r.fetch(f, 0, T) for f in _fields(env)}
    return r, rec


def _state(r, env, n, kw):
    if env in (W.WS_ENV_CONTROL, W.WS_ENV_ACROBOT):
        s, t = H.unpack_control_state(r.fetch_raw(W.WS_F_STATE, 20 * n), n)
        return [s, t]
    if env == W.WS_ENV_LANDSCAPE:
        D = kw["dim"]
        return list(H.unpack_landscape_state(r.fetch_raw(W.WS_F_STATE, (4 * D + 8) * n), n, D))
    sa = r.n_slots - n
    return list(H.unpack_econ_state(r.fetch_raw(W.WS_F_STATE, 72 * sa + 4 * n), sa, n))


@pytest.mark.parametrize("name,env,path,n,h,kw", CASES, ids=[c[0] for c in CASES])
def test_two_shards_equal_one_context(torch, name, env, path, n, h, kw):
    T, limit = 50, 23                   # episodes end and reset inside the window
    whole, rw = _run(env, path, 2 * n, 0, h, kw, T, limit)
    parts = [_run(env, path, n, b, h, kw, T, limit) for b in (0, n)]
    sw = _state(whole, env, 2 * n, kw)
    if env == W.WS_ENV_ECONOMY:
        # slots: agents env by env, then one planner per env
        sa = [p.n_slots - n for p, _ in parts]
        assert whole.n_slots == sum(p.n_slots for p, _ in parts)
        cols = [np.r_[0:sa[0], sum(sa):sum(sa) + n],
                np.r_[sa[0]:sum(sa), sum(sa) + n:sum(sa) + 2 * n]]
        agent_cols = [np.r_[0:sa[0]], np.r_[sa[0]:sum(sa)]]
    else:
        cols = [np.r_[0:n], np.r_[n:2 * n]]
    for i, (p, rp) in enumerate(parts):
        for f, v in rp.items():
            assert np.array_equal(rw[f][..., cols[i]], v), (name, i, f)
        sp = _state(p, env, n, kw)
        if env == W.WS_ENV_ECONOMY:
            assert np.array_equal(sw[0][agent_cols[i]], sp[0])          # wealth
            assert np.array_equal(sw[1][agent_cols[i]], sp[1])          # features
            assert np.array_equal(sw[2][i * n:(i + 1) * n], sp[2])      # episode counters
        else:
            for a, b in zip(sw, sp):
                assert np.array_equal(a[i * n:(i + 1) * n], b), (name, i)
        p.close()
    assert rw[W.WS_F_DONE].sum() > 0
    whole.close()
