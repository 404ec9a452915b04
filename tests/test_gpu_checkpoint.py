"""Checkpoint and resume on the fused tensor-core kernels of every env (paper
Sec. 3 lists checkpointing among the framework's services).  A context runs 30
steps in chunks of 20 (so the checkpoint falls inside a chunk's launch
sequence), its parameters, env parameters and state are fetched with the step
counter, and it runs 40 more.  A fresh context created under another parameter
seed loads the checkpoint and runs the same 40 steps: every ring field and the
final state agree byte for byte with the uninterrupted run, and the resumed
segment is replayed step by step by the oracle from the checkpointed state."""
import numpy as np
import pytest

import oracle
from paper_2408_00930_gb300 import warpsci as W
from tests import classic_replay as CR
from tests import test_gpu_econ_fused as ECON
from tests import test_gpu_land_fused as LAND
from tests import ws_helpers as H
from tests.gpu_common import TOL_BF16, need_gpu

pytestmark = pytest.mark.gpu
BF16 = W.WS_PATH_BATCHED_BF16
K0, T2, CHUNK, LIMIT, RS = 30, 40, 20, 25, 77


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


def _state_bytes(env, n, n_slots, kw):
    if env in (W.WS_ENV_CONTROL, W.WS_ENV_ACROBOT):
        return 20 * n
    if env == W.WS_ENV_LANDSCAPE:
        return (4 * kw["dim"] + 8) * n
    return 72 * (n_slots - n) + 4 * n


def _param_bytes(env, h, kw):
    if env == W.WS_ENV_CONTROL:
        return 4 * oracle.policy_param_count([4, h, h, 2])
    if env == W.WS_ENV_ACROBOT:
        return 4 * oracle.policy_param_count([6, h, h, 3])
    if env == W.WS_ENV_LANDSCAPE:
        return 4 * oracle.policy_param_count([kw["dim"], h, h, 2 * kw["dim"]])
    return 4 * (oracle.policy_param_count([16, h, h, 20]) + oracle.policy_param_count([16, h, h, 10]))


CASES = [
    ("control", W.WS_ENV_CONTROL, 300, 256, {}),
    ("acrobot", W.WS_ENV_ACROBOT, 200, 64, {}),
    ("economy", W.WS_ENV_ECONOMY, 24, 128, {}),
    ("landscape", W.WS_ENV_LANDSCAPE, 130, 256, dict(dim=24, n_gauss=4096)),
]


@pytest.mark.parametrize("name,env,n,h,kw", CASES, ids=[c[0] for c in CASES])
def test_checkpoint_resume_fused(torch, name, env, n, h, kw):
    fl = W.WS_FLAG_DEBUG_LOGITS
    a = W.Rollout(env, BF16, n, K0 + T2, LIMIT, h, h, param_seed=5, chunk_steps=CHUNK, flags=fl,
                  **kw)
    if env == W.WS_ENV_LANDSCAPE:
        a.set_launch(tile_ctas=2)
    a.reset(RS)
    a.rollout(K0)
    a.sync()
    sb = _state_bytes(env, n, a.n_slots, kw)
    ck_state = a.fetch_raw(W.WS_F_STATE, sb).copy()
    ck_par = a.fetch_raw(W.WS_F_PARAMS, _param_bytes(env, h, kw)).copy()
    ck_env = None
    if env == W.WS_ENV_LANDSCAPE:
        M, D = kw["n_gauss"], kw["dim"]
        ck_env = a.fetch_raw(W.WS_F_ENV_PARAMS, 4 * (M * D + 2 * M)).copy()
    counts = None
    if env == W.WS_ENV_ECONOMY:
        counts = a.fetch_raw(W.WS_F_ENV_PARAMS, 4 * n).view(np.int32).copy()
    a.rollout(T2)
    a.sync()
    rec_a = {f: a.fetch(f, K0, T2) for f in _fields(env)}
    fin_a = a.fetch_raw(W.WS_F_STATE, sb)
    # a fresh context under another parameter seed takes everything from the checkpoint
    b = W.Rollout(env, BF16, n, K0 + T2, LIMIT, h, h, param_seed=999, chunk_steps=CHUNK, flags=fl,
                  agents_per_env=counts, **kw)
    if env == W.WS_ENV_LANDSCAPE:
        b.set_launch(tile_ctas=2)
    b.reset(RS)
    b.load_raw(W.WS_F_PARAMS, ck_par)
    if ck_env is not None:
        b.load_raw(W.WS_F_ENV_PARAMS, ck_env)
    b.load_raw(W.WS_F_STATE, ck_state, k=K0)
    b.rollout(T2)
    b.sync()
    rec_b = {f: b.fetch(f, K0, T2) for f in _fields(env)}
    fin_b = b.fetch_raw(W.WS_F_STATE, sb)
    for f in rec_a:
        assert rec_a[f].tobytes() == rec_b[f].tobytes(), (name, f)
    assert fin_a.tobytes() == fin_b.tobytes()
    assert rec_b[W.WS_F_DONE].sum() > 0             # episodes end inside the resumed segment
    # the resumed segment against the oracle, from the checkpointed state
    par = ck_par.view(np.float32)
    if env in (W.WS_ENV_CONTROL, W.WS_ENV_ACROBOT):
        s0, t0 = H.unpack_control_state(ck_state, n)
        s1, t1 = H.unpack_control_state(fin_b, n)
        ids = np.array([0, 1, 127, 128, n - 2, n - 1])
        rec = {k: v[..., ids] for k, v in zip(
            ["obs", "action", "logp", "reward", "done", "pout"],
            [rec_b[f] for f in _fields(env)[:6]])}
        if env == W.WS_ENV_CONTROL:
            c = CR.replay("control", rec, ids, par, [4, h, h, 2], RS, LIMIT, 0b010, TOL_BF16,
                          s1[ids], t1[ids], k0=K0, t_init=t0[ids])
            np.testing.assert_array_equal(rec["obs"][0].T, s0[ids])
        else:
            c = CR.replay("acrobot", rec, ids, par, [6, h, h, 3], RS, LIMIT, 0b010, TOL_BF16,
                          s1[ids], t1[ids], k0=K0, t_init=t0[ids], tol_state=3e-5)
        assert c["steps"] == len(ids) * T2
    elif env == W.WS_ENV_ECONOMY:
        sa = a.n_slots - n
        _, _, t0 = H.unpack_econ_state(ck_state, sa, n)
        out = {k: rec_b[f] for k, f in [("obs", W.WS_F_OBS), ("action", W.WS_F_ACTION),
                                        ("logp", W.WS_F_LOGP), ("reward", W.WS_F_REWARD),
                                        ("done", W.WS_F_DONE), ("wealth", W.WS_F_WEALTH)]}
        envs = np.array([0, 7, n - 1])
        checked = ECON._replay_records(out, t0, counts, envs, par, T2, LIMIT, RS, k0=K0)
        assert checked >= len(envs) * T2 // 2
    else:
        M, D = kw["n_gauss"], kw["dim"]
        envp = ck_env.view(np.float32)
        cwa = (envp[:M * D].reshape(M, D).astype(np.float64), envp[M * D:M * D + M].astype(np.float64),
               envp[M * D + M:].astype(np.float64))
        init = H.unpack_landscape_state(ck_state, n, D)
        rec = {f: rec_b[f] for f in LAND.FIELDS}
        LAND._teacher_forced(rec, init, par, cwa, [0, 1, 128, n - 1], T2, LIMIT, RS, k0=K0)
        np.testing.assert_array_equal(rec_b[W.WS_F_OBS][0].T, init[0].astype(np.float32))
    a.close()
    b.close()
