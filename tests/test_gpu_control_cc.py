"""The CUDA-core classic-control kernels (ws_launch.ctrl_envs_per_cta != 0) for
small env counts: teacher-forced full-horizon replays against the FP64 oracle
(the 1,000-env control config on one thread per hidden unit, the 10,000-env
acrobot workload on register tiles), records byte-identical for every (envs
per CTA, threads per env) choice and chunk length, a roll-out that changes
kernel mid-run, and the launch-field checks."""
import numpy as np
import pytest

import oracle
from paper_2408_00930_gb300 import warpsci as W
from tests import classic_replay as CR
from tests import ws_helpers as H
from tests.gpu_common import TOL_BF16, control_rollout, need_gpu
from tests.test_gpu_acrobot import HEIGHT_BAND, TOL_STEP, acro
from tests.test_gpu_control import ORACLE_BF16_LAYERS

pytestmark = pytest.mark.gpu
BF16 = W.WS_PATH_BATCHED_BF16
FIELDS = (W.WS_F_OBS, W.WS_F_ACTION, W.WS_F_LOGP, W.WS_F_REWARD, W.WS_F_DONE,
          W.WS_F_POLICY_OUT)
# (envs per CTA, threads per env): register tiles (W2 in shared memory), then one
# thread per hidden unit (W2 columns in registers; hidden width 64 only)
TILED = [(4, 16), (8, 16), (8, 8), (16, 16), (16, 8), (16, 4), (32, 16), (32, 8), (32, 4)]
UNIT = [(1, 64), (2, 64), (4, 64), (8, 64)]


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


def test_cc_small_control_config_teacher_forced(torch):
    """1,000 envs x 200 steps, 4-64-64-2, chunks of 50, one thread per hidden
    unit and 4 envs per CTA: every step of every env replayed by the oracle from
    the recorded state."""
    n, T, h = 1000, 200, 64
    r = control_rollout(BF16, n, T, 200, h, h, seed=7, chunk_steps=50,
                        flags=W.WS_FLAG_DEBUG_LOGITS)
    r.set_launch(ctrl_envs_per_cta=4, ctrl_threads_per_env=64)
    r.reset(42)
    r.rollout(T)
    r.sync()
    ids = np.arange(n)
    rec = CR.records(r, 0, T, ids)
    s_fin, t_fin = H.unpack_control_state(r.fetch_raw(W.WS_F_STATE, 20 * n), n)
    np.testing.assert_array_equal(
        rec["obs"][0].T, np.array([oracle.control_reset_draw(42, oracle.STEP_INIT, e)
                                   for e in ids]).astype(np.float32))
    params = oracle.policy_init(7, 0, [4, h, h, 2])
    c = CR.replay("control", rec, ids, params, [4, h, h, 2], 42, 200, ORACLE_BF16_LAYERS,
                  TOL_BF16, s_fin, t_fin)
    print("replay", c)
    assert c["steps"] == n * T and c["dones"] > n
    assert c["tie"] <= 2e-4 * n * T and c["done_band"] <= 1e-3 * n * T, c
    r.close()


def test_cc_acrobot_workload_teacher_forced(torch):
    """The 10,000-env acrobot workload (6-64-64-3, 500 steps, chunks of 50) on 32
    envs per CTA: 256 envs (random ones, the ragged last CTA, env n - 1)
    replayed at every step."""
    n, T, limit, h = 10000, 500, 500, 64
    r = acro(BF16, n, T, limit, h=h, seed=1, chunk_steps=50, flags=W.WS_FLAG_DEBUG_LOGITS)
    r.set_launch(ctrl_envs_per_cta=32, ctrl_threads_per_env=4)
    r.reset(1000)
    for _ in range(T // 50):
        r.rollout(50)
    r.sync()
    g = np.random.default_rng(2)
    ids = np.unique(np.concatenate([g.choice(9984, 240, replace=False), np.arange(9984, n)]))
    assert len(ids) == 256 and ids[-1] == n - 1
    rec = CR.records(r, 0, T, ids)
    s_all, t_all = H.unpack_control_state(r.fetch_raw(W.WS_F_STATE, 20 * n), n)
    c = CR.replay("acrobot", rec, ids, oracle.policy_init(1, 0, [6, h, h, 3]), [6, h, h, 3], 1000,
                  limit, ORACLE_BF16_LAYERS, TOL_BF16, s_all[ids], t_all[ids], tol_state=TOL_STEP,
                  height_band=HEIGHT_BAND)
    print("replay", c)
    assert c["steps"] == len(ids) * T and c["dones"] > 0
    assert c["tie"] <= 2e-4 * len(ids) * T and c["done_band"] <= 1e-3 * len(ids) * T, c
    r.close()


@pytest.mark.parametrize("env,h", [("control", 64), ("control", 128), ("acrobot", 64),
                                   ("acrobot", 128)])
def test_cc_tiles_and_chunks_do_not_change_records(torch, env, h):
    n, T = 1001, 90            # a ragged last CTA for every tile size
    make = {"control": lambda ch: control_rollout(BF16, n, T, 60, h, h, seed=5, chunk_steps=ch,
                                                  flags=W.WS_FLAG_DEBUG_LOGITS),
            "acrobot": lambda ch: acro(BF16, n, T, 60, h=h, seed=5, chunk_steps=ch,
                                       flags=W.WS_FLAG_DEBUG_LOGITS)}[env]
    base = None
    for i, (ne, tpe) in enumerate(TILED + (UNIT if h == 64 else [])):
        r = make((40, 7, 90)[i % 3])
        r.set_launch(ctrl_envs_per_cta=ne, ctrl_threads_per_env=tpe)
        r.reset(3)
        r.rollout(T)
        r.sync()
        got = [r.fetch(f, 0, T).tobytes() for f in FIELDS]
        got.append(r.fetch_raw(W.WS_F_STATE, 20 * n).tobytes())
        assert r.fetch(W.WS_F_DONE, 0, T).sum() > 0
        r.close()
        if base is None:
            base = got
        assert got == base, (ne, tpe)


def test_cc_after_tensor_core_kernel_mid_run(torch):
    """60 steps on the tensor-core kernel, then 80 on the CUDA-core kernel, and
    the reverse: the env state hands over, and every step replays against the
    oracle."""
    n, T, h = 600, 140, 64
    params = oracle.policy_init(9, 0, [4, h, h, 2])
    for (first, tf), (second, ts) in (((0, 8), (16, 4)), ((2, 64), (0, 8))):
        r = control_rollout(BF16, n, T, 200, h, h, seed=9, chunk_steps=20,
                            flags=W.WS_FLAG_DEBUG_LOGITS)
        r.reset(77)
        r.set_launch(ctrl_envs_per_cta=first, ctrl_threads_per_env=tf)
        r.rollout(60)
        r.set_launch(ctrl_envs_per_cta=second, ctrl_threads_per_env=ts)
        r.rollout(T - 60)
        r.sync()
        ids = np.array([0, 1, 15, 16, 127, 128, 300, 598, 599])
        rec = CR.records(r, 0, T, ids)
        s_all, t_all = H.unpack_control_state(r.fetch_raw(W.WS_F_STATE, 20 * n), n)
        c = CR.replay("control", rec, ids, params, [4, h, h, 2], 77, 200, ORACLE_BF16_LAYERS,
                      TOL_BF16, s_all[ids], t_all[ids])
        assert c["steps"] == len(ids) * T and c["dones"] > 0, c
        r.close()


def test_cc_launch_fields_are_checked(torch):
    r = control_rollout(BF16, 500, 8, 200, 64, 64)
    for ne, tpe in ((3, 16), (64, 16), (4, 8), (8, 4), (16, 3), (16, 64), (3, 64)):
        with pytest.raises(W.WarpSciError):
            r.set_launch(ctrl_envs_per_cta=ne, ctrl_threads_per_env=tpe)
    r.set_launch(ctrl_envs_per_cta=16, ctrl_threads_per_env=8)
    assert r.launch().ctrl_envs_per_cta == 16
    r.close()
    # one thread per unit needs hidden width 64; width 256 has no CUDA-core kernel
    r = control_rollout(BF16, 500, 8, 200, 128, 128)
    with pytest.raises(W.WarpSciError):
        r.set_launch(ctrl_envs_per_cta=4, ctrl_threads_per_env=64)
    r.close()
    r = control_rollout(BF16, 500, 8, 200, 256, 256)
    with pytest.raises(W.WarpSciError):
        r.set_launch(ctrl_envs_per_cta=16, ctrl_threads_per_env=8)
    r.close()
    # other envs ignore the fields (in range)
    r = W.Rollout(W.WS_ENV_ECONOMY, BF16, 40, 8, 540, 128, 128, param_seed=1)
    r.set_launch(ctrl_envs_per_cta=16, ctrl_threads_per_env=8)
    r.rollout(8)
    r.sync()
    r.close()


def test_tune_offers_the_cuda_core_kernel_for_small_counts(torch):
    n, T, h = 1000, 60, 64
    r = control_rollout(BF16, n, T, 200, h, h, seed=4)
    chosen, ms = r.tune(20)
    assert ms > 0 and r.k == 0
    if chosen["ctrl_envs_per_cta"]:
        assert (chosen["ctrl_envs_per_cta"], chosen["ctrl_threads_per_env"]) in TILED + UNIT
    r.rollout(T)
    r.sync()
    r.close()
