"""GPU parity of the acrobot env (App. C classic control; all paths) against
the FP64 oracle: parameter and reset draws bit-exact, one-step replays of
seeded states, and long roll-outs checked step by step against oracle steps
taken from the GPU's own recorded states (teacher forcing: the dynamics are
chaotic, so free-running FP32 and FP64 trajectories part after a while).  The
BF16 path is the fused classic-control kernel (layer 2 in BF16, layers 1 and 3
at FP32 accuracy), compared with the oracle in that operand mode."""
import numpy as np
import pytest

import oracle
from paper_2408_00930_gb300 import inputs
from paper_2408_00930_gb300 import warpsci as W
from tests import classic_replay as CR
from tests import ws_helpers as H
from tests.gpu_common import TIE_BF16, TIE_F32, TOL_BF16, TOL_F32, need_gpu

pytestmark = pytest.mark.gpu
PATHS = [W.WS_PATH_PLAIN_FP32, W.WS_PATH_BATCHED_FP32, W.WS_PATH_BATCHED_BF16]
# FP32 RK4 with FP32 sin/cos against FP64: per-step error of the state relative
# to the largest magnitude the step passes through (the unclipped RK4 result;
# at |w| ~ 40 rad/s the w^2 terms put FP32 rounding near 1e-5 of it)
TOL_STEP = 3e-5
# the tip-height threshold of the terminal condition
HEIGHT_BAND = 1e-4
# the fused kernel's precision: layer 2 with BF16 operands (and BF16 tanh of h1)
ORACLE_BF16_LAYERS = 0b010


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


def acro(path, n, ring, limit, h=64, seed=1, **kw):
    return W.Rollout(W.WS_ENV_ACROBOT, path, n, ring, limit, h, h, param_seed=seed, **kw)


def test_param_init_and_reset_bit_exact(torch):
    n = 333
    r = acro(W.WS_PATH_PLAIN_FP32, n, 4, 500, h=48, seed=17)
    got = r.fetch_raw(W.WS_F_PARAMS, 4 * oracle.policy_param_count([6, 48, 48, 3])).view(np.float32)
    np.testing.assert_array_equal(got, oracle.policy_init(17, 0, [6, 48, 48, 3]))
    r.reset(55)
    s, t = H.unpack_control_state(r.fetch_raw(W.WS_F_STATE, 20 * n), n)
    exp = np.array([oracle.acrobot_reset_draw(55, oracle.STEP_INIT, e) for e in range(n)])
    np.testing.assert_array_equal(s, exp)
    assert np.all(t == 0)
    r.close()


@pytest.mark.parametrize("path", PATHS)
def test_one_step_replay_seeded_states(torch, path):
    n, h = 1500, 64
    g = inputs.rng(21)
    params = inputs.policy_params(g, [6, h, h, 3], scale=2.0)
    s0 = np.stack([g.uniform(-np.pi, np.pi, n), g.uniform(-np.pi, np.pi, n),
                   g.uniform(-12, 12, n), g.uniform(-27, 27, n)], 1).astype(np.float32)
    s0[:20, 2:] = [14.0, -30.0]                    # beyond the velocity clips
    s0[20:40, 0] = np.float32(2.9)                  # near upright: terminal heights
    t0 = g.integers(0, 400, n).astype(np.int32)
    t0[40:60] = 499                                 # the episode limit
    r = acro(path, n, 8, 500, h=h)
    r.load_raw(W.WS_F_PARAMS, params)
    k0 = 77
    r.load_raw(W.WS_F_STATE, H.pack_control_state(s0, t0), k=k0)
    r.step()
    r.sync()
    obs = r.fetch(W.WS_F_OBS, k0, 1)[0]
    act, lp, rew, dn = (r.fetch(f, k0, 1)[0] for f in (W.WS_F_ACTION, W.WS_F_LOGP,
                                                       W.WS_F_REWARD, W.WS_F_DONE))
    s1, t1 = H.unpack_control_state(r.fetch_raw(W.WS_F_STATE, 20 * n), n)
    bf16 = path == W.WS_PATH_BATCHED_BF16
    tie = TIE_BF16 if bf16 else TIE_F32
    s0d = s0.astype(np.float64)
    n_amb = 0
    for e in range(n):
        o_ref = oracle.acrobot_obs(s0d[e])
        np.testing.assert_allclose(obs[:, e], o_ref, rtol=0, atol=2e-6)
        logits = oracle.mlp_forward([6, h, h, 3], params, obs[:, e].astype(np.float64),
                                    bf16_layers=ORACLE_BF16_LAYERS if bf16 else 0)
        u = oracle.u01(int(oracle.draw(1, k0, e, 0, oracle.TAG_ACTION, 0)[0]))
        a_o, lp_o, mg = oracle.sample_categorical(logits, u)
        if mg < tie:
            n_amb += 1
            continue
        assert act[e] == a_o, e
        assert abs(lp[e] - lp_o) <= (TOL_BF16 if bf16 else TOL_F32) * max(1.0, abs(lp_o))
        nxt, raw = oracle.acrobot_step(s0d[e], a_o)
        term, hm = oracle.acrobot_terminal(nxt)
        if hm < HEIGHT_BAND:
            n_amb += 1
            continue
        done = term or t0[e] + 1 >= 500
        assert dn[e] == done and rew[e] == (0.0 if term else -1.0), e
        if done:
            np.testing.assert_array_equal(s1[e], oracle.acrobot_reset_draw(1, k0, e))
            assert t1[e] == 0
        else:
            d = s1[e] - nxt
            d[:2] = (d[:2] + np.pi) % (2 * np.pi) - np.pi      # angles modulo 2 pi
            assert np.abs(d).max() <= TOL_STEP * max(1.0, np.abs(raw).max()), (e, d)
            assert t1[e] == t0[e] + 1
    assert n_amb <= (0.12 * n if bf16 else 10) and dn[20:40].sum() > 0 and dn[40:60].all()
    r.close()


@pytest.mark.parametrize("path", PATHS)
def test_long_rollout_teacher_forced(torch, path):
    """2,000 envs x 300 steps from a reset, episodes ending inside and across
    chunks: every transition of sampled envs against the oracle's step from the
    recorded pre-step state, the draw against the path's own recorded logits."""
    n, T, limit, h = 2000, 300, 200, 64
    r = acro(path, n, T, limit, h=h, seed=3, chunk_steps=40, flags=W.WS_FLAG_DEBUG_LOGITS)
    r.reset(8)
    r.rollout(T)
    r.sync()
    ids = np.array([0, 1, 2, 127, 128, 999, 1920, 1998, 1999])
    rec = CR.records(r, 0, T, ids)
    s_all, t_all = H.unpack_control_state(r.fetch_raw(W.WS_F_STATE, 20 * n), n)
    np.testing.assert_allclose(
        [CR.acrobot_state_from_obs(rec["obs"][0][:, i].astype(np.float64)) for i in range(len(ids))],
        [oracle.acrobot_reset_draw(8, oracle.STEP_INIT, e) for e in ids], rtol=0, atol=2e-6)
    bf16 = path == W.WS_PATH_BATCHED_BF16
    c = CR.replay("acrobot", rec, ids, oracle.policy_init(3, 0, [6, h, h, 3]), [6, h, h, 3], 8,
                  limit, ORACLE_BF16_LAYERS if bf16 else 0, TOL_BF16 if bf16 else TOL_F32,
                  s_all[ids], t_all[ids], tol_state=TOL_STEP, height_band=HEIGHT_BAND)
    print("replay", c)
    assert c["steps"] == len(ids) * T and c["dones"] >= len(ids)
    assert c["tie"] <= 2 and c["done_band"] <= 2, c
    r.close()


def test_bf16_bench_workload_teacher_forced(torch):
    """The acrobot bench workload on the fused kernel: 10,000 envs x 500 steps,
    6-64-64-3, chunks of 50.  256 envs (random ones, the ragged last tile,
    env n - 1) replayed by the oracle at every step from the recorded state."""
    n, T, limit, h = 10000, 500, 500, 64
    r = acro(W.WS_PATH_BATCHED_BF16, n, T, limit, h=h, seed=1, chunk_steps=50,
             flags=W.WS_FLAG_DEBUG_LOGITS)
    r.reset(1000)
    for _ in range(T // 50):
        r.rollout(50)
    r.sync()
    g = np.random.default_rng(1)
    ids = np.unique(np.concatenate([g.choice(9984, 240, replace=False), np.arange(9984, n)]))
    assert len(ids) == 256 and ids[-1] == n - 1
    rec = CR.records(r, 0, T, ids)
    s_all, t_all = H.unpack_control_state(r.fetch_raw(W.WS_F_STATE, 20 * n), n)
    c = CR.replay("acrobot", rec, ids, oracle.policy_init(1, 0, [6, h, h, 3]), [6, h, h, 3], 1000,
                  limit, ORACLE_BF16_LAYERS, TOL_BF16, s_all[ids], t_all[ids], tol_state=TOL_STEP,
                  height_band=HEIGHT_BAND)
    print("replay", c)
    assert c["steps"] == len(ids) * T
    assert c["tie"] <= 2e-4 * len(ids) * T and c["done_band"] <= 1e-3 * len(ids) * T, c
    r.close()


def test_graph_path_bytes_equal_plain_path(torch):
    out = []
    for path in (W.WS_PATH_PLAIN_FP32, W.WS_PATH_BATCHED_FP32):
        r = acro(path, 300, 30, 25, h=32, seed=4, chunk_steps=7)
        r.rollout(30)
        out.append([r.fetch(f, 0, 30).tobytes() for f in (W.WS_F_OBS, W.WS_F_ACTION, W.WS_F_LOGP,
                                                          W.WS_F_REWARD, W.WS_F_DONE)])
        r.close()
    assert out[0] == out[1]


def test_bf16_fused_deterministic_and_chunk_invariant(torch):
    out = []
    for ch in (40, 7, 40):
        r = acro(W.WS_PATH_BATCHED_BF16, 700, 90, 60, h=128, seed=5, chunk_steps=ch)
        r.reset(2)
        r.rollout(90)
        r.sync()
        out.append([r.fetch(f, 0, 90).tobytes() for f in (W.WS_F_OBS, W.WS_F_ACTION, W.WS_F_LOGP,
                                                          W.WS_F_REWARD, W.WS_F_DONE)])
        r.close()
    assert out[0] == out[1] == out[2]
