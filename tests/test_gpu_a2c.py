"""GPU parity of the actor-critic update (ws_a2c_update) against the oracle's
FP64 loss and gradients (pinned to finite differences and autograd): the
update's parameter change over lr is the gradient of the mean loss over the
ring's recorded rows, for the control env, the acrobot (categorical heads) and
the landscape (diagonal Gaussian head), on the FP32 and the BF16 paths; a
roll-out after the update runs on the new parameters."""
import numpy as np
import pytest

import oracle
from paper_2408_00930_gb300 import warpsci as W
from tests.gpu_common import TIE_BF16, need_gpu

pytestmark = pytest.mark.gpu
F32, BF16 = W.WS_PATH_BATCHED_FP32, W.WS_PATH_BATCHED_BF16


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


def run_update(env, path, n, T, h, lr, c_v, c_e, seed=3, gemm=0):
    od, na = (4, 2) if env == W.WS_ENV_CONTROL else (6, 3)
    r = W.Rollout(env, path, n, T, 25, h, h, param_seed=seed, flags=W.WS_FLAG_TRAIN, chunk_steps=10)
    r.set_launch(update_gemm=gemm)
    r.reset(seed + 1)
    r.rollout(T)
    pa = r.fetch_raw(W.WS_F_PARAMS, 4 * oracle.policy_param_count([od, h, h, na])).view(np.float32).copy()
    pc = r.fetch_raw(W.WS_F_CRITIC, 4 * oracle.policy_param_count([od, h, h, 1])).view(np.float32).copy()
    obs = r.fetch(W.WS_F_OBS, 0, T)                      # [T][od][n]
    act = r.fetch(W.WS_F_ACTION, 0, T)
    rew, done = r.fetch(W.WS_F_REWARD, 0, T), r.fetch(W.WS_F_DONE, 0, T)
    stats = r.a2c_update(T, lr, c_v, c_e)
    ret = r.fetch(W.WS_F_RETURN, 0, T)
    pa2 = r.fetch_raw(W.WS_F_PARAMS, pa.nbytes).view(np.float32).copy()
    pc2 = r.fetch_raw(W.WS_F_CRITIC, pc.nbytes).view(np.float32).copy()
    rows = dict(obs=obs.transpose(0, 2, 1).reshape(-1, od).astype(np.float64),
                act=act.reshape(-1), ret=ret.reshape(-1).astype(np.float64))
    # the update's own returns scan (pinned elsewhere) against the oracle's
    Go = oracle.returns(rew, done, float(np.float32(0.99)))
    assert np.abs(ret - Go).max() <= 1e-6 * max(1.0, np.abs(Go).max())
    return r, (pa, pc, pa2, pc2), rows, stats, (od, na)


def check_grads(params, rows, stats, shape, h, lr, c_v, c_e):
    pa, pc, pa2, pc2 = params
    od, na = shape
    st, ga, gc = oracle.a2c(pa, pc, rows["obs"], rows["act"], rows["ret"], h, h, na, c_v=c_v, c_e=c_e)
    np.testing.assert_allclose(stats, st, rtol=1e-4, atol=1e-7)
    for before, after, g in ((pa, pa2, ga), (pc, pc2, gc)):
        step = (before.astype(np.float64) - after.astype(np.float64)) / lr
        # after = fl(before - lr g): the subtraction loses up to half an ulp of the parameter
        tol = 1e-4 * np.abs(g).max() + 0.6 * np.spacing(np.abs(before)).astype(np.float64) / lr
        assert np.all(np.abs(step - g) <= tol), np.abs(step - g).max()
        assert np.abs(g).max() > 0


@pytest.mark.parametrize("env,gemm", [(W.WS_ENV_CONTROL, 0), (W.WS_ENV_ACROBOT, 0),
                                      (W.WS_ENV_CONTROL, 1), (W.WS_ENV_ACROBOT, 1)])
def test_a2c_update_matches_oracle_fp32(torch, env, gemm):
    """gemm 0: the hidden GEMMs on tcgen05 (FP32 operands split into BF16 hi +
    lo); 1: on the FP32 CUDA cores."""
    n, T, h, lr, c_v, c_e = 3000, 30, 64, 1.0, 0.5, 0.01  # 90,000 rows: two update chunks
    r, params, rows, stats, shape = run_update(env, F32, n, T, h, lr, c_v, c_e, gemm=gemm)
    check_grads(params, rows, stats, shape, h, lr, c_v, c_e)
    r.close()


def test_a2c_update_wide_layers_on_tensor_cores(torch):
    """256-unit hidden layers (128 x 128 tiles with two N tiles per layer) over
    two chunks, the second ragged: the split-BF16 tcgen05 GEMMs against the
    oracle's FP64 gradients."""
    n, T, h, lr, c_v, c_e = 2100, 40, 256, 1.0, 0.5, 0.01  # 84,000 rows
    r, params, rows, stats, shape = run_update(W.WS_ENV_CONTROL, BF16, n, T, h, lr, c_v, c_e,
                                               seed=11)
    check_grads(params, rows, stats, shape, h, lr, c_v, c_e)
    r.close()


@pytest.mark.parametrize("h", [150, 200])
def test_a2c_update_ragged_wide_tile(torch, h):
    """Hidden widths between 128 and 256: a second, ragged 128-column tile
    whose columns past the width are masked, with rows whose length is a
    multiple of 4 (16-byte loads and stores) and one that is not (element
    loads and stores)."""
    n, T, lr, c_v, c_e = 1300, 20, 1.0, 0.5, 0.01  # 26,000 rows
    r, params, rows, stats, shape = run_update(W.WS_ENV_CONTROL, F32, n, T, h, lr, c_v, c_e, seed=5)
    check_grads(params, rows, stats, shape, h, lr, c_v, c_e)
    r.close()


def test_a2c_update_bf16_acrobot_and_next_rollout(torch):
    n, T, h, lr, c_v, c_e = 257, 20, 64, 0.5, 0.5, 0.0
    r, params, rows, stats, shape = run_update(W.WS_ENV_ACROBOT, BF16, n, T, h, lr, c_v, c_e, seed=8)
    check_grads(params, rows, stats, shape, h, lr, c_v, c_e)
    # the next step's draws follow the updated policy (BF16 images repacked)
    k = r.k
    r.step()
    r.sync()
    obs = r.fetch(W.WS_F_OBS, k, 1)[0].T.astype(np.float64)
    act = r.fetch(W.WS_F_ACTION, k, 1)[0]
    pa2 = params[2]
    n_ok = 0
    for e in range(n):
        lg = oracle.mlp_forward([6, h, h, 3], pa2, obs[e], bf16_layers=0b010)
        u = oracle.u01(int(oracle.draw(9, k, e, 0, oracle.TAG_ACTION, 0)[0]))
        a_o, _, mg = oracle.sample_categorical(lg, u)
        if mg >= TIE_BF16:
            assert act[e] == a_o, e
            n_ok += 1
    assert n_ok > 0.8 * n
    r.close()


def test_a2c_errors(torch):
    r = W.Rollout(W.WS_ENV_CONTROL, F32, 16, 4, 100, 16, 16)
    r.rollout(2)
    assert W.ws_a2c_update(r.ctx, 2, 0.1, 0.5, 0.0) == W.WS_ERR_STATE      # no WS_FLAG_TRAIN
    r.close()
    r = W.Rollout(W.WS_ENV_CONTROL, F32, 16, 4, 100, 16, 16, flags=W.WS_FLAG_TRAIN)
    r.rollout(2)
    assert W.ws_a2c_update(r.ctx, 3, 0.1, 0.5, 0.0) == W.WS_ERR_RANGE
    assert W.ws_a2c_update(r.ctx, 2, float("nan"), 0.5, 0.0) == W.WS_ERR_INVALID
    assert W.ws_a2c_update(r.ctx, 2, 0.1, 0.5, 0.0) == W.WS_OK
    r.sync()
    r.close()
    cfg, _ = W.make_config(W.WS_ENV_CONTROL, F32, 8, 4, 10, 16, 16, flags=W.WS_FLAG_TRAIN | 64)
    assert W.ws_query_bytes(cfg)[0] == W.WS_ERR_INVALID                    # unknown flag


@pytest.mark.parametrize("path", [F32, BF16])
def test_a2c_update_landscape_gaussian_head(torch, path):
    D, M, n, T, h, lr, c_v, c_e = 8, 64, 200, 12, 256, 1.0, 0.5, 0.01
    if path == F32:
        h = 32
    r = W.Rollout(W.WS_ENV_LANDSCAPE, path, n, T, 7, h, h, dim=D, n_gauss=M, param_seed=4,
                  flags=W.WS_FLAG_TRAIN, chunk_steps=5)
    r.reset(6)
    r.rollout(T)
    na = oracle.policy_param_count([D, h, h, 2 * D])
    nc = oracle.policy_param_count([D, h, h, 1])
    pa = r.fetch_raw(W.WS_F_PARAMS, 4 * na).view(np.float32).copy()
    pc = r.fetch_raw(W.WS_F_CRITIC, 4 * nc).view(np.float32).copy()
    obs = r.fetch(W.WS_F_OBS, 0, T)
    stats = r.a2c_update(T, lr, c_v, c_e)
    ret = r.fetch(W.WS_F_RETURN, 0, T)
    pa2 = r.fetch_raw(W.WS_F_PARAMS, 4 * na).view(np.float32).copy()
    pc2 = r.fetch_raw(W.WS_F_CRITIC, 4 * nc).view(np.float32).copy()
    X = obs.transpose(0, 2, 1).reshape(-1, D).astype(np.float64)
    Z = np.array([oracle.landscape_action_normals(6, t, e, D) for t in range(T) for e in range(n)])
    st, ga, gc = oracle.a2c_gauss(pa, pc, X, Z, ret.reshape(-1).astype(np.float64), h, h,
                                  c_v=c_v, c_e=c_e)
    np.testing.assert_allclose(stats, st, rtol=1e-4, atol=1e-7)
    for before, after, g in ((pa, pa2, ga), (pc, pc2, gc)):
        step = (before.astype(np.float64) - after.astype(np.float64)) / lr
        tol = 1e-4 * np.abs(g).max() + 0.6 * np.spacing(np.abs(before)).astype(np.float64) / lr
        assert np.all(np.abs(step - g) <= tol), np.abs(step - g).max()
    # the next roll-out runs on the updated policy
    r.rollout(2)
    r.sync()
    r.close()


@pytest.mark.parametrize("path", [F32, BF16])
def test_a2c_update_economy_agents_and_planner(torch, path):
    """Two updates in one call: the agents' policy and critic on the agent
    slots, the planner's on the planner slots, each the mean over its rows."""
    n_env, T, lr, c_v, c_e = 40, 12, 1.0, 0.5, 0.01
    counts = [oracle.econ_agent_count(5, e) for e in range(n_env)]
    Sa = sum(counts)
    r = W.Rollout(W.WS_ENV_ECONOMY, path, n_env, T, 540, 128, 128, param_seed=5,
                  flags=W.WS_FLAG_TRAIN, chunk_steps=6)
    r.reset(2)
    r.rollout(T)
    AW, PW = [16, 128, 128, 20], [16, 128, 128, 10]
    na, npl = oracle.policy_param_count(AW), oracle.policy_param_count(PW)
    nca, ncp = oracle.policy_param_count([16, 128, 128, 1]), oracle.policy_param_count([16, 128, 128, 1])
    par = r.fetch_raw(W.WS_F_PARAMS, 4 * (na + npl)).view(np.float32).copy()
    cri = r.fetch_raw(W.WS_F_CRITIC, 4 * (nca + ncp)).view(np.float32).copy()
    obs, act = r.fetch(W.WS_F_OBS, 0, T), r.fetch(W.WS_F_ACTION, 0, T)
    stats = r.a2c_update(T, lr, c_v, c_e)
    ret = r.fetch(W.WS_F_RETURN, 0, T)
    par2 = r.fetch_raw(W.WS_F_PARAMS, par.nbytes).view(np.float32).copy()
    cri2 = r.fetch_raw(W.WS_F_CRITIC, cri.nbytes).view(np.float32).copy()
    r.close()
    tot = np.zeros(3)
    for sl, pw, p0, c0, nap, ncr in ((slice(0, Sa), AW, 0, 0, na, nca),
                                     (slice(Sa, Sa + n_env), PW, na, nca, npl, ncp)):
        X = obs[:, :, sl].transpose(0, 2, 1).reshape(-1, 16).astype(np.float64)
        A = act[:, sl].reshape(-1)
        G = ret[:, sl].reshape(-1).astype(np.float64)
        st, ga, gc = oracle.a2c(par[p0:p0 + nap], cri[c0:c0 + ncr], X, A, G, 128, 128, pw[3],
                                c_v=c_v, c_e=c_e)
        tot += st * len(G)
        for before, after, g in ((par[p0:p0 + nap], par2[p0:p0 + nap], ga),
                                 (cri[c0:c0 + ncr], cri2[c0:c0 + ncr], gc)):
            step = (before.astype(np.float64) - after.astype(np.float64)) / lr
            tol = 1e-4 * np.abs(g).max() + 0.6 * np.spacing(np.abs(before)).astype(np.float64) / lr
            assert np.all(np.abs(step - g) <= tol), np.abs(step - g).max()
    np.testing.assert_allclose(stats, tot / (T * (Sa + n_env)), rtol=1e-4, atol=1e-7)


def test_a2c_update_window_over_wrapped_ring(torch):
    """The update's window is the last n steps of a ring that has wrapped: rows
    gathered modulo the ring, returns scanned over the same window."""
    n_env, R, T, n, h, lr, c_v, c_e = 500, 20, 33, 14, 32, 1.0, 0.5, 0.0
    r = W.Rollout(W.WS_ENV_CONTROL, F32, n_env, R, 25, h, h, param_seed=6, flags=W.WS_FLAG_TRAIN,
                  chunk_steps=7)
    r.reset(3)
    r.rollout(T)
    pa = r.fetch_raw(W.WS_F_PARAMS, 4 * oracle.policy_param_count([4, h, h, 2])).view(np.float32).copy()
    pc = r.fetch_raw(W.WS_F_CRITIC, 4 * oracle.policy_param_count([4, h, h, 1])).view(np.float32).copy()
    obs, act = r.fetch(W.WS_F_OBS, T - n, n), r.fetch(W.WS_F_ACTION, T - n, n)
    rew, done = r.fetch(W.WS_F_REWARD, T - n, n), r.fetch(W.WS_F_DONE, T - n, n)
    stats = r.a2c_update(n, lr, c_v, c_e)
    ret = r.fetch(W.WS_F_RETURN, T - n, n)
    pa2 = r.fetch_raw(W.WS_F_PARAMS, pa.nbytes).view(np.float32).copy()
    pc2 = r.fetch_raw(W.WS_F_CRITIC, pc.nbytes).view(np.float32).copy()
    r.close()
    Go = oracle.returns(rew, done, float(np.float32(0.99)))
    assert np.abs(ret - Go).max() <= 1e-6 * max(1.0, np.abs(Go).max())
    rows = dict(obs=obs.transpose(0, 2, 1).reshape(-1, 4).astype(np.float64), act=act.reshape(-1),
                ret=ret.reshape(-1).astype(np.float64))
    check_grads((pa, pc, pa2, pc2), rows, stats, (4, 2), h, lr, c_v, c_e)
