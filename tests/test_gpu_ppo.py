"""GPU parity of the PPO update (ws_advantages + ws_ppo_update) against the
oracle's FP64 clipped-surrogate loss and gradients (pinned to finite
differences and autograd): the ADVANTAGE field is G - V(s) under the critic
before the update; each epoch's parameter change over lr is the gradient of
the mean loss at the parameters that epoch started from, with the advantage
held and the ring's recorded log-probabilities as the behaviour policy; for
the control env, the acrobot and the economy's agents and planners
(categorical heads) and the landscape (diagonal Gaussian head, its behaviour
samples rebuilt into the SAMPLE field), on the FP32 and the BF16 roll-out
paths.  The actor is perturbed after the roll-out
(output layer) so that rows fall on both sides of the clip range."""
import numpy as np
import pytest

import oracle
from paper_2408_00930_gb300 import warpsci as W
from tests.gpu_common import need_gpu

pytestmark = pytest.mark.gpu
F32, BF16 = W.WS_PATH_BATCHED_FP32, W.WS_PATH_BATCHED_BF16
# relative reach of the FP32 ratio around a clip boundary: rows closer than
# this may take either side of the min, so their policy term is in the tolerance
AMBIG = 1e-4


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


def log_pi(actor, widths, X, A):
    lg = oracle.mlp_forward(widths, actor, X)
    m = lg.max(1, keepdims=True)
    lp = lg - m - np.log(np.exp(lg - m).sum(1, keepdims=True))
    return lp[np.arange(len(A)), A]


def perturb_output_layer(p, widths, scale, seed):
    """The actor with Gaussian noise (scale x the layer's spread) on its last
    layer's weights and bias."""
    n3 = widths[2] * widths[3] + widths[3]
    g = np.random.default_rng(seed)
    q = p.copy()
    q[-n3:] += (scale * p[-n3:].std() * g.standard_normal(n3)).astype(np.float32)
    return q


def check_epoch(pa, pc, pa2, pc2, widths, X, A, G, adv, lpo, lr, eps, c_v, c_e, stats):
    """The epoch's parameter change against the oracle's gradient at (pa, pc)
    (and stats, unless None, against the oracle's loss terms); returns the
    oracle's loss terms and the count of rows near a clip boundary."""
    h0, h1, na = widths[1], widths[2], widths[3]
    st, ga, gc = oracle.ppo(pa, pc, X, A, G, adv, lpo, h0, h1, na, eps, c_v, c_e)
    rho = np.exp(log_pi(pa, widths, X, A) - lpo)
    amb = ((np.abs(rho - (1 + eps)) < AMBIG * rho) | (np.abs(rho - (1 - eps)) < AMBIG * rho))
    extra = np.zeros_like(ga)
    if amb.any():                      # their policy term, as a share of the mean over all rows
        _, g_amb, _ = oracle.ppo(pa, pc, X[amb], A[amb], G[amb], adv[amb], lpo[amb], h0, h1, na,
                                 1e30, 0.0, 0.0)
        extra = np.abs(g_amb) * amb.sum() / len(G)
    if stats is not None:
        np.testing.assert_allclose(stats[1:3], st[1:3], rtol=1e-4, atol=1e-7)
        assert abs(stats[0] - st[0]) <= 1e-4 * (abs(st[0]) + np.abs(adv).mean()) + 1e-7
        assert abs(stats[3] - st[3]) <= amb.sum() / len(G) + 1e-12
    for before, after, g, ex in ((pa, pa2, ga, extra), (pc, pc2, gc, 0.0)):
        step = (before.astype(np.float64) - after.astype(np.float64)) / lr
        # after = fl(before - lr g): the subtraction loses up to half an ulp of the parameter
        tol = (1e-4 * np.abs(g).max() + ex +
               0.6 * np.spacing(np.abs(before)).astype(np.float64) / lr)
        assert np.all(np.abs(step - g) <= tol), np.abs(step - g).max()
        assert np.abs(g).max() > 0
    return st, int(amb.sum())


def advantages_and_rows(r, widths, T, critic, slots=None):
    """Fetch the update's rows (steps 0..T-1) and check ADVANTAGE = G - V(s)
    against the oracle critic's values; returns the rows (with the oracle's
    advantage) and the field as fetched."""
    od = widths[0]
    sl = slice(None) if slots is None else slots
    obs, act = r.fetch(W.WS_F_OBS, 0, T)[:, :, sl], r.fetch(W.WS_F_ACTION, 0, T)[:, sl]
    lpo, ret = r.fetch(W.WS_F_LOGP, 0, T)[:, sl], r.fetch(W.WS_F_RETURN, 0, T)[:, sl]
    adv_gpu = r.fetch(W.WS_F_ADVANTAGE, 0, T)[:, sl]
    X = obs.transpose(0, 2, 1).reshape(-1, od).astype(np.float64)
    G = ret.reshape(-1).astype(np.float64)
    V = oracle.mlp_forward([od, widths[1], widths[2], 1], critic, X)[:, 0]
    adv = G - V
    err = np.abs(adv_gpu.reshape(-1) - adv)
    assert np.all(err <= 1e-5 * (1 + np.abs(G) + np.abs(V))), err.max()
    return (X, act.reshape(-1), G, adv, lpo.reshape(-1).astype(np.float64)), adv_gpu


# perturbation scales that put roughly half of the first epoch's rows outside
# the clip range for these seeds
@pytest.mark.parametrize("env,path,n,h,scale", [(W.WS_ENV_CONTROL, F32, 3000, 64, 0.8),
                                                (W.WS_ENV_ACROBOT, F32, 3000, 64, 2.0),
                                                (W.WS_ENV_CONTROL, BF16, 1000, 256, 5.0)])
def test_ppo_epochs_match_oracle(torch, env, path, n, h, scale):
    """Two epochs over T x n rows (3000 x 30 = 90,000 rows: two update chunks)."""
    od, na = (4, 2) if env == W.WS_ENV_CONTROL else (6, 3)
    widths = [od, h, h, na]
    T, lr, eps, c_v, c_e = 30, 0.5, 0.15, 0.5, 0.01
    r = W.Rollout(env, path, n, T, 25, h, h, param_seed=3, flags=W.WS_FLAG_TRAIN, chunk_steps=10)
    r.reset(4)
    r.rollout(T)
    na_p, nc_p = oracle.policy_param_count(widths), oracle.policy_param_count([od, h, h, 1])
    pa = r.fetch_raw(W.WS_F_PARAMS, 4 * na_p).view(np.float32).copy()
    pc = r.fetch_raw(W.WS_F_CRITIC, 4 * nc_p).view(np.float32).copy()
    r.advantages(T)
    (X, A, G, adv, lpo), adv_gpu = advantages_and_rows(r, widths, T, pc)
    pa = perturb_output_layer(pa, widths, scale, seed=11)
    r.load_raw(W.WS_F_PARAMS, pa)
    fracs = []
    for _ in range(2):
        stats = r.ppo_update(T, lr, eps, c_v, c_e)
        pa2 = r.fetch_raw(W.WS_F_PARAMS, pa.nbytes).view(np.float32).copy()
        pc2 = r.fetch_raw(W.WS_F_CRITIC, pc.nbytes).view(np.float32).copy()
        st, _ = check_epoch(pa, pc, pa2, pc2, widths, X, A, G, adv, lpo, lr, eps, c_v, c_e, stats)
        fracs.append(st[3])
        pa, pc = pa2, pc2
    # the advantage stayed as ws_advantages wrote it
    np.testing.assert_array_equal(r.fetch(W.WS_F_ADVANTAGE, 0, T), adv_gpu)
    assert 0.02 < fracs[0] < 0.98, fracs      # rows on both sides of the clip range
    r.close()


@pytest.mark.parametrize("path", [F32, BF16])
def test_ppo_economy_agents_and_planner(torch, path):
    """Two updates in one call: the agents' policy and critic on the agent
    slots, the planner's on the planner slots, each the mean over its rows."""
    n_env, T, lr, eps, c_v, c_e = 40, 12, 0.5, 0.2, 0.5, 0.01
    counts = [oracle.econ_agent_count(5, e) for e in range(n_env)]
    Sa = sum(counts)
    r = W.Rollout(W.WS_ENV_ECONOMY, path, n_env, T, 540, 128, 128, param_seed=5,
                  flags=W.WS_FLAG_TRAIN, chunk_steps=6)
    r.reset(2)
    r.rollout(T)
    AW, PW = [16, 128, 128, 20], [16, 128, 128, 10]
    na, npl = oracle.policy_param_count(AW), oracle.policy_param_count(PW)
    nc = oracle.policy_param_count([16, 128, 128, 1])
    par = r.fetch_raw(W.WS_F_PARAMS, 4 * (na + npl)).view(np.float32).copy()
    cri = r.fetch_raw(W.WS_F_CRITIC, 4 * 2 * nc).view(np.float32).copy()
    r.advantages(T)
    groups = []
    for sl, pw, p0, c0, nap in ((slice(0, Sa), AW, 0, 0, na),
                                (slice(Sa, Sa + n_env), PW, na, nc, npl)):
        rows, _ = advantages_and_rows(r, pw, T, cri[c0:c0 + nc], slots=sl)
        groups.append((pw, p0, c0, nap, rows))
    par = np.concatenate([perturb_output_layer(par[:na], AW, 1.0, seed=12),
                          perturb_output_layer(par[na:], PW, 3.0, seed=13)])
    r.load_raw(W.WS_F_PARAMS, par)
    stats = r.ppo_update(T, lr, eps, c_v, c_e)
    par2 = r.fetch_raw(W.WS_F_PARAMS, par.nbytes).view(np.float32).copy()
    cri2 = r.fetch_raw(W.WS_F_CRITIC, cri.nbytes).view(np.float32).copy()
    r.close()
    tot, n_rows, n_amb = np.zeros(4), 0, 0
    for pw, p0, c0, nap, (X, A, G, adv, lpo) in groups:
        # per group its gradient; the stats are means over both groups' rows
        st, amb = check_epoch(par[p0:p0 + nap], cri[c0:c0 + nc], par2[p0:p0 + nap],
                              cri2[c0:c0 + nc], pw, X, A, G, adv, lpo, lr, eps, c_v, c_e, None)
        tot += st * len(G)
        n_rows += len(G)
        n_amb += amb
    np.testing.assert_allclose(stats[1:3], tot[1:3] / n_rows, rtol=1e-4, atol=1e-7)
    assert abs(stats[3] - tot[3] / n_rows) <= n_amb / n_rows + 1e-12
    assert 0.02 < stats[3] < 0.98, stats


def test_ppo_window_over_wrapped_ring(torch):
    """Advantages and the epoch over the last n steps of a ring that has
    wrapped."""
    n_env, R, T, n, h, lr, eps = 500, 20, 33, 14, 32, 0.5, 0.1
    widths = [4, h, h, 2]
    r = W.Rollout(W.WS_ENV_CONTROL, F32, n_env, R, 25, h, h, param_seed=6, flags=W.WS_FLAG_TRAIN,
                  chunk_steps=7)
    r.reset(3)
    r.rollout(T)
    pa = r.fetch_raw(W.WS_F_PARAMS, 4 * oracle.policy_param_count(widths)).view(np.float32).copy()
    pc = r.fetch_raw(W.WS_F_CRITIC, 4 * oracle.policy_param_count([4, h, h, 1])).view(np.float32).copy()
    r.advantages(n)
    obs, act = r.fetch(W.WS_F_OBS, T - n, n), r.fetch(W.WS_F_ACTION, T - n, n)
    lpo, ret = r.fetch(W.WS_F_LOGP, T - n, n), r.fetch(W.WS_F_RETURN, T - n, n)
    adv_gpu = r.fetch(W.WS_F_ADVANTAGE, T - n, n)
    X = obs.transpose(0, 2, 1).reshape(-1, 4).astype(np.float64)
    G = ret.reshape(-1).astype(np.float64)
    V = oracle.mlp_forward([4, h, h, 1], pc, X)[:, 0]
    assert np.all(np.abs(adv_gpu.reshape(-1) - (G - V)) <= 1e-5 * (1 + np.abs(G) + np.abs(V)))
    pa = perturb_output_layer(pa, widths, 2.0, seed=14)
    r.load_raw(W.WS_F_PARAMS, pa)
    stats = r.ppo_update(n, lr, eps, 0.5, 0.0)
    pa2 = r.fetch_raw(W.WS_F_PARAMS, pa.nbytes).view(np.float32).copy()
    pc2 = r.fetch_raw(W.WS_F_CRITIC, pc.nbytes).view(np.float32).copy()
    r.close()
    check_epoch(pa, pc, pa2, pc2, widths, X, act.reshape(-1), G, G - V,
                lpo.reshape(-1).astype(np.float64), lr, eps, 0.5, 0.0, stats)


def test_ppo_errors(torch):
    r = W.Rollout(W.WS_ENV_CONTROL, F32, 16, 4, 100, 16, 16)
    r.rollout(2)
    assert W.ws_advantages(r.ctx, 2) == W.WS_ERR_STATE                      # no WS_FLAG_TRAIN
    assert W.ws_ppo_update(r.ctx, 2, 0.1, 0.2, 0.5, 0.0) == W.WS_ERR_STATE
    r.close()
    r = W.Rollout(W.WS_ENV_CONTROL, F32, 16, 4, 100, 16, 16, flags=W.WS_FLAG_TRAIN)
    r.rollout(3)
    assert W.ws_ppo_update(r.ctx, 2, 0.1, 0.2, 0.5, 0.0) == W.WS_ERR_STATE   # no advantages yet
    assert W.ws_advantages(r.ctx, 4) == W.WS_ERR_RANGE
    assert W.ws_advantages(r.ctx, 2) == W.WS_OK
    assert W.ws_ppo_update(r.ctx, 3, 0.1, 0.2, 0.5, 0.0) == W.WS_ERR_STATE   # covers 2 steps only
    assert W.ws_ppo_update(r.ctx, 2, 0.1, 0.0, 0.5, 0.0) == W.WS_ERR_INVALID  # clip_eps not > 0
    assert W.ws_ppo_update(r.ctx, 2, float("nan"), 0.2, 0.5, 0.0) == W.WS_ERR_INVALID
    assert W.ws_ppo_update(r.ctx, 2, 0.1, 0.2, 0.5, 0.0) == W.WS_OK
    assert W.ws_ppo_update(r.ctx, 1, 0.1, 0.2, 0.5, 0.0) == W.WS_OK           # a shorter window
    r.rollout(1)
    assert W.ws_ppo_update(r.ctx, 2, 0.1, 0.2, 0.5, 0.0) == W.WS_ERR_STATE   # stale advantages
    assert W.ws_advantages(r.ctx, 3) == W.WS_OK
    r.reset(1)
    assert W.ws_ppo_update(r.ctx, 1, 0.1, 0.2, 0.5, 0.0) in (W.WS_ERR_STATE, W.WS_ERR_RANGE)
    r.sync()
    r.close()
    r = W.Rollout(W.WS_ENV_LANDSCAPE, F32, 16, 4, 100, 16, 16, dim=8, n_gauss=16)
    r.rollout(2)
    dst = np.empty((2, 8, 16), np.float32)
    assert W.ws_fetch(r.ctx, W.WS_F_SAMPLE, 0, 2, dst.ctypes.data, dst.nbytes, 0) != W.WS_OK
    r.close()


@pytest.mark.parametrize("path,h", [(F32, 32), (BF16, 256)])
def test_ppo_landscape_gaussian_head(torch, path, h):
    """ws_advantages rebuilds each row's unclipped sample u = mean + sigma z
    (checked against the oracle's forward and normals, and on the FP32 path
    against the step the env took); two epochs score u under the perturbed
    and then updated Gaussian."""
    D, M, n, T, lr, eps, c_v, c_e = 8, 64, 200, 12, 0.5, 0.15, 0.5, 0.01
    widths = [D, h, h, 2 * D]
    r = W.Rollout(W.WS_ENV_LANDSCAPE, path, n, T, 7, h, h, dim=D, n_gauss=M, param_seed=4,
                  flags=W.WS_FLAG_TRAIN, chunk_steps=5)
    r.reset(6)
    r.rollout(T)
    pa = r.fetch_raw(W.WS_F_PARAMS, 4 * oracle.policy_param_count(widths)).view(np.float32).copy()
    pc = r.fetch_raw(W.WS_F_CRITIC, 4 * oracle.policy_param_count([D, h, h, 1])).view(np.float32).copy()
    r.advantages(T)
    obs, dx, smp = (r.fetch(f, 0, T) for f in (W.WS_F_OBS, W.WS_F_ACTION, W.WS_F_SAMPLE))
    lpo = r.fetch(W.WS_F_LOGP, 0, T).reshape(-1).astype(np.float64)
    G = r.fetch(W.WS_F_RETURN, 0, T).reshape(-1).astype(np.float64)
    adv_gpu = r.fetch(W.WS_F_ADVANTAGE, 0, T).reshape(-1)
    X = obs.transpose(0, 2, 1).reshape(-1, D).astype(np.float64)
    U_gpu = smp.transpose(0, 2, 1).reshape(-1, D).astype(np.float64)
    Z = np.array([oracle.landscape_action_normals(6, t, e, D) for t in range(T) for e in range(n)])
    out0 = oracle.mlp_forward(widths, pa, X)
    sig0 = np.exp(np.clip(out0[:, D:], -5.0, 2.0))
    U = out0[:, :D] + sig0 * Z
    assert np.all(np.abs(U_gpu - U) <= 1e-5 * (1 + np.abs(out0[:, :D]) + sig0 * np.abs(Z)))
    if path == F32:      # the env took the clipped sample
        step = dx.transpose(0, 2, 1).reshape(-1, D).astype(np.float64)
        assert np.abs(np.clip(U_gpu, -0.1, 0.1) - step).max() <= 1e-6
    V = oracle.mlp_forward([D, h, h, 1], pc, X)[:, 0]
    adv = G - V
    assert np.all(np.abs(adv_gpu - adv) <= 1e-5 * (1 + np.abs(G) + np.abs(V)))
    pa = perturb_output_layer(pa, widths, 0.2, seed=15)
    r.load_raw(W.WS_F_PARAMS, pa)
    fracs = []
    for _ in range(2):
        stats = r.ppo_update(T, lr, eps, c_v, c_e)
        pa2 = r.fetch_raw(W.WS_F_PARAMS, pa.nbytes).view(np.float32).copy()
        pc2 = r.fetch_raw(W.WS_F_CRITIC, pc.nbytes).view(np.float32).copy()
        st, ga, gc = oracle.ppo_gauss(pa, pc, X, U, G, adv, lpo, h, h, eps, c_v, c_e)
        # rows within FP32 reach of a clip boundary: their policy term is in the tolerance
        o = oracle.mlp_forward(widths, pa, X)
        ls = np.clip(o[:, D:], -5.0, 2.0)
        y = (U - o[:, :D]) / np.exp(ls)
        rho = np.exp((-0.5 * y * y - ls - 0.5 * np.log(2 * np.pi)).sum(1) - lpo)
        amb = (np.abs(rho - (1 + eps)) < AMBIG * rho) | (np.abs(rho - (1 - eps)) < AMBIG * rho)
        extra = np.zeros_like(ga)
        if amb.any():
            _, g_amb, _ = oracle.ppo_gauss(pa, pc, X[amb], U[amb], G[amb], adv[amb], lpo[amb], h,
                                           h, 1e30, 0.0, 0.0)
            extra = np.abs(g_amb) * amb.sum() / len(G)
        np.testing.assert_allclose(stats[1:3], st[1:3], rtol=1e-4, atol=1e-7)
        assert abs(stats[3] - st[3]) <= amb.sum() / len(G) + 1e-12
        for before, after, g, ex in ((pa, pa2, ga, extra), (pc, pc2, gc, 0.0)):
            dstep = (before.astype(np.float64) - after.astype(np.float64)) / lr
            tol = (1e-4 * np.abs(g).max() + ex +
                   0.6 * np.spacing(np.abs(before)).astype(np.float64) / lr)
            assert np.all(np.abs(dstep - g) <= tol), np.abs(dstep - g).max()
        fracs.append(st[3])
        pa, pc = pa2, pc2
    assert 0.02 < fracs[0] < 0.98, fracs
    r.close()
