"""GPU parity of the multi-agent economy (plain and graph-batched FP32 paths)."""
import numpy as np
import pytest

import oracle
from paper_2408_00930_gb300 import inputs
from paper_2408_00930_gb300 import warpsci as W
from tests import ws_helpers as H
from tests.gpu_common import TIE_F32, TOL_F32, need_gpu

pytestmark = pytest.mark.gpu
AW, PW = [16, 128, 128, 20], [16, 128, 128, 10]
NA, NP = oracle.policy_param_count(AW), oracle.policy_param_count(PW)


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


def econ(path, counts=None, n_envs=None, ring=8, limit=540, seed=1, **kw):
    n = len(counts) if counts is not None else n_envs
    return W.Rollout(W.WS_ENV_ECONOMY, path, n, ring, limit, 128, 128, param_seed=seed,
                     agents_per_env=counts, **kw)


def _fetch_state(r, n_agents, n_envs):
    return H.unpack_econ_state(r.fetch_raw(W.WS_F_STATE, 72 * n_agents + 4 * n_envs), n_agents, n_envs)


def test_init_counts_params_and_reset(torch):
    r = econ(W.WS_PATH_PLAIN_FP32, n_envs=37, seed=13)
    counts = r.fetch_raw(W.WS_F_ENV_PARAMS, 4 * 37).view(np.int32)
    assert list(counts) == [oracle.econ_agent_count(13, e) for e in range(37)]
    par = r.fetch_raw(W.WS_F_PARAMS, 4 * (NA + NP)).view(np.float32)
    np.testing.assert_array_equal(par[:NA], oracle.policy_init(13, 0, AW))
    np.testing.assert_array_equal(par[NA:], oracle.policy_init(13, 1, PW))
    sa = int(counts.sum())
    w, f, t = _fetch_state(r, sa, 37)
    off = np.concatenate([[0], np.cumsum(counts)])
    for e in (0, 17, 36):
        for i in (0, int(counts[e]) - 1):
            wo, fo = oracle.econ_reset_agent(13, oracle.STEP_INIT, e, i)
            assert w[off[e] + i] == wo
            np.testing.assert_allclose(f[off[e] + i], fo, rtol=0, atol=2e-6)
    assert np.all(t == 0)
    r.close()


@pytest.mark.parametrize("path", [W.WS_PATH_PLAIN_FP32, W.WS_PATH_BATCHED_FP32])
def test_one_step_replay_seeded(torch, path):
    g = inputs.rng(5)
    counts = inputs.econ_agent_counts(g, 40)
    counts[:3] = [8, 256, 2]
    sa = int(counts.sum())
    ap = inputs.policy_params(g, AW, scale=3.0)
    pp = inputs.policy_params(g, PW, scale=3.0)
    w0, f0 = inputs.econ_state(g, counts)
    t0 = g.integers(0, 540, len(counts)).astype(np.int32)
    t0[:4] = 539                                   # done + reset in this step
    r = econ(path, counts=counts)
    r.load_raw(W.WS_F_PARAMS, np.concatenate([ap, pp]))
    k0 = 4242
    r.load_raw(W.WS_F_STATE, H.pack_econ_state(w0, f0, t0), k=k0)
    r.step()
    r.sync()
    rec = {f: r.fetch(fid, k0, 1)[0] for f, fid in [
        ("obs", W.WS_F_OBS), ("action", W.WS_F_ACTION), ("logp", W.WS_F_LOGP),
        ("reward", W.WS_F_REWARD), ("done", W.WS_F_DONE), ("wealth", W.WS_F_WEALTH)]}
    w1, f1, t1 = _fetch_state(r, sa, len(counts))
    o = oracle.econ_rollout(ap, pp, seed=1, env_ids=np.arange(len(counts)), n_agents=counts,
                            n_steps=1, episode_limit=540, k0=k0, wealth0=w0, feat0=f0, t0=t0)
    off = np.concatenate([[0], np.cumsum(counts)])
    amb_env = np.zeros(len(counts), bool)
    for e in range(len(counts)):
        amb_env[e] = (o["act_margin"][0, off[e]:off[e + 1]] < TIE_F32).any() or \
            o["act_margin"][0, sa + e] < TIE_F32
    assert amb_env.sum() <= 2
    # pre-step records: observations (agents exact, planner mean), wealth exact
    np.testing.assert_array_equal(rec["obs"][:, :sa].T, f0.astype(np.float32))
    np.testing.assert_allclose(rec["obs"][:, sa:].T, o["obs"][0, sa:], rtol=0, atol=1e-6)
    np.testing.assert_array_equal(rec["wealth"], o["wealth"][0])
    for e in np.nonzero(~amb_env)[0]:
        sl = np.r_[off[e]:off[e + 1], sa + e]
        assert np.array_equal(rec["action"][sl], o["action"][0][sl])
        assert np.array_equal(rec["done"][sl], o["done"][0][sl])
        np.testing.assert_allclose(rec["logp"][sl], o["logp"][0][sl], rtol=TOL_F32, atol=TOL_F32)
        np.testing.assert_allclose(rec["reward"][sl], o["reward"][0][sl], rtol=TOL_F32, atol=TOL_F32)
        a = slice(off[e], off[e + 1])
        assert np.array_equal(w1[a], o["wealth_out"][a]), e          # int64, bit-exact
        err = H.rel_err_rows(f1[a], o["feat_out"][a])
        assert err.max() <= TOL_F32, (e, err.max())
        assert t1[e] == o["t"][e]
    r.close()


def _forced(orc_counts_agent_const, planner_tau):
    ap = np.zeros(NA, np.float32)
    ap[-20 + orc_counts_agent_const] = 1000.0
    pp = np.zeros(NP, np.float32)
    pp[-10 + planner_tau] = 1000.0
    return ap, pp


def test_forced_policy_long_rollout_exact_wealth_and_returns(torch):
    """Saturated policies make every action deterministic: 540 steps + reset, wealth
    bit-exact against the oracle, returns over the episode within 1e-6."""
    g = inputs.rng(9)
    counts = np.array([8, 31, 256, 100], np.int32)
    ap, pp = _forced(13, 4)
    T = 560
    r = econ(W.WS_PATH_BATCHED_FP32, counts=counts, ring=T, limit=540, seed=2, chunk_steps=40)
    r.load_raw(W.WS_F_PARAMS, np.concatenate([ap, pp]))
    r.reset(77)
    r.rollout(T)
    r.returns(T)
    r.sync()
    wealth = r.fetch(W.WS_F_WEALTH, 0, T)
    act = r.fetch(W.WS_F_ACTION, 0, T)
    rew = r.fetch(W.WS_F_REWARD, 0, T)
    dn = r.fetch(W.WS_F_DONE, 0, T)
    G = r.fetch(W.WS_F_RETURN, 0, T)
    o = oracle.econ_rollout(ap, pp, seed=77, env_ids=np.arange(4), n_agents=counts, n_steps=T,
                            episode_limit=540)
    assert np.array_equal(act, o["action"])
    assert np.array_equal(dn, o["done"])
    assert np.array_equal(wealth, o["wealth"])
    sa = int(counts.sum())
    assert np.all(wealth[:540, sa:] == wealth[0, sa:])      # conservation through the episode
    np.testing.assert_allclose(rew, o["reward"], rtol=1e-5, atol=1e-6)
    Go = oracle.returns(o["reward"], o["done"], float(np.float32(0.99)))
    scale = oracle.returns(np.abs(o["reward"]), o["done"], float(np.float32(0.99)))
    err = np.abs(G - Go) / np.maximum(scale, 1.0)
    assert err.max() <= 1e-5, err.max()
    r.close()


def test_random_policy_conservation_every_step(torch):
    r = econ(W.WS_PATH_BATCHED_FP32, n_envs=64, ring=100, limit=540, seed=3, chunk_steps=25)
    r.rollout(100)
    w = r.fetch(W.WS_F_WEALTH, 0, 100)
    counts = r.fetch_raw(W.WS_F_ENV_PARAMS, 4 * 64).view(np.int32)
    off = np.concatenate([[0], np.cumsum(counts)])
    sa = int(off[-1])
    for e in range(64):
        tot = w[:, off[e]:off[e + 1]].sum(1)
        assert np.all(tot == w[:, sa + e])
        assert np.all(tot == tot[0])
    a = r.fetch(W.WS_F_ACTION, 0, 100)
    assert a[:, :sa].min() >= 0 and a[:, :sa].max() <= 19 and a[:, sa:].max() <= 9
    r.close()


def test_graph_path_bytes_equal_plain_path(torch):
    out = []
    for path in (W.WS_PATH_PLAIN_FP32, W.WS_PATH_BATCHED_FP32):
        r = econ(path, n_envs=20, ring=30, seed=4, chunk_steps=8)
        r.rollout(30)
        out.append([r.fetch(f, 0, 30).tobytes() for f in (W.WS_F_ACTION, W.WS_F_WEALTH,
                                                          W.WS_F_OBS, W.WS_F_REWARD)])
        r.close()
    assert out[0] == out[1]


def test_returns_horizon_1000_compensated_fp32_within_1e6(torch):
    """Returns over a 1,000-step window with no episode end: the float-float scan
    stays within 1e-6 of the FP64 oracle (relative to sum_t gamma^t |r_t|), so no
    FP64 is needed on the device.  Saturated policies make every reward
    deterministic, isolating the scan's own rounding."""
    counts = np.array([8, 40], np.int32)
    ap, pp = _forced(7, 3)
    T = 1000
    r = econ(W.WS_PATH_BATCHED_FP32, counts=counts, ring=T, limit=5000, seed=5, chunk_steps=100)
    r.load_raw(W.WS_F_PARAMS, np.concatenate([ap, pp]))
    r.reset(31)
    r.rollout(T)
    r.returns(T)
    r.sync()
    G = r.fetch(W.WS_F_RETURN, 0, T).astype(np.float64)
    rew = r.fetch(W.WS_F_REWARD, 0, T).astype(np.float64)
    dn = r.fetch(W.WS_F_DONE, 0, T)
    assert dn.sum() == 0
    o = oracle.econ_rollout(ap, pp, seed=31, env_ids=np.arange(2), n_agents=counts, n_steps=T,
                            episode_limit=5000)
    assert np.array_equal(r.fetch(W.WS_F_WEALTH, 0, T), o["wealth"])
    gam = float(np.float32(0.99))
    # end to end against the oracle's FP64 rewards and FP64 scan; the FP32
    # rounding of each reward contributes ~3e-8 of the scale, the rest is the scan
    Go = oracle.returns(o["reward"], o["done"], gam)
    scale = oracle.returns(np.abs(o["reward"]), o["done"], gam)
    err = np.abs(G - Go) / np.maximum(scale, 1.0)
    assert err.max() <= 1e-6, err.max()
    np.testing.assert_allclose(rew, o["reward"], rtol=1e-6, atol=1e-7)
    r.close()
