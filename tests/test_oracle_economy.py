"""Pins of the multi-agent economy: exact conservation, hand steps, special cases."""
import os

import numpy as np
import pytest

from paper_2408_00930_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
AW = [16, 128, 128, 20]
PW = [16, 128, 128, 10]


def _forced_agent_params(orc, by_sign=None, const=None):
    """Saturated agent policy: class `const`, or class by_sign[0] if feature 0 > 0
    else by_sign[1] (tanh(+-100) = +-1 exactly in FP64)."""
    p = np.zeros(orc.policy_param_count(AW), np.float32)
    o1 = 16 * 128 + 128
    o2 = o1 + 128 * 128 + 128
    b3 = o2 + 128 * 20
    if const is not None:
        p[b3 + const] = 1000.0
        return p
    p[0 * 128 + 0] = 100.0            # W1[0][0]
    p[o1 + 0 * 128 + 0] = 100.0       # W2[0][0]
    p[o2 + 0 * 20 + by_sign[0]] = 1000.0   # W3[0][c+]
    p[o2 + 0 * 20 + by_sign[1]] = -1000.0  # W3[0][c-]
    return p


def _forced_planner_params(orc, tau):
    p = np.zeros(orc.policy_param_count(PW), np.float32)
    p[-10 + tau] = 1000.0
    return p


def test_econ_hand_step(orc):
    ln = [l for l in open(os.path.join(GOLDEN, "econ_hand_step.txt")) if not l.startswith("#")][0]
    w0, acts, w1, rew, f = [list(map(float, part.split())) for part in ln.split("|")]
    ap = _forced_agent_params(orc, by_sign=(int(acts[0]), int(acts[1])))
    pp = _forced_planner_params(orc, int(acts[2]))
    feat = np.zeros((2, 16))
    feat[0, 0], feat[1, 0] = 1.0, -1.0
    r = orc.econ_rollout(ap, pp, seed=3, env_ids=[0], n_agents=[2], n_steps=1, episode_limit=540,
                         wealth0=np.array(w0, np.int64), feat0=feat, t0=[0])
    assert list(r["action"][0]) == [int(a) for a in acts]
    assert list(r["wealth_out"]) == [int(v) for v in w1]
    np.testing.assert_allclose(r["reward"][0], rew, rtol=0, atol=1e-12)
    np.testing.assert_allclose(r["feat_out"][0, :2], f, rtol=0, atol=1e-10)
    assert r["feat_out"][0, 15] == pytest.approx(np.log(1038) / np.log(1e6), abs=1e-12)
    assert r["wealth"][0, 2] == 3000            # planner slot records total wealth


def test_econ_conservation_random_policies(orc):
    g = inputs.rng(4)
    ap = inputs.policy_params(g, AW, scale=3.0)
    pp = inputs.policy_params(g, PW, scale=3.0)
    n_agents = [8, 13, 40, 256]
    r = orc.econ_rollout(ap, pp, seed=9, env_ids=[0, 1, 2, 3], n_agents=n_agents, n_steps=30,
                         episode_limit=540)
    off = np.cumsum([0] + n_agents)
    for e in range(4):
        tot = r["wealth"][:, off[e]:off[e + 1]].sum(axis=1)
        assert np.all(tot == tot[0])                       # exact, every step
        assert np.all(r["wealth"][:, off[-1] + e] == tot)  # planner record = total
        assert r["wealth_out"][off[e]:off[e + 1]].sum() == tot[0]
        assert np.all(r["wealth"][:, off[e]:off[e + 1]] > 0)
    acts = r["action"][:, :off[-1]]
    assert acts.min() >= 0 and acts.max() <= 19
    assert len(np.unique(acts)) > 10                      # random policies explore
    pl = r["action"][:, off[-1]:]
    assert pl.min() >= 0 and pl.max() <= 9


def test_econ_zero_activity_keeps_wealth(orc):
    ap = _forced_agent_params(orc, const=0)
    pp = _forced_planner_params(orc, 9)
    g = inputs.rng(5)
    w, f = inputs.econ_state(g, [12])
    r = orc.econ_rollout(ap, pp, seed=1, env_ids=[7], n_agents=[12], n_steps=5, episode_limit=540,
                         wealth0=w, feat0=f, t0=[0])
    assert np.all(r["wealth"][:, :12] == w[None, :])
    assert np.all(r["wealth_out"] == w)
    np.testing.assert_allclose(r["reward"][:, :12], 0.0, atol=0)


def test_econ_zero_tax_is_pure_transfer(orc):
    """tau = 0: each agent ends with w - t_i + income_i, partners from the PARTNER draw."""
    ap = _forced_agent_params(orc, const=19)
    pp = _forced_planner_params(orc, 0)
    g = inputs.rng(6)
    n = 9
    w, f = inputs.econ_state(g, [n])
    r = orc.econ_rollout(ap, pp, seed=2, env_ids=[5], n_agents=[n], n_steps=1, episode_limit=540,
                         wealth0=w, feat0=f, t0=[0], k0=17)
    exp = w.copy()
    for i in range(n):
        wd = orc.draw(2, 17, 5, i, orc.TAG_PARTNER)
        p = (i + 1 + orc.bounded(int(wd[0]), n - 1)) % n
        assert p != i
        amt = (int(w[i]) * 19) // 400
        exp[i] -= amt
        exp[p] += amt
    assert list(r["wealth_out"]) == list(exp)


def test_econ_tax_pool_remainder_goes_to_low_indices(orc):
    """With all wealth moving, the pool remainder T mod n lands on agents 0..rem-1."""
    ap = _forced_agent_params(orc, const=19)
    g = inputs.rng(7)
    n = 11
    w, f = inputs.econ_state(g, [n])
    r0 = orc.econ_rollout(ap, _forced_planner_params(orc, 0), seed=2, env_ids=[1], n_agents=[n],
                          n_steps=1, episode_limit=540, wealth0=w, feat0=f, t0=[0])
    r9 = orc.econ_rollout(ap, _forced_planner_params(orc, 9), seed=2, env_ids=[1], n_agents=[n],
                          n_steps=1, episode_limit=540, wealth0=w, feat0=f, t0=[0])
    income = np.zeros(n, np.int64)
    after = w.copy()
    for i in range(n):
        wd = orc.draw(2, 0, 1, i, orc.TAG_PARTNER)
        p = (i + 1 + orc.bounded(int(wd[0]), n - 1)) % n
        amt = (int(w[i]) * 19) // 400
        after[i] -= amt; after[p] += amt; income[p] += amt
    assert list(r0["wealth_out"]) == list(after)
    tax = income * 9 // 20
    T = int(tax.sum())
    exp = after - tax + T // n + (np.arange(n) < T % n)
    assert list(r9["wealth_out"]) == list(exp)
    assert r9["wealth_out"].sum() == w.sum()


def test_econ_done_and_reset(orc):
    g = inputs.rng(8)
    ap = inputs.policy_params(g, AW)
    pp = inputs.policy_params(g, PW)
    r = orc.econ_rollout(ap, pp, seed=4, env_ids=[3], n_agents=[10], n_steps=6, episode_limit=5)
    assert list(r["done"][:, 0]) == [0, 0, 0, 0, 1, 0]
    assert np.all(r["done"][4] == 1)                      # whole env incl. planner
    for i in range(10):
        wi, fi = orc.econ_reset_agent(4, 4, 3, i)          # redraw at step k = 4
        assert r["wealth"][5, i] == wi
        np.testing.assert_array_equal(r["obs"][5, i], fi)
        w0, f0 = orc.econ_reset_agent(4, orc.STEP_INIT, 3, i)
        assert r["wealth"][0, i] == w0
        assert 10_000 <= wi <= 1_000_000


def test_econ_agent_counts_range(orc):
    c = [orc.econ_agent_count(11, e) for e in range(4000)]
    assert min(c) == 8 and max(c) == 256
    assert abs(np.mean(c) - 132) < 3


def test_econ_pool_split_is_floor_for_negative_pools(orc):
    """With negative wealth the transfers, incomes and the tax pool turn negative; the
    split floor(T/n) plus the remainder T - n floor(T/n) in [0, n) still conserves."""
    ap = _forced_agent_params(orc, const=19)
    pp = _forced_planner_params(orc, 9)
    n = 7
    w = np.array([-50_003, -120_007, -9_999, 40_001, -77_777, -3_001, -1_000_000], np.int64)
    f = np.zeros((n, 16))
    r = orc.econ_rollout(ap, pp, seed=2, env_ids=[0], n_agents=[n], n_steps=3, episode_limit=540,
                         wealth0=w, feat0=f, t0=[0])
    for t in range(3):
        assert r["wealth"][t, :n].sum() == w.sum()
    assert r["wealth_out"].sum() == w.sum()
