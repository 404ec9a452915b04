"""BF16 tensor-core policy layers (economy and landscape BF16 paths) against the
oracle's MLP in BF16-operand mode (inputs and weights of every layer rounded to
bfloat16, exact accumulation)."""
import numpy as np
import pytest

import oracle
from paper_2408_00930_gb300 import inputs
from paper_2408_00930_gb300 import warpsci as W
from tests import ws_helpers as H
from tests.gpu_common import TOL_BF16, TOL_F32, need_gpu

pytestmark = pytest.mark.gpu
BF16 = W.WS_PATH_BATCHED_BF16
ALL_BF16 = 0b111
AW, PW = [16, 128, 128, 20], [16, 128, 128, 10]
NA, NP = oracle.policy_param_count(AW), oracle.policy_param_count(PW)
# tie band of the categorical draw when the logits carry BF16 operand rounding
TIE = 5e-3
# energy of the BF16 path (hi+lo cross-term, ex2.approx epilogue), relative to
# the scale sum_m |a_m| e_m: the missing y_lo.c_lo term and the bf16 rounding of
# y_lo, c_lo give |d(d2)| <~ 2^-15 |y||c| D, i.e. ~1e-3 of a term at w ~ 1
ENERGY_TOL_BF16 = 5e-3


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


def logit_err(g, o):
    return np.abs(g - o).max(axis=1) / np.maximum(np.abs(o).max(axis=1), 1.0)


def test_econ_bf16_logits_actions_and_wealth(torch):
    g = inputs.rng(41)
    counts = inputs.econ_agent_counts(g, 30, lo=2, hi=12)
    counts[:3] = [2, 3, 257 // 2]
    sa = int(counts.sum())
    ap = inputs.policy_params(g, AW, scale=3.0)
    pp = inputs.policy_params(g, PW, scale=3.0)
    w0, f0 = inputs.econ_state(g, counts)
    t0 = np.zeros(len(counts), np.int32)
    r = W.Rollout(W.WS_ENV_ECONOMY, BF16, len(counts), 8, 540, 128, 128, agents_per_env=counts,
                  flags=W.WS_FLAG_DEBUG_LOGITS)
    r.load_raw(W.WS_F_PARAMS, np.concatenate([ap, pp]))
    k0 = 99
    r.load_raw(W.WS_F_STATE, H.pack_econ_state(w0, f0, t0), k=k0)
    r.step()
    r.sync()
    lg = r.fetch_raw(W.WS_F_LOGITS, 4 * (20 * sa + 10 * len(counts))).view(np.float32)
    lg_a = lg[:20 * sa].reshape(sa, 20)
    lg_p = lg[20 * sa:].reshape(len(counts), 10)
    o_a = oracle.mlp_forward(AW, ap, f0, bf16_layers=ALL_BF16)
    o_p_obs = np.array([f0[a:b].mean(0) for a, b in zip(np.r_[0, np.cumsum(counts)[:-1]], np.cumsum(counts))])
    o_p = oracle.mlp_forward(PW, pp, o_p_obs, bf16_layers=ALL_BF16)
    assert logit_err(lg_a, o_a).max() <= TOL_BF16
    assert logit_err(lg_p, o_p).max() <= TOL_BF16
    act = r.fetch(W.WS_F_ACTION, k0, 1)[0]
    wealth1, _, _ = H.unpack_econ_state(r.fetch_raw(W.WS_F_STATE, 72 * sa + 4 * len(counts)), sa,
                                       len(counts))
    o = oracle.econ_rollout(ap, pp, seed=1, env_ids=np.arange(len(counts)), n_agents=counts,
                            n_steps=1, episode_limit=540, k0=k0, wealth0=w0, feat0=f0, t0=t0,
                            bf16_layers=ALL_BF16)
    ok = o["act_margin"][0] >= TIE
    assert ok.mean() > 0.6
    assert np.array_equal(act[ok], o["action"][0][ok])
    off = np.r_[0, np.cumsum(counts)]
    n_exact = 0
    for e in range(len(counts)):
        sl = np.r_[off[e]:off[e + 1], sa + e]
        if ok[sl].all():
            assert np.array_equal(wealth1[off[e]:off[e + 1]], o["wealth_out"][off[e]:off[e + 1]])
            n_exact += 1
        assert wealth1[off[e]:off[e + 1]].sum() == w0[off[e]:off[e + 1]].sum()   # always conserved
    assert n_exact >= 3
    r.close()


def test_econ_bf16_graph_rollout_conserves_and_is_deterministic(torch):
    out = []
    for _ in range(2):
        r = W.Rollout(W.WS_ENV_ECONOMY, BF16, 48, 60, 540, 128, 128, param_seed=8, chunk_steps=20)
        r.rollout(60)
        out.append((r.fetch(W.WS_F_WEALTH, 0, 60), r.fetch(W.WS_F_ACTION, 0, 60)))
        counts = r.fetch_raw(W.WS_F_ENV_PARAMS, 4 * 48).view(np.int32)
        r.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    w = out[0][0]
    off = np.r_[0, np.cumsum(counts)]
    for e in range(48):
        tot = w[:, off[e]:off[e + 1]].sum(1)
        assert np.all(tot == tot[0]) and np.all(w[:, off[-1] + e] == tot)


def test_landscape_bf16_outputs_and_step(torch):
    D, M, n, h = 24, 4096, 300, (256, 256)
    g = inputs.rng(43)
    c, wd, am = inputs.landscape_params(g, M, D)
    x0, eobs0, t0 = inputs.landscape_state(g, n, D)
    x0[:30] = (c[:30] + g.normal(0, 0.3, (30, D))).astype(np.float32)
    params = inputs.policy_params(g, [D, *h, 2 * D])
    r = W.Rollout(W.WS_ENV_LANDSCAPE, BF16, n, 8, 1000, *h, dim=D, n_gauss=M,
                  flags=W.WS_FLAG_DEBUG_LOGITS)
    r.load_raw(W.WS_F_ENV_PARAMS, np.concatenate([c.astype(np.float32).ravel(),
                                                  wd.astype(np.float32), am.astype(np.float32)]))
    r.load_raw(W.WS_F_PARAMS, params)
    r.load_raw(W.WS_F_STATE, H.pack_landscape_state(x0, eobs0, t0), k=3)
    r.step()
    r.sync()
    out = r.fetch_raw(W.WS_F_LOGITS, 4 * n * 2 * D).view(np.float32).reshape(n, 2 * D)
    o_out = oracle.mlp_forward([D, *h, 2 * D], params, x0, bf16_layers=ALL_BF16)
    assert logit_err(out, o_out).max() <= TOL_BF16
    act = r.fetch(W.WS_F_ACTION, 3, 1)[0].T.astype(np.float64)
    en = r.fetch(W.WS_F_ENERGY, 3, 1)[0]
    o = oracle.landscape_rollout(c, wd, am, params, *h, seed=1, env_ids=np.arange(n), n_steps=1,
                                 episode_limit=1000, k0=3, x0=x0, eobs0=eobs0, t0=t0,
                                 bf16_layers=ALL_BF16)
    # dx = clip(mean + sigma z): BF16 error of mean and log sigma, scaled by |z| <~ 5
    assert np.abs(act - o["act"][0]).max() <= 0.1 * TOL_BF16 * 10
    # energy at the post-step state: the oracle's E at its own x' plus the first-order
    # effect of a BF16-sized step difference (|dx_gpu - dx_oracle| <= 2e-3 per coordinate)
    x1o = x0 + o["act"][0]
    for e in range(n):
        grad = oracle.landscape_grad(c, wd, am, x1o[e])
        tol = ENERGY_TOL_BF16 * max(o["energy_scale"][0][e], 1e-3) + 2.0 * np.abs(grad).sum() * 2e-3 + 1e-7
        assert abs(en[e] - o["energy"][0][e]) <= tol, e
    r.close()


def test_landscape_bf16_energy_against_fp64(torch):
    """Energies on the tensor-core path at states the oracle fixes exactly (the
    Philox reset draws, some placed near centres by a seeded landscape)."""
    D, M, n, h = 24, 4096, 512, (64, 64)
    g = inputs.rng(47)
    c, wd, am = inputs.landscape_params(g, M, D)
    x0, eobs0, t0 = inputs.landscape_state(g, n, D)
    t0[:] = 999                       # every env resets in this step
    params = inputs.policy_params(g, [D, *h, 2 * D])
    r = W.Rollout(W.WS_ENV_LANDSCAPE, BF16, n, 8, 1000, *h, dim=D, n_gauss=M)
    # centres of the first Gaussians moved onto the reset draws of the first envs
    # so that a share of the energies are O(1), not only tails
    xr = np.array([oracle.landscape_reset_draw(1, 7, e, D) for e in range(n)])
    c = c.copy()
    c[:64] = (xr[:64] + g.normal(0, 0.4, (64, D))).astype(np.float32)
    r.load_raw(W.WS_F_ENV_PARAMS, np.concatenate([c.astype(np.float32).ravel(),
                                                  wd.astype(np.float32), am.astype(np.float32)]))
    r.load_raw(W.WS_F_PARAMS, params)
    r.load_raw(W.WS_F_STATE, H.pack_landscape_state(x0, eobs0, t0), k=7)
    r.step()
    r.sync()
    x1, e1, t1 = H.unpack_landscape_state(r.fetch_raw(W.WS_F_STATE, 4 * D * n + 8 * n), n, D)
    np.testing.assert_array_equal(x1, xr.astype(np.float32).astype(np.float64))
    assert np.all(t1 == 0)
    errs = []
    for e in range(n):
        E = oracle.landscape_energy(c, wd, am, xr[e])
        sc = oracle.landscape_energy_scale(c, wd, am, xr[e])
        ref = E + 0.05 * oracle.landscape_noise(1, 7, e, 1)
        errs.append(abs(e1[e] - ref) / max(sc, 1e-3))
    errs = np.array(errs)
    assert errs.max() <= ENERGY_TOL_BF16, errs.max()
    assert np.median(errs) < 1e-3
    r.close()
