"""GPU parity of the fused persistent economy kernel (BF16 path): a device work
queue of env groups, the agents' 16-128-128-20 MLP per 128-row tile and the
planner's 16-128-128-10 MLP with swapped operands on tcgen05, transfers and tax
in shared memory.  Compared with the oracle in BF16-operand mode (inputs and
weights of every layer rounded to bfloat16, exact accumulation)."""
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


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


def econ(counts=None, n_envs=None, ring=8, limit=540, seed=1, **kw):
    n = len(counts) if counts is not None else n_envs
    return W.Rollout(W.WS_ENV_ECONOMY, BF16, n, ring, limit, 128, 128, param_seed=seed,
                     agents_per_env=counts, **kw)


def state(r, sa, ne):
    return H.unpack_econ_state(r.fetch_raw(W.WS_F_STATE, 72 * sa + 4 * ne), sa, ne)


def logit_err(g, o):
    return np.abs(g - o).max(axis=1) / np.maximum(np.abs(o).max(axis=1), 1.0)


def test_fused_one_step_replay_many_items(torch):
    """One step from a seeded state over envs that force every kind of work
    item: a full 384-agent env, the 2- and 3-agent minimum, runs of tiny envs
    that hit the 64-envs-per-item cap, and drawn counts."""
    g = inputs.rng(61)
    counts = np.concatenate([[384, 2, 3, 256, 129, 128, 127],
                             inputs.econ_agent_counts(g, 90, lo=2, hi=6),
                             inputs.econ_agent_counts(g, 25)]).astype(np.int32)
    ne, sa = len(counts), int(counts.sum())
    ap = inputs.policy_params(g, AW, scale=3.0)
    pp = inputs.policy_params(g, PW, scale=3.0)
    w0, f0 = inputs.econ_state(g, counts)
    t0 = g.integers(0, 540, ne).astype(np.int32)
    t0[:5] = 539                                   # done + reset in this step
    r = econ(counts, flags=W.WS_FLAG_DEBUG_LOGITS)
    r.load_raw(W.WS_F_PARAMS, np.concatenate([ap, pp]))
    k0 = 777
    r.load_raw(W.WS_F_STATE, H.pack_econ_state(w0, f0, t0), k=k0)
    r.step()
    r.sync()
    rec = {f: r.fetch(fid, k0, 1)[0] for f, fid in [
        ("obs", W.WS_F_OBS), ("action", W.WS_F_ACTION), ("logp", W.WS_F_LOGP),
        ("reward", W.WS_F_REWARD), ("done", W.WS_F_DONE), ("wealth", W.WS_F_WEALTH)]}
    lg = r.fetch_raw(W.WS_F_LOGITS, 4 * (20 * sa + 10 * ne)).view(np.float32)
    w1, f1, t1 = state(r, sa, ne)
    off = np.r_[0, np.cumsum(counts)]
    # logits against the oracle's BF16-operand MLPs
    o_a = oracle.mlp_forward(AW, ap, f0, bf16_layers=ALL_BF16)
    pobs = np.array([f0[off[e]:off[e + 1]].mean(0) for e in range(ne)])
    o_p = oracle.mlp_forward(PW, pp, pobs, bf16_layers=ALL_BF16)
    assert logit_err(lg[:20 * sa].reshape(sa, 20), o_a).max() <= TOL_BF16
    assert logit_err(lg[20 * sa:].reshape(ne, 10), o_p).max() <= TOL_BF16
    o = oracle.econ_rollout(ap, pp, seed=1, env_ids=np.arange(ne), n_agents=counts, n_steps=1,
                            episode_limit=540, k0=k0, wealth0=w0, feat0=f0, t0=t0,
                            bf16_layers=ALL_BF16)
    # pre-step records: agent observations and wealth exact, planner mean and total
    np.testing.assert_array_equal(rec["obs"][:, :sa].T, f0.astype(np.float32))
    np.testing.assert_allclose(rec["obs"][:, sa:].T, o["obs"][0, sa:], rtol=0, atol=1e-6)
    np.testing.assert_array_equal(rec["wealth"], o["wealth"][0])
    ok = o["act_margin"][0] >= TIE
    assert ok.mean() > 0.6
    assert np.array_equal(rec["action"][ok], o["action"][0][ok])
    np.testing.assert_allclose(rec["logp"][ok], o["logp"][0][ok], rtol=TOL_BF16, atol=TOL_BF16)
    same = rec["action"] == o["action"][0]
    n_exact = 0
    for e in range(ne):
        a = slice(off[e], off[e + 1])
        assert w1[a].sum() == w0[a].sum() or t0[e] == 539   # conserved unless reset
        sl = np.r_[off[e]:off[e + 1], sa + e]
        assert np.array_equal(rec["done"][sl], o["done"][0][sl])
        if not same[sl].all():
            continue
        n_exact += 1
        assert np.array_equal(w1[a], o["wealth_out"][a]), e            # int64, bit-exact
        np.testing.assert_allclose(rec["reward"][sl], o["reward"][0][sl], rtol=TOL_F32, atol=TOL_F32)
        err = H.rel_err_rows(f1[a], o["feat_out"][a])
        assert err.max() <= TOL_F32, (e, err.max())
        assert t1[e] == o["t"][e]
    assert n_exact >= ne // 2
    r.close()


def _run(counts, T, chunk, limit, seed, reset_seed):
    r = econ(counts, ring=T, limit=limit, seed=seed, chunk_steps=chunk)
    r.reset(reset_seed)
    ne, sa = len(counts), int(np.sum(counts))
    init = state(r, sa, ne)
    r.rollout(T)
    r.sync()
    out = {f: r.fetch(fid, 0, T) for f, fid in [
        ("obs", W.WS_F_OBS), ("action", W.WS_F_ACTION), ("logp", W.WS_F_LOGP),
        ("reward", W.WS_F_REWARD), ("done", W.WS_F_DONE), ("wealth", W.WS_F_WEALTH)]}
    par = r.fetch_raw(W.WS_F_PARAMS, 4 * (NA + NP)).view(np.float32)
    fin = state(r, sa, ne)
    r.close()
    return out, init, fin, par


def _replay_records(out, t_init, counts, envs, par, T, limit, seed, k0=0):
    """Teacher-forced one-step replays along the kernel's own trajectory: the
    ring holds every step's pre-step state (features as the observation, wealth),
    so for each step t the oracle steps the listed envs from the recorded state
    and must reproduce the recorded draws, rewards and dones and the state
    recorded at t + 1.  A draw may differ from the oracle's only inside the tie
    band (its CDF margin below TIE); an env with such a draw is skipped at that
    step only.  The records start at step k0.  Returns the number of env-steps
    compared in full."""
    off = np.r_[0, np.cumsum(counts)]
    sa = int(off[-1])
    na = counts[envs]
    sl_a = np.concatenate([np.arange(off[e], off[e + 1]) for e in envs])
    ooff = np.r_[0, np.cumsum(na)]
    osa = int(ooff[-1])
    t_env = np.asarray(t_init, np.int32)[envs].copy()
    checked = 0
    for t in range(T):
        w0 = out["wealth"][t][sl_a]
        f0 = out["obs"][t][:, sl_a].T.astype(np.float64)
        o = oracle.econ_rollout(par[:NA], par[NA:], seed=seed, env_ids=envs, n_agents=na,
                                n_steps=1, episode_limit=limit, k0=k0 + t, wealth0=w0, feat0=f0,
                                t0=t_env, bf16_layers=ALL_BF16)
        for i, e in enumerate(envs):
            g_a, o_a = np.arange(off[e], off[e + 1]), np.arange(ooff[i], ooff[i + 1])
            g_sl, o_sl = np.r_[g_a, sa + e], np.r_[o_a, osa + i]
            assert np.array_equal(out["done"][t][g_sl], o["done"][0][o_sl]), (t, e)
            assert out["wealth"][t][sa + e] == o["wealth"][0][osa + i]
            np.testing.assert_allclose(out["obs"][t][:, sa + e], o["obs"][0][osa + i], rtol=0,
                                       atol=1e-6)
            diff = out["action"][t][g_sl] != o["action"][0][o_sl]
            amb = o["act_margin"][0][o_sl] < TIE
            assert not (diff & ~amb).any(), (t, e)   # draws differ only inside the tie band
            if diff.any():
                continue
            checked += 1
            np.testing.assert_allclose(out["logp"][t][g_sl], o["logp"][0][o_sl], rtol=TOL_BF16,
                                       atol=TOL_BF16)
            np.testing.assert_allclose(out["reward"][t][g_sl], o["reward"][0][o_sl],
                                       rtol=TOL_F32, atol=TOL_F32)
            if t + 1 < T:
                assert np.array_equal(out["wealth"][t + 1][g_a], o["wealth_out"][o_a]), (t, e)
                err = H.rel_err_rows(out["obs"][t + 1][:, g_a].T, o["feat_out"][o_a])
                assert err.max() <= TOL_F32, (t, e, err.max())
        t_env = np.where(out["done"][t][sa + envs] != 0, 0, t_env + 1).astype(np.int32)
    return checked


def test_fused_free_running_chunked_resets_deterministic(torch):
    """Drawn agent counts (many work items), episodes that end inside and across
    launches, chunking: every step of sampled envs matches a teacher-forced
    oracle replay; the run is byte-for-byte the same twice and with another
    chunk length; wealth is conserved in every env between resets."""
    T, limit, rs = 45, 20, 5
    counts = np.array([oracle.econ_agent_count(3, e) for e in range(96)], np.int32)
    out, init, fin, par = _run(counts, T, 16, limit, 3, rs)
    out2, _, fin2, _ = _run(counts, T, 16, limit, 3, rs)
    out3, _, fin3, _ = _run(counts, T, 7, limit, 3, rs)
    for f in out:
        assert out[f].tobytes() == out2[f].tobytes() == out3[f].tobytes(), f
    for a, b, c in zip(fin, fin2, fin3):
        assert np.array_equal(a, b) and np.array_equal(a, c)
    off = np.r_[0, np.cumsum(counts)]
    sa = int(off[-1])
    wr, dn = out["wealth"], out["done"]
    for e in range(96):
        tot = wr[:, off[e]:off[e + 1]].sum(1)
        assert np.array_equal(tot, wr[:, sa + e])
        same = dn[:-1, sa + e] == 0
        assert np.all(tot[1:][same] == tot[:-1][same])
    assert dn[:, sa:].sum(0).min() == 2                      # resets at steps 20 and 40
    act = out["action"]
    assert act[:, :sa].min() >= 0 and act[:, :sa].max() <= 19 and act[:, sa:].max() <= 9
    envs = np.array([0, 1, 2, 17, 40, 41, 63, 94, 95])
    assert _replay_records(out, init[2], counts, envs, par, T, limit, rs) >= len(envs) * T // 2


def test_fused_bench_launch_shape_sampled(torch):
    """The bench's launch: 2,048 envs with U{8..256} agents, one 50-step chunk
    per launch.  Conservation in every env; every step of sampled envs against
    teacher-forced oracle replays."""
    T, limit, rs = 50, 540, 11
    counts = np.array([oracle.econ_agent_count(1, e) for e in range(2048)], np.int32)
    out, init, fin, par = _run(counts, T, 50, limit, 1, rs)
    off = np.r_[0, np.cumsum(counts)]
    sa = int(off[-1])
    wr = out["wealth"]
    tot = np.add.reduceat(wr[:, :sa], off[:-1], axis=1)
    assert np.array_equal(tot, wr[:, sa:])
    assert np.all(tot == tot[:1])
    assert out["done"].sum() == 0
    envs = np.array([0, 511, 1024, 1500, 2046, 2047])
    assert _replay_records(out, init[2], counts, envs, par, T, limit, rs) >= len(envs) * T // 2
