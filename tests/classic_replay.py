"""Teacher-forced replay of classic-control roll-outs (the control env and the
acrobot) against the FP64 oracle, from the records the kernel wrote.

With WS_FLAG_DEBUG_LOGITS every path records, beside each transition, the FP32
policy outputs its sampler read (the POLICY_OUT ring field).  For every step of
every listed env the replay then checks, from the recorded pre-step
observation:

* the recorded logits against the oracle's MLP on that observation (in the
  operand precision of the path);
* the recorded action against the oracle's inverse-CDF draw (softmax in FP64)
  on the recorded logits with the same Philox counter (seed; step, env, agent 0,
  ACTION), and the recorded log-probability against the oracle's;
* the env step with the recorded action: the done flag and the reward, the next
  recorded observation (the post-step state, or after a done the Philox RESET
  draw of that step, bit for bit), and at the end of the window the final state
  and episode counter the context holds.

A draw is accepted either way only when the uniform lies within ``tie`` of a
CDF boundary of the recorded logits (FP32 softmax in the kernel against FP64
here), a done flag only when the deciding quantity lies within ``done_band`` of
its threshold; both are counted and returned.
"""
import numpy as np

import oracle
from tests import ws_helpers as H

# the kernel's FP32 softmax (expf, running sums) against FP64 on the same logits
TIE_OWN = 1e-6


def fetch_cols(r, field, t0, T, ids):
    """Ring field [T][...][S] of a context, columns ``ids`` only (gathered on the
    device, so that a large ring is not copied whole to the host)."""
    torch = r.torch
    dt, shp = r._ring_spec(field)
    tdt = {np.dtype(np.float32): torch.float32, np.dtype(np.int32): torch.int32,
           np.dtype(np.uint8): torch.uint8, np.dtype(np.int64): torch.int64}[np.dtype(dt)]
    buf = torch.empty((T,) + shp, dtype=tdt, device=r.state_buf.device)
    r.fetch_device(field, t0, T, buf)
    r.sync()
    sel = buf[..., torch.as_tensor(np.asarray(ids, np.int64), device=buf.device)]
    return sel.cpu().numpy()


def records(r, t0, T, ids):
    from paper_2408_00930_gb300 import warpsci as W
    return {name: fetch_cols(r, fid, t0, T, ids) for name, fid in [
        ("obs", W.WS_F_OBS), ("action", W.WS_F_ACTION), ("logp", W.WS_F_LOGP),
        ("reward", W.WS_F_REWARD), ("done", W.WS_F_DONE), ("pout", W.WS_F_POLICY_OUT)]}


def mlp_rows(widths, params, X, bf16_layers, workers=8):
    """oracle.mlp_forward over the rows of X, split across threads (the C call
    releases the interpreter lock)."""
    from concurrent.futures import ThreadPoolExecutor
    parts = [p for p in np.array_split(X, workers) if len(p)]
    with ThreadPoolExecutor(len(parts)) as ex:
        outs = list(ex.map(lambda p: np.atleast_2d(
            oracle.mlp_forward(widths, params, p, bf16_layers=bf16_layers)), parts))
    return np.concatenate(outs)


def action_uniforms(seed, k, ids):
    ctr = np.zeros((len(ids), 4), np.uint32)
    ctr[:, 0] = k & 0xFFFFFFFF
    ctr[:, 1] = np.asarray(ids, np.uint32)
    ctr[:, 3] = oracle.TAG_ACTION << 24
    words = oracle.philox(ctr, oracle.seed_key(seed))
    return [oracle.u01(int(w)) for w in words[:, 0]]


def acrobot_state_from_obs(o):
    """(th1, th2, w1, w2) from a recorded observation (cos, sin, cos, sin, w1, w2)."""
    return np.array([np.arctan2(o[1], o[0]), np.arctan2(o[3], o[2]), o[4], o[5]])


def replay(env, rec, ids, params, widths, seed, limit, bf16_layers, tol_logits, s_final,
           t_final, k0=0, t_init=None, tol_state=1e-5, tie=TIE_OWN, done_band=1e-5,
           height_band=1e-4):
    """Replay every step of envs ``ids`` (see the module docstring).  ``rec``
    holds [T][...][n] records (``records``); ``s_final`` [n][4] and ``t_final``
    [n] the context's state after the window.  Returns counts of the compared
    env-steps, the draws in the tie band, the done decisions in the band and the
    episodes that ended inside the window."""
    acro = env == "acrobot"
    T, n = rec["action"].shape
    t_env = np.zeros(n, np.int64) if t_init is None else np.asarray(t_init, np.int64).copy()
    c = dict(steps=0, tie=0, done_band=0, dones=0, logit_err=0.0, state_err=0.0)
    for s in range(T):
        k = k0 + s
        X = rec["obs"][s].T.astype(np.float64)           # [n][obs_dim] pre-step observations
        lg = rec["pout"][s].T.astype(np.float64)         # [n][n_act] the sampler's logits
        o_lg = mlp_rows(widths, params, X, bf16_layers)
        err = H.rel_err_rows(lg, o_lg)
        assert err.max() <= tol_logits, (s, int(ids[int(err.argmax())]), float(err.max()))
        c["logit_err"] = max(c["logit_err"], float(err.max()))
        us = action_uniforms(seed, k, ids)
        for i, e in enumerate(ids):
            a = int(rec["action"][s][i])
            a_o, lp_o, mg = oracle.sample_categorical(lg[i], us[i])
            if mg < tie:
                c["tie"] += 1
                assert a in (a_o - 1, a_o, a_o + 1), (s, e)
            else:
                assert a == a_o, (s, e, a, a_o, mg)
                assert abs(rec["logp"][s][i] - lp_o) <= 1e-5 * max(1.0, abs(lp_o)), (s, e)
            # the env step from the recorded state with the recorded action
            if acro:
                st = acrobot_state_from_obs(X[i])
                nxt, raw = oracle.acrobot_step(st, a)
                term, hm = oracle.acrobot_terminal(nxt)
                ambiguous = hm < height_band
                done_o = term or t_env[i] + 1 >= limit
                scale = max(1.0, float(np.abs(raw).max()))
            else:
                nxt = oracle.control_dynamics(X[i], a)
                done_o, dm = oracle.control_done(nxt, int(t_env[i] + 1), limit)
                term = done_o and t_env[i] + 1 < limit
                ambiguous = dm < done_band and t_env[i] + 1 < limit
                scale = 1.0
            dn = bool(rec["done"][s][i])
            if ambiguous:
                c["done_band"] += 1
            else:
                assert dn == done_o, (s, e, dn, done_o)
                if acro:
                    assert rec["reward"][s][i] == (0.0 if term else -1.0), (s, e)
            if not acro:
                assert rec["reward"][s][i] == 1.0
            last = s + 1 == T
            if dn:
                c["dones"] += 1
                t_env[i] = 0
                if acro:
                    reset = oracle.acrobot_reset_draw(seed, k, e).astype(np.float32)
                    if last:
                        np.testing.assert_array_equal(s_final[i], reset)
                    else:
                        o_next = rec["obs"][s + 1][:, i]
                        np.testing.assert_array_equal(o_next[4:], reset[2:])
                        np.testing.assert_allclose(acrobot_state_from_obs(o_next.astype(np.float64)),
                                                   reset, rtol=0, atol=2e-6)
                else:
                    reset = oracle.control_reset_draw(seed, k, e).astype(np.float32)
                    got = s_final[i] if last else rec["obs"][s + 1][:, i]
                    np.testing.assert_array_equal(got, reset)
            else:
                t_env[i] += 1
                if acro:
                    if last:
                        d = np.asarray(s_final[i], np.float64) - nxt
                        d[:2] = (d[:2] + np.pi) % (2 * np.pi) - np.pi   # angles modulo 2 pi
                    else:
                        d = rec["obs"][s + 1][:, i].astype(np.float64) - oracle.acrobot_obs(nxt)
                    e_rel = float(np.abs(d).max()) / scale
                else:
                    got = s_final[i] if last else rec["obs"][s + 1][:, i]
                    e_rel = float(H.rel_err_rows(np.asarray(got, np.float64)[None], nxt[None])[0])
                assert e_rel <= tol_state, (s, e, e_rel)
                c["state_err"] = max(c["state_err"], e_rel)
            c["steps"] += 1
    np.testing.assert_array_equal(t_env, np.asarray(t_final, np.int64))
    return c
