"""GPU parity of the fused persistent landscape kernel (BF16 path): the
D-256-256-2D policy on tcgen05 with its hidden layers kept in tensor memory,
the Gaussian head, and the hi+lo energy cross-term swept in blocks of 64
Gaussians by one CTA or a CTA pair (cluster) per 128-env tile.  Compared with
the oracle in BF16-operand mode, and with the FP64 energy."""
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
D, M = 24, 4096
PW = [D, 256, 256, 2 * D]
# energy of the BF16 path relative to sum_m |a_m| e_m (hi+lo cross-term, ex2.approx)
ENERGY_TOL = 5e-3
FIELDS = (W.WS_F_OBS, W.WS_F_ACTION, W.WS_F_LOGP, W.WS_F_REWARD, W.WS_F_DONE, W.WS_F_ENERGY)


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


def land(n, ring, limit, seed=1, dim=D, **kw):
    return W.Rollout(W.WS_ENV_LANDSCAPE, BF16, n, ring, limit, 256, 256, dim=dim, n_gauss=M,
                     param_seed=seed, **kw)


def energy_close(E_gpu, c, w, a, x):
    E = oracle.landscape_energy(c, w, a, x)
    sc = oracle.landscape_energy_scale(c, w, a, x)
    return abs(E_gpu - E) <= ENERGY_TOL * max(sc, 1e-3) + 1e-6, (E_gpu, E, sc)


@pytest.mark.parametrize("tile_ctas", [1, 2])
def test_fused_one_step_replay(torch, tile_ctas):
    n = 300                                     # three tiles, the last one ragged
    g = inputs.rng(71)
    c, wd, am = inputs.landscape_params(g, M, D)
    x0, eobs0, t0 = inputs.landscape_state(g, n, D)
    x0[:40] = (c[:40] + g.normal(0, 0.3, (40, D))).astype(np.float32)
    t0[40:50] = 999                             # these envs reset in this step
    params = inputs.policy_params(g, PW)
    r = land(n, 8, 1000, flags=W.WS_FLAG_DEBUG_LOGITS)
    r.set_launch(tile_ctas=tile_ctas)
    r.load_raw(W.WS_F_ENV_PARAMS, np.concatenate([c.astype(np.float32).ravel(),
                                                  wd.astype(np.float32), am.astype(np.float32)]))
    r.load_raw(W.WS_F_PARAMS, params)
    k0 = 5
    r.load_raw(W.WS_F_STATE, H.pack_landscape_state(x0, eobs0, t0), k=k0)
    r.step()
    r.sync()
    out = r.fetch_raw(W.WS_F_LOGITS, 4 * n * 2 * D).view(np.float32).reshape(n, 2 * D)
    o_out = oracle.mlp_forward(PW, params, x0, bf16_layers=ALL_BF16)
    err = np.abs(out - o_out).max(1) / np.maximum(np.abs(o_out).max(1), 1.0)
    assert err.max() <= TOL_BF16, err.max()
    rec = {f: r.fetch(f, k0, 1)[0] for f in FIELDS}
    x1, e1, t1 = H.unpack_landscape_state(r.fetch_raw(W.WS_F_STATE, 4 * D * n + 8 * n), n, D)
    np.testing.assert_array_equal(rec[W.WS_F_OBS].T, x0.astype(np.float32))
    for e in range(n):
        z = oracle.landscape_action_normals(1, k0, e, D)
        dx_o, lp_o = oracle.gaussian_action(out[e].astype(np.float64), z, 0.1)
        dx = rec[W.WS_F_ACTION][:, e].astype(np.float64)
        # dx from the kernel's own logits: only the FP32 head arithmetic differs
        np.testing.assert_allclose(dx, dx_o, rtol=0, atol=1e-6)
        assert abs(rec[W.WS_F_LOGP][e] - lp_o) <= TOL_F32 * max(1.0, abs(lp_o))
        x2 = x0[e] + dx.astype(np.float32).astype(np.float64)
        ok, info = energy_close(rec[W.WS_F_ENERGY][e], c, wd, am, x2.astype(np.float32))
        assert ok, (e, info)
        eobs2 = rec[W.WS_F_ENERGY][e] + 0.05 * oracle.landscape_noise(1, k0, e, 0)
        assert abs(rec[W.WS_F_REWARD][e] - (eobs0[e] - eobs2)) <= 1e-5 * max(1.0, abs(eobs2))
        done = t0[e] + 1 >= 1000
        assert rec[W.WS_F_DONE][e] == done
        if done:
            xr = oracle.landscape_reset_draw(1, k0, e, D)
            np.testing.assert_array_equal(x1[e], xr.astype(np.float32).astype(np.float64))
            ok, info = energy_close(e1[e] - 0.05 * oracle.landscape_noise(1, k0, e, 1), c, wd, am, xr)
            assert ok, (e, info)
            assert t1[e] == 0
        else:
            np.testing.assert_array_equal(x1[e], (x0[e].astype(np.float32) + dx.astype(np.float32)))
            assert t1[e] == t0[e] + 1
            assert abs(e1[e] - eobs2) <= 1e-6 * max(1.0, abs(eobs2))
    r.close()


def _run(n, T, limit, chunk, tile_ctas, seed=3, rs=4):
    r = land(n, T, limit, seed=seed, chunk_steps=chunk)
    r.set_launch(tile_ctas=tile_ctas)
    r.reset(rs)
    init = H.unpack_landscape_state(r.fetch_raw(W.WS_F_STATE, 4 * D * n + 8 * n), n, D)
    r.rollout(T)
    r.sync()
    rec = {f: r.fetch(f, 0, T) for f in FIELDS}
    par = r.fetch_raw(W.WS_F_PARAMS, 4 * oracle.policy_param_count(PW)).view(np.float32).copy()
    envp = r.fetch_raw(W.WS_F_ENV_PARAMS, 4 * (M * D + 2 * M)).view(np.float32)
    c = envp[:M * D].reshape(M, D).astype(np.float64)
    w, a = envp[M * D:M * D + M].astype(np.float64), envp[M * D + M:].astype(np.float64)
    r.close()
    return rec, init, par, (c, w, a)


def test_fused_chunks_tile_ctas_determinism(torch):
    """Chunk length changes nothing; a CTA pair per tile changes only the
    grouping of the energy sum (trajectories and draws are bit-identical, since
    the state moves by dx alone); runs are deterministic."""
    n, T, limit = 600, 30, 12
    a, _, _, _ = _run(n, T, limit, 50, 2)
    b, _, _, _ = _run(n, T, limit, 7, 2)
    c1, _, _, _ = _run(n, T, limit, 50, 2)
    s1, _, _, _ = _run(n, T, limit, 50, 1)
    for f in FIELDS:
        assert a[f].tobytes() == b[f].tobytes() == c1[f].tobytes(), f
    for f in (W.WS_F_OBS, W.WS_F_ACTION, W.WS_F_LOGP, W.WS_F_DONE):
        assert a[f].tobytes() == s1[f].tobytes(), f
    for f in (W.WS_F_ENERGY, W.WS_F_REWARD):
        assert np.abs(a[f] - s1[f]).max() <= 1e-5 * max(1.0, np.abs(a[f]).max()), f
    assert a[W.WS_F_DONE].sum(1).tolist() == [n if t in (11, 23) else 0 for t in range(T)]


def _teacher_forced(rec, init, par, cwa, envs, T, limit, rs, k0=0):
    """Each step of the listed envs from the recorded pre-step state: the
    oracle's BF16-operand policy and head give the action, the FP64 energy at the
    kernel's own x + dx bounds its energy, and the recorded next state is x + dx
    or the Philox reset draw.  The records start at step k0 from the state
    ``init`` (x, observed energy, episode counters)."""
    c, w, a = cwa
    x_t = rec[W.WS_F_OBS]                      # [T][D][n]
    eobs = init[1].copy()
    t_ep = np.asarray(init[2], np.int64).copy()
    for s in range(T):
        t = k0 + s
        for e in envs:
            x = x_t[s][:, e].astype(np.float64)
            out = oracle.mlp_forward(PW, par, x, bf16_layers=ALL_BF16)
            z = oracle.landscape_action_normals(rs, t, e, D)
            dx_o, lp_o = oracle.gaussian_action(out, z, 0.1)
            dx = rec[W.WS_F_ACTION][s][:, e].astype(np.float64)
            assert np.abs(dx - dx_o).max() <= 2e-2, (t, e)       # BF16 logits through the head
            assert abs(rec[W.WS_F_LOGP][s][e] - lp_o) <= 0.5, (t, e)
            x2 = (x_t[s][:, e] + rec[W.WS_F_ACTION][s][:, e]).astype(np.float32)
            E = rec[W.WS_F_ENERGY][s][e]
            ok, info = energy_close(E, c, w, a, x2)
            assert ok, (t, e, info)
            eobs2 = E + 0.05 * oracle.landscape_noise(rs, t, e, 0)
            assert abs(rec[W.WS_F_REWARD][s][e] - (eobs[e] - eobs2)) <= 2e-5 * max(1.0, abs(eobs2))
            done = t_ep[e] + 1 >= limit
            t_ep[e] = 0 if done else t_ep[e] + 1
            assert rec[W.WS_F_DONE][s][e] == done
            if s + 1 < T:
                nxt = x_t[s + 1][:, e]
                if done:
                    xr = oracle.landscape_reset_draw(rs, t, e, D)
                    np.testing.assert_array_equal(nxt, xr.astype(np.float32))
                else:
                    np.testing.assert_array_equal(nxt, x2)
            if done:
                xr = oracle.landscape_reset_draw(rs, t, e, D)
                E0 = oracle.landscape_energy(c, w, a, xr)
                eobs[e] = E0 + 0.05 * oracle.landscape_noise(rs, t, e, 1)
            else:
                eobs[e] = eobs2


def test_fused_multi_step_teacher_forced(torch):
    n, T, limit = 256, 24, 10
    rec, init, par, cwa = _run(n, T, limit, 16, 2)
    # the reward carries the observed energy forward: the reset energies enter
    # through eobs, whose FP64 value the comparison uses (ENERGY_TOL covers it)
    _teacher_forced(rec, init, par, cwa, [0, 1, 130, 255], T, limit, 4)


def test_fused_bench_launch_shape(torch):
    """The bench's launch: 8,192 envs, one 50-step chunk, a CTA pair per tile.
    Every env moves by exactly its recorded dx; sampled envs step by step
    against the oracle."""
    n, T = 8192, 50
    rec, init, par, cwa = _run(n, T, 1000, 50, 2, seed=1, rs=11)
    x = rec[W.WS_F_OBS]
    assert np.array_equal(x[1:], (x[:-1] + rec[W.WS_F_ACTION][:-1]).astype(np.float32))
    assert rec[W.WS_F_DONE].sum() == 0
    assert np.all(np.abs(rec[W.WS_F_ACTION]) <= np.float32(0.1))
    _teacher_forced(rec, init, par, cwa, [0, 4097, 8191], T, 1000, 11)


@pytest.mark.parametrize("tile_ctas", [1, 2])
def test_fused_energy_target_terminal(torch, tile_ctas):
    """Episodes end on reaching the energy target (the product basin) as well
    as at the step limit: every done flag against the FP64 energy of the
    recorded post-step state (decisions within the BF16 energy error of the
    target may go either way), every reset against its Philox draw."""
    n, T, limit, target = 256, 24, 1000, -0.005
    r = land(n, T, limit, seed=3, chunk_steps=10, energy_target=target)
    r.set_launch(tile_ctas=tile_ctas)
    r.reset(4)
    r.rollout(T)
    r.sync()
    obs, act, dn = (r.fetch(f, 0, T) for f in (W.WS_F_OBS, W.WS_F_ACTION, W.WS_F_DONE))
    envp = r.fetch_raw(W.WS_F_ENV_PARAMS, 4 * (M * D + 2 * M)).view(np.float32)
    c = envp[:M * D].reshape(M, D).astype(np.float64)
    w, a = envp[M * D:M * D + M].astype(np.float64), envp[M * D + M:].astype(np.float64)
    r.close()
    n_target, n_band = H.check_landscape_dones(obs, act, dn, (c, w, a), limit, target, 4,
                                               ENERGY_TOL)
    assert n_target >= 20 and n_band <= 0.05 * n * T, (n_target, n_band)
