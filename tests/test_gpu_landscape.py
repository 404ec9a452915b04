"""GPU parity of the reaction-path landscape (plain and graph-batched FP32 paths)."""
import numpy as np
import pytest

import oracle
from paper_2408_00930_gb300 import inputs
from paper_2408_00930_gb300 import warpsci as W
from tests import ws_helpers as H
from tests.gpu_common import TOL_F32, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


def land(path, n, D=24, M=4096, ring=8, limit=1000, seed=1, h=(256, 256), **kw):
    return W.Rollout(W.WS_ENV_LANDSCAPE, path, n, ring, limit, *h, dim=D, n_gauss=M,
                     param_seed=seed, **kw)


def test_landscape_init_and_reset(torch):
    D, M, n = 24, 4096, 300
    r = land(W.WS_PATH_PLAIN_FP32, n, seed=21)
    raw = r.fetch_raw(W.WS_F_ENV_PARAMS, 4 * (M * D + 2 * M))
    c = raw[:4 * M * D].view(np.float32).reshape(M, D)
    wd = raw[4 * M * D:4 * M * D + 4 * M].view(np.float32)
    am = raw[4 * M * D + 4 * M:].view(np.float32)
    co, wo, ao = oracle.landscape_init(21, D, M)
    np.testing.assert_array_equal(c, co.astype(np.float32))
    np.testing.assert_allclose(wd, wo, rtol=2e-6)
    np.testing.assert_allclose(am, ao, rtol=0, atol=2e-6)
    x, eobs, t = H.unpack_landscape_state(r.fetch_raw(W.WS_F_STATE, 4 * D * n + 8 * n), n, D)
    for e in (0, 151, n - 1):
        np.testing.assert_array_equal(x[e], oracle.landscape_reset_draw(21, oracle.STEP_INIT, e, D))
        # the GPU keeps FP32 copies of the landscape; the oracle evaluates them in FP64
        E = oracle.landscape_energy(c.astype(np.float64), wd.astype(np.float64), am.astype(np.float64), x[e])
        sc = oracle.landscape_energy_scale(c.astype(np.float64), wd.astype(np.float64), am.astype(np.float64), x[e])
        ref = E + 0.05 * oracle.landscape_noise(21, oracle.STEP_INIT, e, 1)
        assert abs(eobs[e] - ref) <= 1e-5 * max(sc, 1e-3) + 1e-7
    assert np.all(t == 0)
    r.close()


@pytest.mark.parametrize("path", [W.WS_PATH_PLAIN_FP32, W.WS_PATH_BATCHED_FP32])
def test_one_step_replay_seeded(torch, path):
    """Seeded landscape, policy and states: one step against the oracle."""
    D, M, n, h = 24, 4096, 333, (256, 256)
    g = inputs.rng(31)
    c, wd, am = inputs.landscape_params(g, M, D)
    # put a few states near centres so the energies are not all negligible
    x0, eobs0, t0 = inputs.landscape_state(g, n, D)
    x0[:40] = (c[:40] + g.normal(0, 0.3, (40, D))).astype(np.float32)
    t0[:10] = 999
    params = inputs.policy_params(g, [D, *h, 2 * D])
    r = land(path, n)
    r.load_raw(W.WS_F_ENV_PARAMS, np.concatenate([c.astype(np.float32).ravel(),
                                                  wd.astype(np.float32), am.astype(np.float32)]))
    r.load_raw(W.WS_F_PARAMS, params)
    k0 = 5
    r.load_raw(W.WS_F_STATE, H.pack_landscape_state(x0, eobs0, t0), k=k0)
    r.step()
    r.sync()
    act = r.fetch(W.WS_F_ACTION, k0, 1)[0].T.astype(np.float64)
    lp = r.fetch(W.WS_F_LOGP, k0, 1)[0]
    rew = r.fetch(W.WS_F_REWARD, k0, 1)[0]
    en = r.fetch(W.WS_F_ENERGY, k0, 1)[0]
    dn = r.fetch(W.WS_F_DONE, k0, 1)[0]
    x1, e1, t1 = H.unpack_landscape_state(r.fetch_raw(W.WS_F_STATE, 4 * D * n + 8 * n), n, D)
    o = oracle.landscape_rollout(c, wd, am, params, *h, seed=1, env_ids=np.arange(n), n_steps=1,
                                 episode_limit=1000, k0=k0, x0=x0, eobs0=eobs0, t0=t0)
    np.testing.assert_allclose(act, o["act"][0], rtol=0, atol=1e-6)
    np.testing.assert_allclose(lp, o["logp"][0], rtol=TOL_F32, atol=1e-5)
    sc = o["energy_scale"][0]
    assert np.all(np.abs(en - o["energy"][0]) <= TOL_F32 * np.maximum(sc, 1e-3) + 1e-7)
    assert np.all(np.abs(rew - o["reward"][0]) <= TOL_F32 * np.maximum(sc, 1e-3) + 1e-6)
    assert list(dn) == list(o["done"][0]) and dn[:10].all() and not dn[10:].any()
    err = H.rel_err_rows(x1, o["x"])
    assert err.max() <= TOL_F32, err.max()
    np.testing.assert_allclose(e1, o["eobs"], rtol=0, atol=1e-5)
    assert np.array_equal(t1, o["t"])
    # near-centre states really exercise the energy (not all ~0)
    assert np.abs(o["energy"][0][:40]).max() > 1e-3
    r.close()


def test_multi_step_with_reset(torch):
    D, M, n, h = 8, 64, 100, (32, 32)
    r = land(W.WS_PATH_BATCHED_FP32, n, D=D, M=M, ring=25, limit=10, seed=6, h=h, chunk_steps=6)
    r.reset(12)
    r.rollout(25)
    r.sync()
    obs = r.fetch(W.WS_F_OBS, 0, 25)
    act = r.fetch(W.WS_F_ACTION, 0, 25)
    dn = r.fetch(W.WS_F_DONE, 0, 25)
    raw = r.fetch_raw(W.WS_F_ENV_PARAMS, 4 * (M * D + 2 * M))
    c = raw[:4 * M * D].view(np.float32).reshape(M, D).astype(np.float64)
    wd = raw[4 * M * D:4 * M * D + 4 * M].view(np.float32).astype(np.float64)
    am = raw[4 * M * D + 4 * M:].view(np.float32).astype(np.float64)
    params = oracle.policy_init(6, 0, [D, *h, 2 * D])
    o = oracle.landscape_rollout(c, wd, am, params, *h, seed=12, env_ids=np.arange(n), n_steps=25,
                                 episode_limit=10)
    assert np.array_equal(dn, o["done"])
    np.testing.assert_allclose(obs.transpose(0, 2, 1), o["obs"], rtol=0, atol=1e-4)
    np.testing.assert_allclose(act.transpose(0, 2, 1), o["act"], rtol=0, atol=1e-4)
    # right after each reset the state is the exact Philox draw
    np.testing.assert_array_equal(obs[10].T, o["obs"][10].astype(np.float32))
    np.testing.assert_array_equal(obs[20].T, o["obs"][20].astype(np.float32))
    r.close()


def test_graph_path_bytes_equal_plain_path(torch):
    out = []
    for path in (W.WS_PATH_PLAIN_FP32, W.WS_PATH_BATCHED_FP32):
        r = land(path, 50, D=12, M=256, ring=14, limit=9, seed=3, h=(64, 64), chunk_steps=5)
        r.rollout(14)
        out.append([r.fetch(f, 0, 14).tobytes() for f in (W.WS_F_ACTION, W.WS_F_ENERGY,
                                                          W.WS_F_OBS, W.WS_F_REWARD)])
        r.close()
    assert out[0] == out[1]


@pytest.mark.parametrize("path", [W.WS_PATH_PLAIN_FP32, W.WS_PATH_BATCHED_FP32])
def test_energy_target_terminal(torch, path):
    """Episodes end at the step limit or on reaching the energy target (the
    product basin); every done flag against the FP64 energy of the recorded
    post-step state, every reset against its Philox draw."""
    D, M, n, h, T, limit = 8, 64, 120, (32, 32), 40, 30
    r = land(path, n, D=D, M=M, ring=T, limit=limit, seed=6, h=h, chunk_steps=7,
             energy_target=-0.01)
    r.reset(13)
    r.rollout(T)
    r.sync()
    obs, act, dn = (r.fetch(f, 0, T) for f in (W.WS_F_OBS, W.WS_F_ACTION, W.WS_F_DONE))
    raw = r.fetch_raw(W.WS_F_ENV_PARAMS, 4 * (M * D + 2 * M))
    c = raw[:4 * M * D].view(np.float32).reshape(M, D).astype(np.float64)
    wd = raw[4 * M * D:4 * M * D + 4 * M].view(np.float32).astype(np.float64)
    am = raw[4 * M * D + 4 * M:].view(np.float32).astype(np.float64)
    n_target, n_band = H.check_landscape_dones(obs, act, dn, (c, wd, am), limit, -0.01, 13,
                                               TOL_F32)
    assert n_target >= 5 and n_band <= 2, (n_target, n_band)
    r.close()
