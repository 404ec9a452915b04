"""GPU parity of the landscape force F = -grad E(x') (ws_forces, FORCE field)
against the oracle's analytic gradient (itself pinned to central differences)
at the post-step states recorded in the ring, on every path."""
import numpy as np
import pytest

import oracle
from paper_2408_00930_gb300 import warpsci as W
from tests.gpu_common import need_gpu

pytestmark = pytest.mark.gpu
# FP32 sums over M Gaussians, tile partials added once per 64 Gaussians
TOL_FORCE_F32 = 2e-5
# BF16 tensor-core path: the exponents carry the energy sweep's hi+lo error
# (~5e-3 of a term, as the energy), P and the force image are split hi + lo,
# and the force is formed as y sum(p) - sum(p c): the error is measured against
# sum_m |a_m| e_m (|y_j| + |c_mj|) / w_m^2, the size of the terms of that form
TOL_FORCE_BF16 = 5e-3


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


def force_scale(c, w, a, y, split=False):
    """sum_m |a_m| e_m |y_j - c_mj| / w_m^2 per coordinate (the size of the
    terms of the direct form), or with split sum_m |a_m| e_m (|y_j| + |c_mj|) /
    w_m^2 (the terms of y sum(p) - sum(p c))."""
    d = y[None, :] - c
    e = np.exp(-(d * d).sum(1) / (2 * w * w))
    size = np.abs(y[None, :]) + np.abs(c) if split else np.abs(d)
    return ((np.abs(a) * e / (w * w))[:, None] * size).sum(0)


def env_params(r, M, D):
    envp = r.fetch_raw(W.WS_F_ENV_PARAMS, 4 * (M * D + 2 * M)).view(np.float32)
    c = envp[:M * D].reshape(M, D).astype(np.float64)
    return c, envp[M * D:M * D + M].astype(np.float64), envp[M * D + M:].astype(np.float64)


def check_forces(r, T, M, D, rows, tol, split=False):
    obs, act, F = (r.fetch(f, 0, T) for f in (W.WS_F_OBS, W.WS_F_ACTION, W.WS_F_FORCE))
    c, w, a = env_params(r, M, D)
    worst = 0.0
    for t, e in rows:
        y = (obs[t][:, e] + act[t][:, e]).astype(np.float32).astype(np.float64)
        ref = -oracle.landscape_grad(c, w, a, y)
        sc = np.maximum(force_scale(c, w, a, y, split), 1e-3)
        err = np.abs(F[t][:, e] - ref) / sc
        worst = max(worst, err.max())
        assert err.max() <= tol, (t, e, err.max())
    return worst


@pytest.mark.parametrize("path", [W.WS_PATH_PLAIN_FP32, W.WS_PATH_BATCHED_FP32,
                                  W.WS_PATH_BATCHED_BF16])
def test_forces_match_oracle_gradient(torch, path):
    D, M, n, T = 24, 4096, 300, 12
    r = W.Rollout(W.WS_ENV_LANDSCAPE, path, n, T, 7, 256, 256, dim=D, n_gauss=M, param_seed=5,
                  flags=W.WS_FLAG_FORCE, chunk_steps=5)
    r.reset(9)
    r.rollout(T)
    r.forces(T)
    r.sync()
    g = np.random.default_rng(0)
    rows = [(t, int(e)) for t in range(T) for e in g.choice(n, 6, replace=False)]
    rows += [(6, 0), (6, n - 1)]          # steps that end an episode: the pre-reset x'
    bf16 = path == W.WS_PATH_BATCHED_BF16
    worst = check_forces(r, T, M, D, rows, TOL_FORCE_BF16 if bf16 else TOL_FORCE_F32, split=bf16)
    r.close()
    if bf16:
        assert worst > 1e-7          # the tensor-core kernel ran (not the FP32 one)


def test_forces_tc_near_centres_and_all_rows(torch):
    """BF16 tensor-core force: states placed near Gaussian centres (large,
    cancelling terms), several 128-row tiles with a ragged tail, D = 8 and 16
    as well as 24, every row compared."""
    for D, n, T in ((24, 200, 3), (16, 130, 2), (8, 70, 4)):
        M = 1000
        g = np.random.default_rng(D)
        r = W.Rollout(W.WS_ENV_LANDSCAPE, W.WS_PATH_BATCHED_BF16, n, T, 1000, 256, 256, dim=D,
                      n_gauss=M, param_seed=7, flags=W.WS_FLAG_FORCE)
        c, w, a = env_params(r, M, D)
        x0 = (c[g.integers(0, M, n)] + g.normal(0, 0.3, (n, D))).astype(np.float32)
        r.load_raw(W.WS_F_STATE, np.concatenate([np.ascontiguousarray(x0.T).view(np.uint8).ravel(),
                                                 np.zeros(n, np.float32).view(np.uint8),
                                                 np.zeros(n, np.int32).view(np.uint8)]), k=0)
        r.rollout(T)
        r.forces(T)
        r.sync()
        rows = [(t, e) for t in range(T) for e in range(n)]
        check_forces(r, T, M, D, rows, TOL_FORCE_BF16, split=True)
        r.close()


def test_forces_window_ring_wrap_and_small_dims(torch):
    """A window of the last steps over a wrapped ring; D of 8 and 40 (other
    register tiles); M not a multiple of the 64-Gaussian staging tile."""
    for D, M in ((8, 100), (40, 333)):
        n, R, T = 130, 6, 15
        r = W.Rollout(W.WS_ENV_LANDSCAPE, W.WS_PATH_BATCHED_FP32, n, R, 1000, 32, 32, dim=D,
                      n_gauss=M, param_seed=2, flags=W.WS_FLAG_FORCE)
        r.reset(3)
        r.rollout(T)
        r.forces(4)                       # steps 11..14 (ring rows 5, 0, 1, 2)
        r.sync()
        obs, act, F = (r.fetch(f, T - 4, 4) for f in (W.WS_F_OBS, W.WS_F_ACTION, W.WS_F_FORCE))
        c, w, a = env_params(r, M, D)
        for t in range(4):
            for e in (0, 64, n - 1):
                y = (obs[t][:, e] + act[t][:, e]).astype(np.float32).astype(np.float64)
                ref = -oracle.landscape_grad(c, w, a, y)
                sc = np.maximum(force_scale(c, w, a, y), 1e-3)
                assert (np.abs(F[t][:, e] - ref) / sc).max() <= TOL_FORCE_F32, (D, t, e)
        r.close()


def test_forces_errors(torch):
    r = W.Rollout(W.WS_ENV_LANDSCAPE, W.WS_PATH_PLAIN_FP32, 16, 4, 100, 16, 16, dim=8, n_gauss=16)
    r.rollout(2)
    assert W.ws_forces(r.ctx, 1) == W.WS_ERR_STATE          # no FORCE field
    r.close()
    r = W.Rollout(W.WS_ENV_LANDSCAPE, W.WS_PATH_PLAIN_FP32, 16, 4, 100, 16, 16, dim=8, n_gauss=16,
                  flags=W.WS_FLAG_FORCE)
    r.rollout(2)
    assert W.ws_forces(r.ctx, 3) == W.WS_ERR_RANGE          # only 2 steps taken
    assert W.ws_forces(r.ctx, 0) == W.WS_ERR_RANGE
    r.rollout(4)
    assert W.ws_forces(r.ctx, 5) == W.WS_ERR_RANGE          # the ring holds 4
    assert W.ws_forces(r.ctx, 4) == W.WS_OK
    r.sync()
    r.close()
