"""The returns scan (S7) on every kernel variant against the oracle's FP64 scan
of the same recorded rewards and done flags: the segmented scan of rings with
few slots (8,192 slots x 1,000 steps, the landscape's shape, and a window that
crosses the ring's end), the float4 scan of many slots, the scalar scan of a
slot count that is not a multiple of four.  Errors relative to the discounted
sum of |r| (the scale of the return), within the 1e-6 the float-float scan
promises at horizons up to 1,000."""
import numpy as np
import pytest

import oracle
from paper_2408_00930_gb300 import warpsci as W
from tests.gpu_common import need_gpu

pytestmark = pytest.mark.gpu
GAMMA = float(np.float32(0.99))


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


@pytest.mark.parametrize("n_envs,ring,run,window,limit", [
    (8192, 1000, 1000, 1000, 1000),   # segmented scan, landscape shape, one episode
    (8192, 600, 1350, 600, 137),      # segmented scan over a window crossing the ring end
    (3000, 300, 300, 300, 40),        # segmented, a ragged last block of slots
    (40000, 120, 120, 120, 30),       # float4 scan (many slots, a multiple of four)
    (40001, 100, 100, 100, 30),       # scalar scan
])
def test_returns_scan_against_fp64(torch, n_envs, ring, run, window, limit):
    # the acrobot's rewards (-1, and 0 on a terminal step) vary per env and step
    r = W.Rollout(W.WS_ENV_ACROBOT, W.WS_PATH_BATCHED_BF16, n_envs, ring, limit, 64, 64,
                  param_seed=3, chunk_steps=50)
    r.reset(5)
    r.rollout(run)
    r.returns(window)
    r.sync()
    k0 = run - window
    rew = r.fetch(W.WS_F_REWARD, k0, window).astype(np.float64)
    dn = r.fetch(W.WS_F_DONE, k0, window)
    G = r.fetch(W.WS_F_RETURN, k0, window).astype(np.float64)
    cols = np.unique(np.r_[0:64, n_envs - 64:n_envs, np.arange(0, n_envs, 97)])
    Go = oracle.returns(rew[:, cols], dn[:, cols], GAMMA)
    scale = oracle.returns(np.abs(rew[:, cols]), dn[:, cols], GAMMA)
    err = np.abs(G[:, cols] - Go) / np.maximum(scale, 1.0)
    assert err.max() <= 1e-6, err.max()
    assert dn.sum() > 0 or limit >= window
    r.close()
