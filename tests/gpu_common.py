"""Shared fixtures/rules of the GPU parity tests (all marked gpu)."""
import numpy as np
import pytest

from paper_2408_00930_gb300 import warpsci as W

# FP32 path tolerances: relative float error per env (‖g-o‖∞ / max(‖o‖∞, 1)),
# the tie band of the categorical decision (|u - CDF_i| below it -> either
# neighbouring action is accepted) and the relative band around a done threshold.
TOL_F32 = 1e-5
# Free-running multi-step comparisons: the per-step error (pinned at TOL_F32 by
# the one-step replays) compounds through the unstable pole dynamics within an
# episode (growth ~ (1 + dt sqrt(9.8)) per step); actions and dones are still
# compared bit-exactly, so a real divergence cannot hide inside this band.
TOL_F32_FREE = 1e-3
TIE_F32 = 1e-5
DONE_BAND_F32 = 1e-5
# BF16 tensor-core path: logits carry bfloat16 operand rounding (8-bit mantissa).
TOL_BF16 = 2e-2
TIE_BF16 = 2e-2
DONE_BAND_BF16 = 2e-3


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_00930_gb300 import build
    build.build()
    W.lib()
    return torch


def control_rollout(path, n_envs, ring, limit, h0, h1, seed=1, **kw):
    return W.Rollout(W.WS_ENV_CONTROL, path, n_envs, ring, limit, h0, h1, param_seed=seed, **kw)
