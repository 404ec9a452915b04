"""The allocation-free policy forward (ws_policy_forward_noalloc).

Callers that cannot call cudaMalloc (code running under CUDA-graph capture,
hosts whose allocator forbids foreign allocations, fixed-memory embedded
runtimes) use this entry point: it keeps its hidden activations in a
library-owned static device array.  Its output must equal the logits the
regular plain-FP32 step computes with its own scratch (ws_step, then ws_fetch
of LOGITS), call after call, even though every call reuses the same array:
bit for bit (both run the same FP32 layer kernel in the same summation order),
and within the FP32 tolerance of the oracle's FP64 forward pass.
This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

import oracle
from paper_2408_00930_gb300 import inputs
from paper_2408_00930_gb300 import warpsci as W
from tests import ws_helpers as H
from tests.gpu_common import TOL_F32, control_rollout, need_gpu

pytestmark = pytest.mark.gpu


def _logits_from_step(params, s0, t0, h):
    """Logits the existing entry points compute: ws_load, ws_step, ws_fetch(LOGITS)."""
    n = len(s0)
    r = control_rollout(W.WS_PATH_PLAIN_FP32, n, 4, 200, h, h)
    r.load_raw(W.WS_F_PARAMS, params)
    r.load_raw(W.WS_F_STATE, H.pack_control_state(s0, t0), k=0)
    r.step()
    r.sync()
    out = r.fetch_raw(W.WS_F_LOGITS, 8 * n).view(np.float32).reshape(n, 2).copy()
    r.close()
    return out


def test_noalloc_forward_matches_step_logits_twice():
    torch = need_gpu()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    g = inputs.rng(99)
    # two calls in a row with different sizes and inputs: stale array contents
    # from the first call must not leak into the second
    for n, h in [(1500, 64), (700, 128)]:
        params = inputs.policy_params(g, [4, h, h, 2], scale=2.0)
        s0, t0 = inputs.control_states(g, n)
        ref = _logits_from_step(params, s0, t0, h)
        obs = torch.from_numpy(np.ascontiguousarray(s0.astype(np.float32))).to(dev)
        p = torch.from_numpy(params).to(dev)
        out = torch.full((n, 2), float("nan"), dtype=torch.float32, device=dev)
        st = W.ws_policy_forward_noalloc(obs.data_ptr(), n, p.data_ptr(), 4, h, h, 2,
                                         out.data_ptr(), stream.cuda_stream)
        assert st == W.WS_OK
        torch.cuda.synchronize(dev)
        got = out.cpu().numpy()
        err = np.abs(got - ref) / np.maximum(np.abs(ref), 1.0)
        assert np.all(np.isfinite(got))
        assert err.max() <= TOL_F32, err.max()
        assert np.array_equal(got, ref)
        o = oracle.mlp_forward([4, h, h, 2], params, s0.astype(np.float32).astype(np.float64))
        assert H.rel_err_rows(got, o).max() <= TOL_F32


def test_noalloc_rejects_requests_beyond_the_static_array():
    torch = need_gpu()
    dev = torch.device("cuda", 0)
    x = torch.zeros(16, dtype=torch.float32, device=dev)
    # 40,000 rows x (64 + 64) = 5.12 M floats > 4,194,304: refused before any launch
    st = W.ws_policy_forward_noalloc(x.data_ptr(), 40_000, x.data_ptr(), 4, 64, 64, 2,
                                     x.data_ptr(), 0)
    assert st == W.WS_ERR_RANGE
    assert W.ws_policy_forward_noalloc(None, 1, x.data_ptr(), 4, 8, 8, 2, x.data_ptr(), 0) == \
        W.WS_ERR_INVALID
