"""WS_FLAG_BOUNDS_CHECK: every region of the state and ring buffers (each
parameter block, the env state, each scratch array, each ring field) is
followed right at its end by a 256-byte canary that ws_sync verifies.  Every
env on its batched paths (the fused BF16 kernels included) runs roll-outs,
returns and, where the flags add them, the force pass and both training
updates with all canaries intact; a one-byte overrun planted from the host just
past the end of a field (the ring's OBS field, the state's step counter) makes
ws_sync fail with WS_ERR_CUDA and a message naming the buffer and that field,
and the error sticks."""
import pytest

from paper_2408_00930_gb300 import warpsci as W
from tests.gpu_common import need_gpu

pytestmark = pytest.mark.gpu
F32, BF16 = W.WS_PATH_BATCHED_FP32, W.WS_PATH_BATCHED_BF16
BC = W.WS_FLAG_BOUNDS_CHECK


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


CASES = [
    (W.WS_ENV_CONTROL, F32, 300, 64, {}, W.WS_FLAG_TRAIN),
    (W.WS_ENV_CONTROL, BF16, 300, 256, {}, W.WS_FLAG_TRAIN),
    (W.WS_ENV_ACROBOT, BF16, 200, 64, {}, W.WS_FLAG_TRAIN),
    (W.WS_ENV_ECONOMY, BF16, 12, 128, {}, W.WS_FLAG_TRAIN),
    (W.WS_ENV_LANDSCAPE, BF16, 130, 256, dict(dim=24, n_gauss=200),
     W.WS_FLAG_TRAIN | W.WS_FLAG_FORCE),
    (W.WS_ENV_LANDSCAPE, F32, 130, 32, dict(dim=8, n_gauss=100), W.WS_FLAG_TRAIN | W.WS_FLAG_FORCE),
]


@pytest.mark.parametrize("env,path,n,h,kw,extra", CASES)
def test_canaries_intact(torch, env, path, n, h, kw, extra):
    T = 12
    r = W.Rollout(env, path, n, T, 7, h, h, flags=BC | W.WS_FLAG_DEBUG_LOGITS | extra,
                  chunk_steps=5, **kw)
    r.reset(3)
    r.rollout(T)
    r.returns(T)
    if extra & W.WS_FLAG_FORCE:
        r.forces(T)
    r.a2c_update(T, 1e-3)
    r.advantages(T)
    r.ppo_update(T, 1e-3)
    r.rollout(T + 3)                  # past the ring's end: rows wrap
    r.sync()                          # raises if a canary changed
    r.close()


@pytest.mark.parametrize("where", ["ring", "state"])
def test_overrun_past_a_field_detected(torch, where):
    n, R = 64, 8
    r = W.Rollout(W.WS_ENV_CONTROL, F32, n, R, 100, 16, 16, flags=BC)
    r.rollout(4)
    r.sync()
    if where == "ring":
        # OBS is the ring's first field: [R][4][n] f32 from byte 0; one byte past it
        r.ring_buf[R * 4 * n * 4 + 3].fill_(0)
        field = "OBS"
    else:
        # the step counter is the state's first region (8 bytes)
        r.state_buf[8].fill_(0x5A)
        field = "step counter"
    torch.cuda.synchronize()
    assert W.ws_sync(r.ctx, 0) == W.WS_ERR_CUDA
    msg = W.ws_last_error(r.ctx)
    assert "canary" in msg and where in msg and field in msg, msg
    assert W.ws_rollout(r.ctx, 1) == W.WS_ERR_CUDA      # sticky
    r.close()


def test_no_canaries_without_the_flag(torch):
    cfg, _ = W.make_config(W.WS_ENV_CONTROL, F32, 64, 8, 100, 16, 16)
    cfg_b, _ = W.make_config(W.WS_ENV_CONTROL, F32, 64, 8, 100, 16, 16, flags=BC)
    s0, s1 = W.ws_query_bytes(cfg), W.ws_query_bytes(cfg_b)
    # the ring's six fields (OBS, ACTION, LOGP, REWARD, DONE, RETURN) each gain one
    assert s1[2] >= s0[2] + 6 * 256 and s1[1] > s0[1]
