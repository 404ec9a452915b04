"""Launch configuration and the autotuner: every launch parameter of a path
changes speed, not results (byte-for-byte where the arithmetic is unchanged;
the landscape energy's Gaussian chunk count regroups an FP32 sum); ws_tune
picks a valid configuration, leaves the context reset, and caches its choice."""
import time

import numpy as np
import pytest

import oracle
from paper_2408_00930_gb300 import warpsci as W
from tests.gpu_common import need_gpu

pytestmark = pytest.mark.gpu
BF16, F32, PLAIN = W.WS_PATH_BATCHED_BF16, W.WS_PATH_BATCHED_FP32, W.WS_PATH_PLAIN_FP32
FIELDS = (W.WS_F_OBS, W.WS_F_ACTION, W.WS_F_LOGP, W.WS_F_REWARD, W.WS_F_DONE)


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


def records(r, T, fields=FIELDS):
    return [r.fetch(f, 0, T).tobytes() for f in fields]


def run(make, T, seed, **launch):
    r = make()
    if launch:
        r.set_launch(**launch)
    r.reset(seed)
    r.rollout(T)
    r.sync()
    return r


def test_control_grid_and_chunk_do_not_change_records(torch):
    T = 60
    make = lambda: W.Rollout(W.WS_ENV_CONTROL, BF16, 3000, T, 200, 128, 128, param_seed=2)
    a = run(make, T, 9)
    ra = records(a, T)
    a.close()
    for kw in (dict(grid=5), dict(chunk_steps=7), dict(grid=12, chunk_steps=13)):
        b = run(make, T, 9, **kw)
        assert records(b, T) == ra, kw
        b.close()


def test_economy_items_and_order_do_not_change_records(torch):
    T = 30
    counts = np.array([oracle.econ_agent_count(4, e) for e in range(120)], np.int32)
    assert counts.max() <= 256
    make = lambda: W.Rollout(W.WS_ENV_ECONOMY, BF16, 120, T, 540, 128, 128, param_seed=4)
    fields = FIELDS + (W.WS_F_WEALTH,)
    base = run(make, T, 3)
    rb = records(base, T, fields)
    base.close()
    for kw in (dict(econ_tiles=2), dict(econ_lpt=0), dict(econ_tiles=2, econ_lpt=0, chunk_steps=9)):
        r = run(make, T, 3, **kw)
        assert records(r, T, fields) == rb, kw
        r.close()


def test_economy_rejects_tiles_below_the_largest_env(torch):
    r = W.Rollout(W.WS_ENV_ECONOMY, BF16, 3, 8, 540, 128, 128, agents_per_env=[300, 8, 9])
    with pytest.raises(W.WarpSciError):
        r.set_launch(econ_tiles=2)           # 300 agents need three tiles
    assert r.launch().econ_tiles == 3
    r.close()


def test_per_step_block_size_does_not_change_records(torch):
    T = 12
    for env, h, kw in ((W.WS_ENV_CONTROL, 64, {}), (W.WS_ENV_ECONOMY, 128, {}),
                       (W.WS_ENV_LANDSCAPE, 64, dict(dim=8, n_gauss=300))):
        make = lambda: W.Rollout(env, F32, 700, T, 50, h, h, param_seed=5, **kw)
        a = run(make, T, 1)
        ra = records(a, T)
        a.close()
        for th in (128, 512):
            b = run(make, T, 1, env_threads=th)
            assert records(b, T) == ra, (env, th)
            b.close()


def test_landscape_energy_chunks_regroup_only_the_sum(torch):
    T, D, M, n = 6, 24, 4096, 512
    make = lambda: W.Rollout(W.WS_ENV_LANDSCAPE, BF16, n, T, 1000, 64, 64, dim=D, n_gauss=M,
                             param_seed=6)
    out = {}
    for ec in (1, 2, 4):
        r = run(make, T, 2, energy_chunks=ec)
        out[ec] = r.fetch(W.WS_F_ENERGY, 0, 1)[0].astype(np.float64)
        r.close()
    # the chunk count regroups the FP32 sum over the Gaussians: rounding-level changes only
    for ec in (2, 4):
        assert np.abs(out[ec] - out[1]).max() <= 1e-5 * max(1.0, np.abs(out[1]).max())


def test_tune_picks_valid_launch_resets_and_caches(torch):
    T = 40
    make = lambda: W.Rollout(W.WS_ENV_ECONOMY, BF16, 200, T, 540, 128, 128, param_seed=7)
    r = make()
    t0 = time.perf_counter()
    chosen, ms = r.tune(20)
    t_first = time.perf_counter() - t0
    assert ms > 0 and 1 <= chosen["econ_tiles"] <= 3 and chosen["econ_lpt"] in (0, 1)
    assert r.k == 0
    assert r.launch().as_dict() == chosen
    r.rollout(T)
    r.sync()
    tuned = records(r, T, FIELDS + (W.WS_F_WEALTH,))
    r.close()
    # a second context of the same shape takes the cached choice without trials
    r2 = make()
    t0 = time.perf_counter()
    chosen2, ms2 = r2.tune(20)
    t_second = time.perf_counter() - t0
    assert chosen2 == chosen and ms2 == ms
    assert t_second < t_first
    r2.close()
    # the tuned roll-out equals one under the default launch, from the same reset
    d = make()
    d.reset(7)
    d.rollout(T)
    d.sync()
    assert records(d, T, FIELDS + (W.WS_F_WEALTH,)) == tuned
    d.close()


def test_tune_each_path(torch):
    for env, path, n, h, kw in ((W.WS_ENV_CONTROL, BF16, 2048, 256, {}),
                                (W.WS_ENV_CONTROL, PLAIN, 2048, 64, {}),
                                (W.WS_ENV_LANDSCAPE, BF16, 512, 64, dict(dim=24, n_gauss=1024))):
        r = W.Rollout(env, path, n, 16, 200, h, h, param_seed=8, **kw)
        chosen, ms = r.tune(8)
        assert ms > 0 and r.k == 0
        r.rollout(16)
        r.sync()
        r.close()
