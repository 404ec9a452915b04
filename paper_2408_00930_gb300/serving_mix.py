"""Seeded synthetic request stream for the serving loop.

Poisson arrivals (mean rate `rate` per second) of roll-out requests drawn
across the three env types: env counts log-uniform in [256, 65,536], agents
1 (control, landscape) or U{8..256} (economy, drawn by the engine from the
request seed), horizons uniform over {100, 150, ..., 1,000}, delivered in
chunks of 50 steps.  Holds no arithmetic of the roll-out itself.
"""
from __future__ import annotations

import numpy as np

ENV_SHAPES = {
    0: dict(hidden=(256, 256), episode_limit=200, dim=0, n_gauss=0),
    1: dict(hidden=(128, 128), episode_limit=540, dim=0, n_gauss=0),
    2: dict(hidden=(256, 256), episode_limit=1000, dim=24, n_gauss=4096),
}


def request_stream(seed: int, n_requests: int, rate: float = 200.0, env_lo: int = 256,
                   env_hi: int = 65536, econ_env_hi: int | None = None):
    """Yield dicts: t_arrival (s), env, n_envs, horizon, seed."""
    g = np.random.default_rng(seed)
    t = 0.0
    for i in range(n_requests):
        t += g.exponential(1.0 / rate)
        env = int(g.integers(0, 3))
        hi = econ_env_hi if (env == 1 and econ_env_hi) else env_hi
        n = int(round(np.exp(g.uniform(np.log(env_lo), np.log(hi)))))
        horizon = int(g.choice(np.arange(100, 1001, 50)))
        yield dict(t_arrival=t, env=env, n_envs=n, horizon=horizon, seed=int(g.integers(1, 2**31)),
                   **ENV_SHAPES[env])
