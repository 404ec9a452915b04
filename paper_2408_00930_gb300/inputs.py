"""Seeded synthetic inputs shared by the oracle tests and the CUDA parity tests.

This module holds none of the method's arithmetic: it only draws numpy random
arrays with the shapes and value distributions of the workloads (control state
near the upright equilibrium, economy features N(0,1) and wealth in
[1e4, 1e6], landscape coordinates in [-3, 3]^D, small uniform policy weights).
Every float it returns is exactly representable in FP32, so the FP32 CUDA path
and the FP64 oracle start from identical values.
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def _f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def policy_params(g: np.random.Generator, widths, scale: float = 1.0) -> np.ndarray:
    """Flat FP32 parameters in the layout W_l[n_in][n_out] then b_l, per layer."""
    parts = []
    for n_in, n_out in zip(widths[:-1], widths[1:]):
        b = scale / np.sqrt(n_in)
        parts.append(g.uniform(-b, b, size=n_in * n_out))
        parts.append(g.uniform(-b, b, size=n_out))
    return np.concatenate(parts).astype(np.float32)


def control_states(g: np.random.Generator, n: int, spread: float = 0.15, limit: int = 200):
    """States (x, v, th, w) and episode step counts for n envs."""
    s = _f32(np.stack([g.uniform(-2.0, 2.0, n), g.uniform(-1.0, 1.0, n),
                       g.uniform(-spread, spread, n), g.uniform(-1.0, 1.0, n)], axis=1))
    t = g.integers(0, limit, size=n).astype(np.int32)
    return s, t


def econ_state(g: np.random.Generator, n_agents):
    """Wealth (int64) and 16 features per agent, in slot order."""
    n = int(np.sum(n_agents))
    wealth = g.integers(10_000, 1_000_001, size=n).astype(np.int64)
    feat = _f32(g.standard_normal((n, 16)))
    return wealth, feat


def econ_agent_counts(g: np.random.Generator, n_envs: int, lo: int = 8, hi: int = 256):
    return g.integers(lo, hi + 1, size=n_envs).astype(np.int32)


def landscape_state(g: np.random.Generator, n: int, D: int, limit: int = 1000):
    x = _f32(g.uniform(-3.0, 3.0, (n, D)))
    eobs = _f32(g.normal(0.0, 0.05, n))
    t = g.integers(0, limit, size=n).astype(np.int32)
    return x, eobs, t


def landscape_params(g: np.random.Generator, M: int, D: int):
    c = _f32(g.uniform(-3.0, 3.0, (M, D)))
    w = _f32(np.exp(0.3 * g.standard_normal(M)))
    a = _f32(g.standard_normal(M))
    return c, w, a


def rewards_dones(g: np.random.Generator, T: int, S: int, p_done: float = 0.02):
    r = _f32(g.normal(0.5, 1.0, (T, S)))
    d = (g.random((T, S)) < p_done).astype(np.uint8)
    return r, d
