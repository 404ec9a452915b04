"""Test helpers: state/parameter packing in the layouts of include/warpsci.h,
and the comparison rules (tie band, threshold band, per-env relative error)."""
import numpy as np

from paper_2408_00930_gb300 import warpsci as W


def pack_control_state(s, t):
    s = np.asarray(s, np.float64)
    return np.concatenate([np.ascontiguousarray(s.T.astype(np.float32)).view(np.uint8).ravel(),
                           np.asarray(t, np.int32).view(np.uint8)])


def unpack_control_state(raw, n):
    s = raw[:16 * n].view(np.float32).reshape(4, n).T.astype(np.float64)
    t = raw[16 * n:20 * n].view(np.int32)
    return s, t


def pack_econ_state(wealth, feat, t):
    return np.concatenate([np.asarray(wealth, np.int64).view(np.uint8),
                           np.ascontiguousarray(np.asarray(feat).T.astype(np.float32)).view(np.uint8).ravel(),
                           np.asarray(t, np.int32).view(np.uint8)])


def unpack_econ_state(raw, n_agents, n_envs):
    w = raw[:8 * n_agents].view(np.int64)
    f = raw[8 * n_agents:8 * n_agents + 64 * n_agents].view(np.float32).reshape(16, n_agents).T
    t = raw[72 * n_agents:72 * n_agents + 4 * n_envs].view(np.int32)
    return w, f.astype(np.float64), t


def pack_landscape_state(x, eobs, t):
    return np.concatenate([np.ascontiguousarray(np.asarray(x).T.astype(np.float32)).view(np.uint8).ravel(),
                           np.asarray(eobs, np.float32).view(np.uint8),
                           np.asarray(t, np.int32).view(np.uint8)])


def unpack_landscape_state(raw, n, D):
    x = raw[:4 * D * n].view(np.float32).reshape(D, n).T.astype(np.float64)
    eobs = raw[4 * D * n:4 * D * n + 4 * n].view(np.float32).astype(np.float64)
    t = raw[4 * D * n + 4 * n:4 * D * n + 8 * n].view(np.int32)
    return x, eobs, t


def rel_err_rows(g, o):
    """Per row: max |g - o| / max(max |o|, 1)."""
    g = np.asarray(g, np.float64).reshape(len(g), -1)
    o = np.asarray(o, np.float64).reshape(len(o), -1)
    return np.abs(g - o).max(1) / np.maximum(np.abs(o).max(1), 1.0)


def first_divergence(ambiguous):
    """[T][n] bool -> per env the first step index flagged (T if none)."""
    T = ambiguous.shape[0]
    amb = ambiguous.any(axis=tuple(range(2, ambiguous.ndim))) if ambiguous.ndim > 2 else ambiguous
    idx = np.where(amb.any(0), amb.argmax(0), T)
    return idx


def valid_mask(first, T):
    """[T][n] True for steps strictly before each env's first ambiguous step."""
    return np.arange(T)[:, None] < first[None, :]


def check_landscape_dones(obs, act, done, cwa, limit, target, seed, tol):
    """Done flags of a landscape roll-out recorded from a reset at step 0 (obs
    and act [T][D][n]): done at the step limit or when the FP64 energy of the
    recorded post-step state x + dx is below the target.  A decision whose FP64
    energy lies within tol * max(scale, 1e-3) of the target may go either way
    (the GPU decides on its own FP32 or BF16 estimate).  The state after a done
    is the Philox reset draw.  Returns (energy-target dones, borderline cases)."""
    import oracle
    c, w, a = cwa
    T, D, n = obs.shape
    n_target = n_band = 0
    for e in range(n):
        t = 0
        for s in range(T):
            y = (obs[s][:, e] + act[s][:, e]).astype(np.float32).astype(np.float64)
            E = oracle.landscape_energy(c, w, a, y)
            t += 1
            if abs(E - target) <= tol * max(oracle.landscape_energy_scale(c, w, a, y), 1e-3):
                n_band += 1
            else:
                assert bool(done[s][e]) == (t >= limit or E < target), (s, e, E, target)
            if done[s][e]:
                n_target += int(t < limit)
                t = 0
                if s + 1 < T:
                    np.testing.assert_array_equal(
                        obs[s + 1][:, e], oracle.landscape_reset_draw(seed, s, e, D).astype(np.float32))
            elif s + 1 < T:
                np.testing.assert_array_equal(obs[s + 1][:, e], y.astype(np.float32))
    return n_target, n_band
