"""FP64 CPU oracle of the in-place RL roll-out loop (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline and
reference legs may import this package.  The product path (the CUDA library and
its Python binding) never imports, links or executes it.

The arithmetic lives in ``ws_oracle.c`` (plain C, FP64, env by env and step by
step); this module only compiles it with gcc and marshals numpy arrays through
ctypes.  Each wrapper names the C function, whose comment cites the passage of
the paper (and the reading) it follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ws_oracle.c")
_LIB = os.path.join(_HERE, "libws_oracle.so")
_lock = threading.Lock()
_lib = None

TAG_ACTION, TAG_RESET, TAG_PARTNER, TAG_NOISE = 0, 1, 2, 3
TAG_POLICY_INIT, TAG_LANDSCAPE_INIT, TAG_ECON_INIT = 4, 5, 6
PLANNER_ID = 0xFFFFFFFF
STEP_INIT = 0xFFFFFFFF


def build(force: bool = False) -> str:
    """Compile ws_oracle.c into libws_oracle.so (IEEE FP, no contraction)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", _SRC, "-lm", "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _declare(_lib)
    return _lib


_P = C.c_void_p


def _declare(L):
    L.or_philox4x32_10.argtypes = [_P, _P, _P]
    L.or_philox_batch.argtypes = [C.c_long, _P, _P, _P]
    L.or_u01.argtypes = [C.c_uint32]
    L.or_u01.restype = C.c_double
    L.or_uniform_f32.argtypes = [C.c_uint32, C.c_float, C.c_float]
    L.or_uniform_f32.restype = C.c_float
    L.or_box_muller.argtypes = [C.c_uint32, C.c_uint32, _P, _P]
    L.or_bounded.argtypes = [C.c_uint32, C.c_uint32]
    L.or_bounded.restype = C.c_uint32
    L.or_round_bf16.argtypes = [C.c_float]
    L.or_round_bf16.restype = C.c_float
    L.or_policy_param_count.argtypes = [C.c_int, _P]
    L.or_policy_param_count.restype = C.c_long
    L.or_policy_init.argtypes = [C.c_uint64, C.c_uint32, C.c_int, _P, _P]
    L.or_mlp_forward.argtypes = [C.c_int, _P, _P, C.c_uint32, _P, _P]
    L.or_sample_categorical.argtypes = [C.c_int, _P, C.c_double, _P, _P]
    L.or_sample_categorical.restype = C.c_int
    L.or_gaussian_action.argtypes = [C.c_int, _P, _P, C.c_double, _P, _P]
    L.or_control_dynamics.argtypes = [_P, C.c_int, _P]
    L.or_control_done.argtypes = [_P, C.c_int, C.c_int, _P]
    L.or_control_done.restype = C.c_int
    L.or_control_reset_draw.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, _P]
    L.or_control_rollout.argtypes = ([_P, C.c_int, C.c_int, C.c_uint32, C.c_uint64, C.c_uint32,
                                      _P, C.c_int, _P, _P, C.c_int, C.c_int] + [_P] * 10)
    L.or_acrobot_deriv.argtypes = [_P, C.c_double, _P]
    L.or_acrobot_step.argtypes = [_P, C.c_int, C.c_double, _P, _P]
    L.or_acrobot_obs.argtypes = [_P, _P]
    L.or_acrobot_terminal.argtypes = [_P, _P]
    L.or_acrobot_terminal.restype = C.c_int
    L.or_acrobot_reset_draw.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, _P]
    L.or_acrobot_rollout.argtypes = ([_P, C.c_int, C.c_int, C.c_uint32, C.c_uint64, C.c_uint32,
                                      _P, C.c_int, _P, _P, C.c_int, C.c_int] + [_P] * 11)
    L.or_econ_agent_count.argtypes = [C.c_uint64, C.c_uint32]
    L.or_econ_agent_count.restype = C.c_uint32
    L.or_econ_reset_agent.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, _P, _P]
    L.or_econ_rollout.argtypes = ([_P, _P, C.c_uint32, C.c_uint64, C.c_uint32, _P, _P, C.c_int,
                                   _P, _P, _P, C.c_int, C.c_int] + [_P] * 10)
    L.or_landscape_init.argtypes = [C.c_uint64, C.c_int, C.c_int, _P, _P, _P]
    L.or_landscape_energy.argtypes = [C.c_int, C.c_int, _P, _P, _P, _P]
    L.or_landscape_energy.restype = C.c_double
    L.or_landscape_energy_scale.argtypes = [C.c_int, C.c_int, _P, _P, _P, _P]
    L.or_landscape_energy_scale.restype = C.c_double
    L.or_landscape_grad.argtypes = [C.c_int, C.c_int, _P, _P, _P, _P, _P]
    L.or_landscape_action_normals.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_int, _P]
    L.or_landscape_noise.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32]
    L.or_landscape_noise.restype = C.c_double
    L.or_landscape_reset_draw.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_int, _P]
    L.or_landscape_rollout.argtypes = ([C.c_int, C.c_int, _P, _P, _P, _P, C.c_int, C.c_int,
                                        C.c_uint32, C.c_double, C.c_double, C.c_uint64,
                                        C.c_uint32, _P, C.c_int, _P, _P, _P, C.c_int, C.c_int,
                                        C.c_double]
                                       + [_P] * 10)
    L.or_returns.argtypes = [C.c_int, C.c_long, _P, _P, C.c_double, _P]
    L.or_a2c.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _P, _P, _P, _P, _P, _P,
                         C.c_double, C.c_double, _P, _P, _P]
    L.or_a2c_gauss.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, _P, _P, _P, _P, _P, _P,
                               C.c_double, C.c_double, _P, _P, _P]
    L.or_ppo.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _P, _P, _P, _P, _P, _P, _P,
                         C.c_double, C.c_double, C.c_double, _P, _P, _P]
    L.or_ppo_gauss.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, _P, _P, _P, _P, _P, _P, _P,
                               C.c_double, C.c_double, C.c_double, _P, _P, _P]


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _arr(a, dtype):
    if a is None:
        return None
    return np.ascontiguousarray(a, dtype=dtype)


# --------------------------------------------------------------------------
# random streams
# --------------------------------------------------------------------------
def philox(ctr, key):
    """Philox4x32-10 of counters ``ctr`` ([n,4] or [4]) under ``key`` (2 words)."""
    c = np.ascontiguousarray(np.atleast_2d(np.asarray(ctr, dtype=np.uint32)))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.empty_like(c)
    lib().or_philox_batch(c.shape[0], _ptr(c), _ptr(k), _ptr(out))
    return out[0] if np.asarray(ctr).ndim == 1 else out


def seed_key(seed: int):
    return np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint32)


def draw(seed, c0, c1, c2, tag, sub=0):
    return philox([c0 & 0xFFFFFFFF, c1 & 0xFFFFFFFF, c2 & 0xFFFFFFFF,
                   ((tag << 24) | (sub & 0xFFFFFF)) & 0xFFFFFFFF], seed_key(seed))


def u01(w):
    return lib().or_u01(int(w))


def uniform_f32(w, a, b):
    return np.float32(lib().or_uniform_f32(int(w), float(a), float(b)))


def box_muller(w0, w1):
    zc, zs = C.c_double(), C.c_double()
    lib().or_box_muller(int(w0), int(w1), C.byref(zc), C.byref(zs))
    return zc.value, zs.value


def bounded(w, n):
    return lib().or_bounded(int(w), int(n))


def round_bf16(f):
    return np.float32(lib().or_round_bf16(float(f)))


# --------------------------------------------------------------------------
# policy
# --------------------------------------------------------------------------
def policy_param_count(widths):
    w = _arr(widths, np.int32)
    return lib().or_policy_param_count(len(w) - 1, _ptr(w))


def policy_init(seed, policy_id, widths):
    w = _arr(widths, np.int32)
    out = np.empty(policy_param_count(w), dtype=np.float32)
    lib().or_policy_init(seed, policy_id, len(w) - 1, _ptr(w), _ptr(out))
    return out


def mlp_forward(widths, params, x, bf16_layers=0):
    w = _arr(widths, np.int32)
    p = _arr(params, np.float32)
    xs = np.atleast_2d(_arr(x, np.float64))
    ys = np.empty((xs.shape[0], int(w[-1])), dtype=np.float64)
    for i in range(xs.shape[0]):
        xi = np.ascontiguousarray(xs[i])
        yi = np.empty(int(w[-1]), dtype=np.float64)
        lib().or_mlp_forward(len(w) - 1, _ptr(w), _ptr(p), bf16_layers, _ptr(xi), _ptr(yi))
        ys[i] = yi
    return ys if np.asarray(x).ndim == 2 else ys[0]


def sample_categorical(logits, u):
    lg = _arr(logits, np.float64)
    lp, mg = C.c_double(), C.c_double()
    a = lib().or_sample_categorical(len(lg), _ptr(lg), float(u), C.byref(lp), C.byref(mg))
    return a, lp.value, mg.value


def gaussian_action(out, z, clip):
    o = _arr(out, np.float64)
    zz = _arr(z, np.float64)
    D = len(zz)
    dx = np.empty(D, dtype=np.float64)
    lp = C.c_double()
    lib().or_gaussian_action(D, _ptr(o), _ptr(zz), float(clip), _ptr(dx), C.byref(lp))
    return dx, lp.value


# --------------------------------------------------------------------------
# control env
# --------------------------------------------------------------------------
def control_dynamics(s, action):
    si = _arr(s, np.float64)
    out = np.empty(4, dtype=np.float64)
    lib().or_control_dynamics(_ptr(si), int(action), _ptr(out))
    return out


def control_done(s, t, limit):
    si = _arr(s, np.float64)
    mg = C.c_double()
    d = lib().or_control_done(_ptr(si), int(t), int(limit), C.byref(mg))
    return bool(d), mg.value


def control_reset_draw(seed, k, env):
    out = np.empty(4, dtype=np.float64)
    lib().or_control_reset_draw(seed, k & 0xFFFFFFFF, env, _ptr(out))
    return out


def control_rollout(params, hidden0, hidden1, seed, env_ids, n_steps, episode_limit,
                    k0=0, state0=None, t0=None, bf16_layers=0):
    """Roll out the control env for envs ``env_ids``; arrays are [n_steps][n_envs]."""
    ids = _arr(env_ids, np.uint32)
    n = len(ids)
    p = _arr(params, np.float32)
    s0 = _arr(state0, np.float64)
    tt0 = _arr(t0, np.int32)
    out = dict(
        obs=np.empty((n_steps, n, 4)), action=np.empty((n_steps, n), np.int32),
        logp=np.empty((n_steps, n)), reward=np.empty((n_steps, n)),
        done=np.empty((n_steps, n), np.uint8), logits=np.empty((n_steps, n, 2)),
        act_margin=np.empty((n_steps, n)), done_margin=np.empty((n_steps, n)),
        state=np.empty((n, 4)), t=np.empty(n, np.int32))
    lib().or_control_rollout(
        _ptr(p), hidden0, hidden1, bf16_layers, seed, k0 & 0xFFFFFFFF, _ptr(ids), n,
        _ptr(s0), _ptr(tt0), n_steps, episode_limit,
        _ptr(out["obs"]), _ptr(out["action"]), _ptr(out["logp"]), _ptr(out["reward"]),
        _ptr(out["done"]), _ptr(out["logits"]), _ptr(out["act_margin"]),
        _ptr(out["done_margin"]), _ptr(out["state"]), _ptr(out["t"]))
    return out


# --------------------------------------------------------------------------
# acrobot (App. C classic control; the Sutton & Barto two-link acrobot)
# --------------------------------------------------------------------------
def acrobot_deriv(s, tau):
    out = np.empty(4)
    lib().or_acrobot_deriv(_ptr(_arr(s, np.float64)), float(tau), _ptr(out))
    return out


def acrobot_step(s, action, dt=0.2):
    """One RK4 step with the torque of ``action``; returns (wrapped and clipped
    state, raw RK4 state)."""
    out, raw = np.empty(4), np.empty(4)
    lib().or_acrobot_step(_ptr(_arr(s, np.float64)), int(action), float(dt), _ptr(out), _ptr(raw))
    return out, raw


def acrobot_obs(s):
    o = np.empty(6)
    lib().or_acrobot_obs(_ptr(_arr(s, np.float64)), _ptr(o))
    return o


def acrobot_terminal(s):
    mg = C.c_double()
    t = lib().or_acrobot_terminal(_ptr(_arr(s, np.float64)), C.byref(mg))
    return bool(t), mg.value


def acrobot_reset_draw(seed, k, env):
    out = np.empty(4)
    lib().or_acrobot_reset_draw(seed, k & 0xFFFFFFFF, env, _ptr(out))
    return out


def acrobot_rollout(params, hidden0, hidden1, seed, env_ids, n_steps, episode_limit,
                    k0=0, state0=None, t0=None, bf16_layers=0):
    """Roll out the acrobot for envs ``env_ids``; arrays are [n_steps][n_envs]."""
    ids = _arr(env_ids, np.uint32)
    n = len(ids)
    out = dict(
        obs=np.empty((n_steps, n, 6)), state=np.empty((n_steps, n, 4)),
        action=np.empty((n_steps, n), np.int32), logp=np.empty((n_steps, n)),
        reward=np.empty((n_steps, n)), done=np.empty((n_steps, n), np.uint8),
        logits=np.empty((n_steps, n, 3)), act_margin=np.empty((n_steps, n)),
        done_margin=np.empty((n_steps, n)), state_out=np.empty((n, 4)),
        t=np.empty(n, np.int32))
    lib().or_acrobot_rollout(
        _ptr(_arr(params, np.float32)), hidden0, hidden1, bf16_layers, seed, k0 & 0xFFFFFFFF,
        _ptr(ids), n, _ptr(_arr(state0, np.float64)), _ptr(_arr(t0, np.int32)), n_steps,
        episode_limit, _ptr(out["obs"]), _ptr(out["state"]), _ptr(out["action"]),
        _ptr(out["logp"]), _ptr(out["reward"]), _ptr(out["done"]), _ptr(out["logits"]),
        _ptr(out["act_margin"]), _ptr(out["done_margin"]), _ptr(out["state_out"]),
        _ptr(out["t"]))
    return out


# --------------------------------------------------------------------------
# economy
# --------------------------------------------------------------------------
def econ_agent_count(param_seed, env):
    return lib().or_econ_agent_count(param_seed, env)


def econ_reset_agent(seed, k, env, agent):
    w = C.c_int64()
    f = np.empty(16, dtype=np.float64)
    lib().or_econ_reset_agent(seed, k & 0xFFFFFFFF, env, agent, C.byref(w), _ptr(f))
    return w.value, f


def econ_rollout(agent_params, planner_params, seed, env_ids, n_agents, n_steps, episode_limit,
                 k0=0, wealth0=None, feat0=None, t0=None, bf16_layers=0):
    """Slot layout: agents of each listed env in order, then one planner per env."""
    ids = _arr(env_ids, np.uint32)
    na = _arr(n_agents, np.int32)
    ne = len(ids)
    n_agent_slots = int(na.sum())
    ns = n_agent_slots + ne
    out = dict(
        obs=np.empty((n_steps, ns, 16)), action=np.empty((n_steps, ns), np.int32),
        logp=np.empty((n_steps, ns)), reward=np.empty((n_steps, ns)),
        done=np.empty((n_steps, ns), np.uint8), wealth=np.empty((n_steps, ns), np.int64),
        act_margin=np.empty((n_steps, ns)), wealth_out=np.empty(n_agent_slots, np.int64),
        feat_out=np.empty((n_agent_slots, 16)), t=np.empty(ne, np.int32))
    w0 = _arr(wealth0, np.int64)
    f0 = _arr(feat0, np.float64)
    tt0 = _arr(t0, np.int32)
    lib().or_econ_rollout(
        _ptr(_arr(agent_params, np.float32)), _ptr(_arr(planner_params, np.float32)),
        bf16_layers, seed, k0 & 0xFFFFFFFF, _ptr(ids), _ptr(na), ne, _ptr(w0), _ptr(f0),
        _ptr(tt0), n_steps, episode_limit,
        _ptr(out["obs"]), _ptr(out["action"]), _ptr(out["logp"]), _ptr(out["reward"]),
        _ptr(out["done"]), _ptr(out["wealth"]), _ptr(out["act_margin"]),
        _ptr(out["wealth_out"]), _ptr(out["feat_out"]), _ptr(out["t"]))
    return out


# --------------------------------------------------------------------------
# landscape
# --------------------------------------------------------------------------
def landscape_init(param_seed, D, M):
    c = np.empty((M, D)); w = np.empty(M); a = np.empty(M)
    lib().or_landscape_init(param_seed, D, M, _ptr(c), _ptr(w), _ptr(a))
    return c, w, a


def landscape_energy(c, w, a, x):
    c = _arr(c, np.float64); w = _arr(w, np.float64); a = _arr(a, np.float64)
    x = _arr(x, np.float64)
    return lib().or_landscape_energy(c.shape[1], c.shape[0], _ptr(c), _ptr(w), _ptr(a), _ptr(x))


def landscape_energy_scale(c, w, a, x):
    c = _arr(c, np.float64); w = _arr(w, np.float64); a = _arr(a, np.float64)
    x = _arr(x, np.float64)
    return lib().or_landscape_energy_scale(c.shape[1], c.shape[0], _ptr(c), _ptr(w), _ptr(a),
                                           _ptr(x))


def landscape_grad(c, w, a, x):
    c = _arr(c, np.float64); w = _arr(w, np.float64); a = _arr(a, np.float64)
    x = _arr(x, np.float64)
    g = np.empty(c.shape[1])
    lib().or_landscape_grad(c.shape[1], c.shape[0], _ptr(c), _ptr(w), _ptr(a), _ptr(x), _ptr(g))
    return g


def landscape_action_normals(seed, k, env, D):
    z = np.empty(D)
    lib().or_landscape_action_normals(seed, k & 0xFFFFFFFF, env, D, _ptr(z))
    return z


def landscape_noise(seed, k, env, sub):
    return lib().or_landscape_noise(seed, k & 0xFFFFFFFF, env, sub)


def landscape_reset_draw(seed, k, env, D):
    x = np.empty(D)
    lib().or_landscape_reset_draw(seed, k & 0xFFFFFFFF, env, D, _ptr(x))
    return x


def landscape_rollout(c, w, a, params, hidden0, hidden1, seed, env_ids, n_steps, episode_limit,
                      noise_sigma=0.05, step_clip=0.1, k0=0, x0=None, eobs0=None, t0=None,
                      bf16_layers=0, energy_target=None):
    """Landscape roll-out (App. C stand-in).  An episode ends at the step limit
    or, with energy_target set, when the pure energy of the post-step state
    falls below it."""
    c = _arr(c, np.float64); w = _arr(w, np.float64); a = _arr(a, np.float64)
    M, D = c.shape
    ids = _arr(env_ids, np.uint32)
    n = len(ids)
    out = dict(
        obs=np.empty((n_steps, n, D)), act=np.empty((n_steps, n, D)),
        logp=np.empty((n_steps, n)), reward=np.empty((n_steps, n)),
        done=np.empty((n_steps, n), np.uint8), energy=np.empty((n_steps, n)),
        energy_scale=np.empty((n_steps, n)), x=np.empty((n, D)), eobs=np.empty(n),
        t=np.empty(n, np.int32))
    lib().or_landscape_rollout(
        D, M, _ptr(c), _ptr(w), _ptr(a), _ptr(_arr(params, np.float32)), hidden0, hidden1,
        bf16_layers, noise_sigma, step_clip, seed, k0 & 0xFFFFFFFF, _ptr(ids), n,
        _ptr(_arr(x0, np.float64)), _ptr(_arr(eobs0, np.float64)), _ptr(_arr(t0, np.int32)),
        n_steps, episode_limit, -np.inf if energy_target is None else float(energy_target),
        _ptr(out["obs"]), _ptr(out["act"]), _ptr(out["logp"]), _ptr(out["reward"]),
        _ptr(out["done"]), _ptr(out["energy"]), _ptr(out["energy_scale"]), _ptr(out["x"]),
        _ptr(out["eobs"]), _ptr(out["t"]))
    return out


# --------------------------------------------------------------------------
# returns
# --------------------------------------------------------------------------
def returns(reward, done, gamma):
    r = _arr(reward, np.float64)
    d = _arr(done, np.uint8)
    T = r.shape[0]
    ns = int(np.prod(r.shape[1:])) if r.ndim > 1 else 1
    G = np.empty_like(r)
    lib().or_returns(T, ns, _ptr(r), _ptr(d), float(gamma), _ptr(G))
    return G


# --------------------------------------------------------------------------
# actor-critic update (A2C with Monte-Carlo returns)
# --------------------------------------------------------------------------
def a2c(actor, critic, obs, act, ret, h0, h1, n_act, c_v=0.5, c_e=0.0, adv=None, grads=True):
    """Loss terms {policy, value, entropy} (means over the rows) and, with
    grads, dL/d(actor params) and dL/d(critic params) in FP64.  obs [R][obs_dim],
    act [R], ret [R]; adv (the actor's advantage) defaults to G - V."""
    o = _arr(obs, np.float64)
    R, od = o.shape
    na = policy_param_count([od, h0, h1, n_act])
    nc = policy_param_count([od, h0, h1, 1])
    ga = np.empty(na) if grads else None
    gc = np.empty(nc) if grads else None
    st = np.empty(3)
    lib().or_a2c(R, od, n_act, h0, h1, _ptr(_arr(actor, np.float32)), _ptr(_arr(critic, np.float32)),
                 _ptr(o), _ptr(_arr(act, np.int32)), _ptr(_arr(ret, np.float64)),
                 _ptr(_arr(adv, np.float64)), float(c_v), float(c_e), _ptr(ga), _ptr(gc), _ptr(st))
    return st, ga, gc


def ppo(actor, critic, obs, act, ret, adv, logp_old, h0, h1, n_act, eps, c_v=0.5, c_e=0.0,
        grads=True):
    """PPO clipped-surrogate loss terms {surrogate, value, entropy, clip
    fraction} and, with grads, dL/d(actor) and dL/d(critic) in FP64
    (or_ppo).  adv is the advantage held from before the update, logp_old
    the behaviour policy's log-probability of each row's action."""
    o = _arr(obs, np.float64)
    R, od = o.shape
    na = policy_param_count([od, h0, h1, n_act])
    nc = policy_param_count([od, h0, h1, 1])
    ga = np.empty(na) if grads else None
    gc = np.empty(nc) if grads else None
    st = np.empty(4)
    lib().or_ppo(R, od, n_act, h0, h1, _ptr(_arr(actor, np.float32)), _ptr(_arr(critic, np.float32)),
                 _ptr(o), _ptr(_arr(act, np.int32)), _ptr(_arr(ret, np.float64)),
                 _ptr(_arr(adv, np.float64)), _ptr(_arr(logp_old, np.float64)), float(eps),
                 float(c_v), float(c_e), _ptr(ga), _ptr(gc), _ptr(st))
    return st, ga, gc


def ppo_gauss(actor, critic, obs, u, ret, adv, logp_old, h0, h1, eps, c_v=0.5, c_e=0.0,
              grads=True):
    """PPO for the diagonal Gaussian head (or_ppo_gauss): u [R][D] the
    behaviour samples (unclipped), logp_old their recorded log-densities."""
    o = _arr(obs, np.float64)
    R, D = o.shape
    na = policy_param_count([D, h0, h1, 2 * D])
    nc = policy_param_count([D, h0, h1, 1])
    ga = np.empty(na) if grads else None
    gc = np.empty(nc) if grads else None
    st = np.empty(4)
    lib().or_ppo_gauss(R, D, h0, h1, _ptr(_arr(actor, np.float32)), _ptr(_arr(critic, np.float32)),
                       _ptr(o), _ptr(_arr(u, np.float64)), _ptr(_arr(ret, np.float64)),
                       _ptr(_arr(adv, np.float64)), _ptr(_arr(logp_old, np.float64)), float(eps),
                       float(c_v), float(c_e), _ptr(ga), _ptr(gc), _ptr(st))
    return st, ga, gc


def a2c_gauss(actor, critic, obs, z, ret, h0, h1, c_v=0.5, c_e=0.0, adv=None, grads=True):
    """The actor-critic update for the diagonal Gaussian head (landscape): obs
    and z (the normals the recorded samples used) [R][D]."""
    o = _arr(obs, np.float64)
    R, D = o.shape
    na = policy_param_count([D, h0, h1, 2 * D])
    nc = policy_param_count([D, h0, h1, 1])
    ga = np.empty(na) if grads else None
    gc = np.empty(nc) if grads else None
    st = np.empty(3)
    lib().or_a2c_gauss(R, D, h0, h1, _ptr(_arr(actor, np.float32)), _ptr(_arr(critic, np.float32)),
                       _ptr(o), _ptr(_arr(z, np.float64)), _ptr(_arr(ret, np.float64)),
                       _ptr(_arr(adv, np.float64)), float(c_v), float(c_e), _ptr(ga), _ptr(gc),
                       _ptr(st))
    return st, ga, gc
