"""Thin Python binding of the C ABI in include/warpsci.h (argument marshalling only).

Every step of the roll-out runs in the CUDA library ``libwarpsci.so``; this
module loads it (failing loudly if it is missing), declares the ``ws_*``
functions under the same names, and offers ``Rollout``, a convenience owner of
the two device buffers (PyTorch tensors) and the context.  PyTorch is used for
device memory and streams only.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libwarpsci.so")

WS_OK, WS_ERR_INVALID, WS_ERR_NOMEM, WS_ERR_CUDA = 0, 1, 2, 3
WS_ERR_TIMEOUT, WS_ERR_STATE, WS_ERR_RANGE, WS_ERR_UNSUPPORTED = 4, 5, 6, 7
STATUS_NAMES = {0: "WS_OK", 1: "WS_ERR_INVALID", 2: "WS_ERR_NOMEM", 3: "WS_ERR_CUDA",
                4: "WS_ERR_TIMEOUT", 5: "WS_ERR_STATE", 6: "WS_ERR_RANGE", 7: "WS_ERR_UNSUPPORTED"}

WS_ENV_CONTROL, WS_ENV_ECONOMY, WS_ENV_LANDSCAPE, WS_ENV_ACROBOT = 0, 1, 2, 3
WS_PATH_PLAIN_FP32, WS_PATH_BATCHED_FP32, WS_PATH_BATCHED_BF16 = 0, 1, 2
(WS_F_OBS, WS_F_ACTION, WS_F_LOGP, WS_F_REWARD, WS_F_DONE, WS_F_RETURN, WS_F_WEALTH, WS_F_ENERGY,
 WS_F_STATE, WS_F_PARAMS, WS_F_ENV_PARAMS, WS_F_LOGITS, WS_F_FORCE, WS_F_CRITIC,
 WS_F_ADVANTAGE, WS_F_SAMPLE, WS_F_POLICY_OUT) = range(17)

EXPORTED = ["ws_query_bytes", "ws_create", "ws_reset", "ws_step", "ws_rollout", "ws_returns",
            "ws_forces", "ws_a2c_update", "ws_advantages", "ws_ppo_update",
            "ws_fetch", "ws_load", "ws_get_step", "ws_sync", "ws_last_error", "ws_destroy",
            "ws_policy_forward_noalloc", "ws_get_launch", "ws_set_launch", "ws_tune",
            "ws_server_create", "ws_server_submit",
            "ws_server_wait_chunk", "ws_server_fetch", "ws_server_ack", "ws_server_release",
            "ws_server_get_stats", "ws_server_destroy", "ws_probe_rate", "ws_server_listen"]
PROBE_OPS = ["tanh.approx.f32", "tanh.approx.bf16x2", "ex2.approx.ftz.f32",
             "ex2.approx.ftz.bf16x2", "ex2.approx.f16x2", "rcp.approx.ftz.f32",
             "sin.approx.ftz.f32", "fma.rn.f32", "fma.rn.f32x2", "lg2.approx.ftz.f32",
             "rsqrt.approx.ftz.f32", "tanh.approx.f32 (lanes 0-15)"]
WS_REQ_CONSUME_ON_READY = 1
WS_FLAG_DEBUG_LOGITS = 1
WS_FLAG_ENERGY_TARGET = 2
WS_FLAG_FORCE = 4
WS_FLAG_TRAIN = 8
WS_FLAG_BOUNDS_CHECK = 16


class ws_config(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("env", C.c_int32), ("path", C.c_int32),
                ("n_envs", C.c_uint32), ("ring_steps", C.c_uint32),
                ("episode_limit", C.c_uint32), ("chunk_steps", C.c_uint32),
                ("hidden0", C.c_uint32), ("hidden1", C.c_uint32), ("dim", C.c_uint32),
                ("n_gauss", C.c_uint32), ("noise_sigma", C.c_float), ("step_clip", C.c_float),
                ("gamma", C.c_float), ("flags", C.c_uint32), ("param_seed", C.c_uint64),
                ("agents_per_env", C.POINTER(C.c_int32)), ("energy_target", C.c_float),
                ("env_base", C.c_uint32)]


class ws_launch(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("chunk_steps", C.c_uint32), ("grid", C.c_uint32),
                ("econ_tiles", C.c_uint32), ("econ_lpt", C.c_uint32),
                ("energy_chunks", C.c_uint32), ("env_threads", C.c_uint32),
                ("tile_ctas", C.c_uint32), ("wait_ns", C.c_uint32),
                ("ctrl_envs_per_cta", C.c_uint32), ("ctrl_threads_per_env", C.c_uint32),
                ("update_gemm", C.c_uint32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "struct_size"}


class ws_request(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("env", C.c_int32), ("path", C.c_int32),
                ("n_envs", C.c_uint32), ("horizon", C.c_uint32), ("chunk_steps", C.c_uint32),
                ("episode_limit", C.c_uint32), ("hidden0", C.c_uint32), ("hidden1", C.c_uint32),
                ("dim", C.c_uint32), ("n_gauss", C.c_uint32), ("flags", C.c_uint32),
                ("seed", C.c_uint64), ("agents_per_env", C.POINTER(C.c_int32))]


class ws_server_stats(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("submitted", C.c_uint64), ("admitted", C.c_uint64),
                ("completed", C.c_uint64), ("rejected", C.c_uint64), ("failed", C.c_uint64),
                ("chunks", C.c_uint64),
                ("agent_steps", C.c_double), ("elapsed_s", C.c_double), ("p50_ms", C.c_double),
                ("p99_ms", C.c_double), ("used_bytes", C.c_size_t), ("peak_bytes", C.c_size_t),
                ("budget_bytes", C.c_size_t), ("active", C.c_uint32), ("pending", C.c_uint32)]


class WarpSciError(RuntimeError):
    def __init__(self, status, where, msg=""):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)} {msg}".strip())


_lib = None


def lib():
    """Load libwarpsci.so (build it with paper_2408_00930_gb300.build.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: the CUDA library was not built "
                              "(run __graft_entry__.build()); there is no fallback")
        L = C.CDLL(LIB_PATH)
        P = C.c_void_p
        L.ws_query_bytes.argtypes = [C.POINTER(ws_config), C.POINTER(C.c_size_t),
                                     C.POINTER(C.c_size_t), C.POINTER(C.c_uint32)]
        L.ws_create.argtypes = [C.POINTER(ws_config), P, C.c_size_t, P, C.c_size_t, P,
                                C.POINTER(P)]
        L.ws_reset.argtypes = [P, C.c_uint64]
        L.ws_step.argtypes = [P]
        L.ws_rollout.argtypes = [P, C.c_uint32]
        L.ws_returns.argtypes = [P, C.c_uint32]
        L.ws_forces.argtypes = [P, C.c_uint32]
        L.ws_a2c_update.argtypes = [P, C.c_uint32, C.c_float, C.c_float, C.c_float,
                                    C.POINTER(C.c_double)]
        L.ws_advantages.argtypes = [P, C.c_uint32]
        L.ws_ppo_update.argtypes = [P, C.c_uint32, C.c_float, C.c_float, C.c_float, C.c_float,
                                    C.POINTER(C.c_double)]
        L.ws_fetch.argtypes = [P, C.c_int, C.c_uint64, C.c_uint32, P, C.c_size_t, C.c_int]
        L.ws_load.argtypes = [P, C.c_int, P, C.c_size_t, C.c_int, C.c_uint64]
        L.ws_get_step.argtypes = [P, C.POINTER(C.c_uint64)]
        L.ws_sync.argtypes = [P, C.c_uint32]
        L.ws_last_error.argtypes = [P]
        L.ws_last_error.restype = C.c_char_p
        L.ws_destroy.argtypes = [P]
        L.ws_destroy.restype = None
        L.ws_policy_forward_noalloc.argtypes = [P, C.c_uint32, P, C.c_uint32, C.c_uint32,
                                                C.c_uint32, C.c_uint32, P, P]
        L.ws_get_launch.argtypes = [P, C.POINTER(ws_launch)]
        L.ws_set_launch.argtypes = [P, C.POINTER(ws_launch)]
        L.ws_tune.argtypes = [P, C.c_uint32, C.POINTER(ws_launch), C.POINTER(C.c_float)]
        L.ws_server_create.argtypes = [C.c_size_t, C.POINTER(P)]
        L.ws_server_submit.argtypes = [P, C.POINTER(ws_request), C.POINTER(C.c_uint64)]
        L.ws_server_wait_chunk.argtypes = [P, C.c_uint64, C.c_uint32, C.c_uint32]
        L.ws_server_fetch.argtypes = [P, C.c_uint64, C.c_int, C.c_uint32, P, C.c_size_t, C.c_int]
        L.ws_server_ack.argtypes = [P, C.c_uint64, C.c_uint32]
        L.ws_server_release.argtypes = [P, C.c_uint64]
        L.ws_server_get_stats.argtypes = [P, C.POINTER(ws_server_stats)]
        L.ws_probe_rate.argtypes = [C.c_int, C.c_uint32, P, C.c_size_t, C.POINTER(C.c_double), P]
        L.ws_server_listen.argtypes = [P, C.c_char_p]
        L.ws_server_destroy.argtypes = [P]
        L.ws_server_destroy.restype = None
        for n in EXPORTED:
            if n not in ("ws_last_error", "ws_destroy", "ws_server_destroy"):
                getattr(L, n).restype = C.c_int
        _lib = L
    return _lib


# --- the ABI under the same names ------------------------------------------
def ws_query_bytes(cfg: ws_config):
    s, r, n = C.c_size_t(), C.c_size_t(), C.c_uint32()
    st = lib().ws_query_bytes(C.byref(cfg), C.byref(s), C.byref(r), C.byref(n))
    return st, s.value, r.value, n.value


def ws_create(cfg, state_ptr, state_bytes, ring_ptr, ring_bytes, stream_ptr):
    out = C.c_void_p()
    st = lib().ws_create(C.byref(cfg), state_ptr, state_bytes, ring_ptr, ring_bytes, stream_ptr,
                         C.byref(out))
    return st, out.value


def ws_reset(ctx, seed):
    return lib().ws_reset(ctx, seed)


def ws_step(ctx):
    return lib().ws_step(ctx)


def ws_rollout(ctx, n_steps):
    return lib().ws_rollout(ctx, n_steps)


def ws_returns(ctx, n_steps):
    return lib().ws_returns(ctx, n_steps)


def ws_forces(ctx, n_steps):
    return lib().ws_forces(ctx, n_steps)


def ws_a2c_update(ctx, n_steps, lr, c_v, c_e, stats=None):
    """stats: a ctypes c_double * 3 (or None)."""
    return lib().ws_a2c_update(ctx, n_steps, lr, c_v, c_e, stats)


def ws_advantages(ctx, n_steps):
    return lib().ws_advantages(ctx, n_steps)


def ws_ppo_update(ctx, n_steps, lr, clip_eps, c_v, c_e, stats=None):
    """stats: a ctypes c_double * 4 (or None)."""
    return lib().ws_ppo_update(ctx, n_steps, lr, clip_eps, c_v, c_e, stats)


def ws_fetch(ctx, field, t0, n_steps, dst_ptr, dst_bytes, dst_on_device):
    return lib().ws_fetch(ctx, field, t0, n_steps, dst_ptr, dst_bytes, int(dst_on_device))


def ws_load(ctx, field, src_ptr, src_bytes, src_on_device, k):
    return lib().ws_load(ctx, field, src_ptr, src_bytes, int(src_on_device), k)


def ws_get_step(ctx):
    k = C.c_uint64()
    st = lib().ws_get_step(ctx, C.byref(k))
    return st, k.value


def ws_sync(ctx, timeout_ms=0):
    return lib().ws_sync(ctx, timeout_ms)


def ws_get_launch(ctx):
    out = ws_launch()
    out.struct_size = C.sizeof(ws_launch)
    st = lib().ws_get_launch(ctx, C.byref(out))
    return st, out


def ws_set_launch(ctx, launch: ws_launch):
    return lib().ws_set_launch(ctx, C.byref(launch))


def ws_tune(ctx, trial_steps):
    out = ws_launch()
    ms = C.c_float()
    st = lib().ws_tune(ctx, trial_steps, C.byref(out), C.byref(ms))
    return st, out, ms.value


def ws_last_error(ctx):
    return lib().ws_last_error(ctx).decode()


def ws_destroy(ctx):
    lib().ws_destroy(ctx)


def ws_policy_forward_noalloc(obs_ptr, n_rows, params_ptr, in_dim, hidden0, hidden1, out_dim,
                              out_ptr, stream_ptr):
    return lib().ws_policy_forward_noalloc(obs_ptr, n_rows, params_ptr, in_dim, hidden0, hidden1,
                                           out_dim, out_ptr, stream_ptr)


def ws_probe_rate(op, iters, dev_buf_ptr, buf_bytes, stream_ptr):
    """Results per clock per SM of probe op (index into PROBE_OPS)."""
    out = C.c_double()
    st = lib().ws_probe_rate(op, iters, dev_buf_ptr, buf_bytes, C.byref(out), stream_ptr)
    return st, out.value


# --- convenience owner --------------------------------------------------------
def make_config(env, path, n_envs, ring_steps, episode_limit, hidden0, hidden1, *,
                chunk_steps=0, dim=0, n_gauss=0, noise_sigma=0.05, step_clip=0.1, gamma=0.99,
                param_seed=1, agents_per_env=None, flags=0, energy_target=None, env_base=0):
    cfg = ws_config()
    cfg.struct_size = C.sizeof(ws_config)
    cfg.env, cfg.path, cfg.n_envs = env, path, n_envs
    cfg.ring_steps, cfg.episode_limit, cfg.chunk_steps = ring_steps, episode_limit, chunk_steps
    cfg.hidden0, cfg.hidden1, cfg.dim, cfg.n_gauss = hidden0, hidden1, dim, n_gauss
    cfg.noise_sigma, cfg.step_clip, cfg.gamma = noise_sigma, step_clip, gamma
    cfg.flags, cfg.param_seed, cfg.env_base = flags, param_seed, env_base
    if energy_target is not None:  # landscape: done when E(x') < energy_target
        cfg.flags |= WS_FLAG_ENERGY_TARGET
        cfg.energy_target = energy_target
    keep = None
    if agents_per_env is not None:
        keep = np.ascontiguousarray(agents_per_env, dtype=np.int32)
        cfg.agents_per_env = keep.ctypes.data_as(C.POINTER(C.c_int32))
    return cfg, keep


class Rollout:
    """Owns the two device buffers (torch uint8 tensors) and one ws context.

    Field shapes follow include/warpsci.h; ``fetch`` returns numpy arrays.
    """

    def __init__(self, env, path, n_envs, ring_steps, episode_limit, hidden0, hidden1,
                 device="cuda", stream=None, **kw):
        import torch
        self.torch = torch
        self.cfg, self._keep = make_config(env, path, n_envs, ring_steps, episode_limit, hidden0,
                                           hidden1, **kw)
        st, sb, rb, ns = ws_query_bytes(self.cfg)
        if st != WS_OK:
            raise WarpSciError(st, "ws_query_bytes")
        self.n_slots = ns
        self.state_buf = torch.empty(max(sb, 256), dtype=torch.uint8, device=device)
        self.ring_buf = torch.empty(max(rb, 256), dtype=torch.uint8, device=device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        st, ctx = ws_create(self.cfg, self.state_buf.data_ptr(), sb, self.ring_buf.data_ptr(), rb,
                            self.stream.cuda_stream)
        if st != WS_OK:
            raise WarpSciError(st, "ws_create")
        self.ctx = ctx
        self.env, self.n_envs = env, n_envs
        self.dim = kw.get("dim", 0)
        self.n_gauss = kw.get("n_gauss", 0)
        self.hidden = (hidden0, hidden1)

    # checks
    def _ok(self, st, where):
        if st != WS_OK:
            raise WarpSciError(st, where, ws_last_error(self.ctx))

    def reset(self, seed):
        self._ok(ws_reset(self.ctx, seed), "ws_reset")

    def step(self):
        self._ok(ws_step(self.ctx), "ws_step")

    def rollout(self, n):
        self._ok(ws_rollout(self.ctx, n), "ws_rollout")

    def returns(self, n):
        self._ok(ws_returns(self.ctx, n), "ws_returns")

    def forces(self, n):
        self._ok(ws_forces(self.ctx, n), "ws_forces")

    def a2c_update(self, n, lr, c_v=0.5, c_e=0.0):
        """One actor-critic step on the last n steps; returns the means of
        -A log pi, (G - V)^2 and the entropy."""
        st = (C.c_double * 3)()
        self._ok(ws_a2c_update(self.ctx, n, lr, c_v, c_e, st), "ws_a2c_update")
        return np.array(st[:])

    def advantages(self, n):
        """Returns, then A = G - V(s) of the last n steps into ADVANTAGE."""
        self._ok(ws_advantages(self.ctx, n), "ws_advantages")

    def ppo_update(self, n, lr, clip_eps=0.2, c_v=0.5, c_e=0.0):
        """One PPO epoch on the last n steps (after advantages(n)); returns the
        means of -surrogate, (G - V)^2, the entropy and the clipped fraction."""
        st = (C.c_double * 4)()
        self._ok(ws_ppo_update(self.ctx, n, lr, clip_eps, c_v, c_e, st), "ws_ppo_update")
        return np.array(st[:])

    def sync(self, timeout_ms=0):
        self._ok(ws_sync(self.ctx, timeout_ms), "ws_sync")

    def launch(self):
        st, l = ws_get_launch(self.ctx)
        self._ok(st, "ws_get_launch")
        return l

    def set_launch(self, **kw):
        l = self.launch()
        for k, v in kw.items():
            setattr(l, k, v)
        self._ok(ws_set_launch(self.ctx, l), "ws_set_launch")

    def tune(self, trial_steps):
        """Autotune the launch configuration (ends with a reset under the current seed)."""
        st, l, ms = ws_tune(self.ctx, trial_steps)
        self._ok(st, "ws_tune")
        return l.as_dict(), ms

    @property
    def k(self):
        st, k = ws_get_step(self.ctx)
        self._ok(st, "ws_get_step")
        return k

    # layouts ---------------------------------------------------------------
    def obs_dim(self):
        return {WS_ENV_CONTROL: 4, WS_ENV_ECONOMY: 16, WS_ENV_LANDSCAPE: self.dim,
                WS_ENV_ACROBOT: 6}[self.env]

    def n_out(self):
        return {WS_ENV_CONTROL: 2, WS_ENV_ECONOMY: 20, WS_ENV_LANDSCAPE: 2 * self.dim,
                WS_ENV_ACROBOT: 3}[self.env]

    def _ring_spec(self, field):
        S = self.n_slots
        if field == WS_F_OBS:
            return np.float32, (self.obs_dim(), S)
        if field == WS_F_ACTION:
            return ((np.float32, (self.dim, S)) if self.env == WS_ENV_LANDSCAPE
                    else (np.int32, (S,)))
        if field in (WS_F_LOGP, WS_F_REWARD, WS_F_RETURN, WS_F_ENERGY, WS_F_ADVANTAGE):
            return np.float32, (S,)
        if field == WS_F_DONE:
            return np.uint8, (S,)
        if field == WS_F_WEALTH:
            return np.int64, (S,)
        if field in (WS_F_FORCE, WS_F_SAMPLE):
            return np.float32, (self.dim, S)
        if field == WS_F_POLICY_OUT:
            return np.float32, (self.n_out(), S)
        raise ValueError(field)

    def fetch(self, field, t0, n):
        dt, shp = self._ring_spec(field)
        out = np.empty((n,) + shp, dtype=dt)
        self._ok(ws_fetch(self.ctx, field, t0, n, out.ctypes.data, out.nbytes, 0), "ws_fetch")
        return out

    def fetch_device(self, field, t0, n, dst):
        self._ok(ws_fetch(self.ctx, field, t0, n, dst.data_ptr(), dst.numel() * dst.element_size(),
                          1), "ws_fetch")

    def fetch_raw(self, field, nbytes):
        out = np.empty(nbytes, dtype=np.uint8)
        self._ok(ws_fetch(self.ctx, field, 0, 0, out.ctypes.data, nbytes, 0), "ws_fetch")
        return out

    def load_raw(self, field, arr_bytes, k=2**64 - 1):
        buf = np.ascontiguousarray(arr_bytes).view(np.uint8)
        self._ok(ws_load(self.ctx, field, buf.ctypes.data, buf.nbytes, 0, k), "ws_load")

    def close(self):
        if getattr(self, "ctx", None):
            ws_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --- serving --------------------------------------------------------------------
def make_request(env, path, n_envs, horizon, chunk_steps, episode_limit, hidden0, hidden1, *,
                 dim=0, n_gauss=0, seed=1, flags=0, agents_per_env=None):
    q = ws_request()
    q.struct_size = C.sizeof(ws_request)
    q.env, q.path, q.n_envs, q.horizon, q.chunk_steps = env, path, n_envs, horizon, chunk_steps
    q.episode_limit, q.hidden0, q.hidden1, q.dim, q.n_gauss = episode_limit, hidden0, hidden1, dim, n_gauss
    q.flags, q.seed = flags, seed
    keep = None
    if agents_per_env is not None:
        keep = np.ascontiguousarray(agents_per_env, dtype=np.int32)
        q.agents_per_env = keep.ctypes.data_as(C.POINTER(C.c_int32))
    return q, keep


class Server:
    """Owner of a ws_server (device arena of budget_bytes on the current device)."""

    def __init__(self, budget_bytes):
        out = C.c_void_p()
        st = lib().ws_server_create(budget_bytes, C.byref(out))
        if st != WS_OK:
            raise WarpSciError(st, "ws_server_create")
        self.s = out.value

    def submit(self, q):
        rid = C.c_uint64()
        st = lib().ws_server_submit(self.s, C.byref(q), C.byref(rid))
        return st, rid.value

    def wait_chunk(self, rid, chunk, timeout_ms=0):
        return lib().ws_server_wait_chunk(self.s, rid, chunk, timeout_ms)

    def fetch(self, rid, field, chunk, out):
        return lib().ws_server_fetch(self.s, rid, field, chunk, out.ctypes.data, out.nbytes, 0)

    def ack(self, rid, chunk):
        return lib().ws_server_ack(self.s, rid, chunk)

    def release(self, rid):
        return lib().ws_server_release(self.s, rid)

    def listen(self, path):
        """Serve clients in other processes over a Unix-domain socket at path."""
        rc = lib().ws_server_listen(self.s, path.encode())
        if rc != WS_OK:
            raise WarpSciError(rc, "ws_server_listen")

    def stats(self):
        st = ws_server_stats()
        st.struct_size = C.sizeof(ws_server_stats)
        rc = lib().ws_server_get_stats(self.s, C.byref(st))
        if rc != WS_OK:
            raise WarpSciError(rc, "ws_server_get_stats")
        return {f: getattr(st, f) for f, _ in ws_server_stats._fields_ if f != "struct_size"}

    def close(self):
        if getattr(self, "s", None):
            lib().ws_server_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
