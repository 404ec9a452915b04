"""Benchmark of the in-place RL roll-out loop (agent-steps/s) on one GB300.

One bench step = one full roll-out of the workload through the C ABI:
ws_reset (fresh episode draw), ws_rollout over the horizon in chunks of 50
steps (every env: policy MLP, sampling, env step with auto-reset, store), and
ws_returns over the horizon.  Default workload: the control env at scale,
131,072 envs x 1 agent, horizon 500, policy 4-256-256-2, BF16 tensor-core
path (the FP32 one-launch-per-step path is timed beside it).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                    [--impl ours|reference]

Under torchrun each rank runs one shard of a workload N times the size: rank r
holds the workload's env count at global env ids [r n, (r + 1) n) under the
same parameters (envs are independent and share only read-only parameters, so
there is no collective on the data path) and rank 0 prints one JSON line with
the whole-job throughput.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "agent-steps/sec on 1 GB300, served BF16 vs plain FP32; p50/p99 rollout latency"
CHUNK = 50
# DRAM bytes (read + write) per slot-step of the returns scan, from an ncu
# capture of k_returns on the control workload (summarised under profiles/);
# the traffic scales with the slot-steps scanned
RETURNS_NCU_BYTES_PER_SLOT_STEP = 7.1

WORKLOADS = {
    "control_scale": dict(env=0, n_envs=131072, horizon=500, limit=200, h=(256, 256),
                          desc="control env, 131,072 envs x 1 agent, horizon 500, "
                               "policy 4-256-256-2, episode limit 200"),
    "control_small": dict(env=0, n_envs=1000, horizon=200, limit=200, h=(64, 64),
                          desc="control env, 1,000 envs x 1 agent, horizon 200, "
                               "policy 4-64-64-2, episode limit 200"),
    "economy": dict(env=1, n_envs=2048, horizon=540, limit=540, h=(128, 128),
                    desc="economy, 2,048 envs x U{8..256} agents + 1 planner, horizon 540, "
                         "policy 16-128-128-20 (planner 16-128-128-10)"),
    "landscape": dict(env=2, n_envs=8192, horizon=1000, limit=1000, h=(256, 256), dim=24,
                      n_gauss=4096,
                      desc="landscape, 8,192 envs x 1 agent, D=24, M=4,096 Gaussians, "
                           "horizon 1,000, policy 24-256-256-48"),
    "acrobot": dict(env=3, n_envs=10000, horizon=500, limit=500, h=(64, 64),
                    desc="acrobot, 10,000 envs x 1 agent, horizon 500, policy 6-64-64-3, "
                         "episode limit 500"),
}


def flops_per_agent_step(wl):
    if wl["env"] == 0:
        w = [4, *wl["h"], 2]
    elif wl["env"] == 1:
        w = [16, *wl["h"], 20]
    elif wl["env"] == 3:
        w = [6, *wl["h"], 3]
    else:
        w = [wl["dim"], *wl["h"], 2 * wl["dim"]]
    return 2 * sum(a * b for a, b in zip(w[:-1], w[1:]))


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), \
            d.get("bf16_tflops_sustained", 1700.0), "measured"
    return 6800.0, 1900.0, 1700.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in out.strip().splitlines():
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def shard_of(n_envs, world, rank):
    """(env_base, n_envs) of a rank: weak scaling, every rank holds the
    workload's env count at its own range of global env ids."""
    assert 0 <= rank < world
    return rank * n_envs, n_envs


def job_throughput(units_per_rank_step, steps, world, max_ms):
    """Whole-job rate: the units all ranks processed over the slowest rank's time."""
    return units_per_rank_step * steps * world / (max_ms / 1e3)


def max_over_ranks(v, world):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64,
                     device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------- oracle leg
def _oracle_shard(args):
    wl_name, env_ids, steps = args
    sys.path.insert(0, ROOT)
    import oracle
    wl = WORKLOADS[wl_name]
    t0 = time.perf_counter()
    if wl["env"] == 0:
        p = oracle.policy_init(1, 0, [4, *wl["h"], 2])
        oracle.control_rollout(p, *wl["h"], seed=1, env_ids=env_ids, n_steps=steps,
                               episode_limit=wl["limit"])
        agent_steps = len(env_ids) * steps
    elif wl["env"] == 1:
        ap = oracle.policy_init(1, 0, [16, *wl["h"], 20])
        pp = oracle.policy_init(1, 1, [16, *wl["h"], 10])
        na = [oracle.econ_agent_count(1, int(e)) for e in env_ids]
        oracle.econ_rollout(ap, pp, seed=1, env_ids=env_ids, n_agents=na, n_steps=steps,
                            episode_limit=wl["limit"])
        agent_steps = (sum(na) + len(env_ids)) * steps
    elif wl["env"] == 3:
        p = oracle.policy_init(1, 0, [6, *wl["h"], 3])
        oracle.acrobot_rollout(p, *wl["h"], seed=1, env_ids=env_ids, n_steps=steps,
                               episode_limit=wl["limit"])
        agent_steps = len(env_ids) * steps
    else:
        c, w, a = oracle.landscape_init(1, wl["dim"], wl["n_gauss"])
        p = oracle.policy_init(1, 0, [wl["dim"], *wl["h"], 2 * wl["dim"]])
        oracle.landscape_rollout(c, w, a, p, *wl["h"], seed=1, env_ids=env_ids, n_steps=steps,
                                 episode_limit=wl["limit"])
        agent_steps = len(env_ids) * steps
    return agent_steps, time.perf_counter() - t0


def oracle_throughput(wl_name, target_s=20.0):
    """The FP64 oracle, as it stands, on the host cores: one process per core
    (spawned), each rolling out its own envs; a bounded sample of the workload."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    wl = WORKLOADS[wl_name]
    steps = min(wl["horizon"], 50)
    # calibrate on one env
    a, dt = _oracle_shard((wl_name, np.array([0], np.uint32), 5))
    per_agent_step = dt / max(a, 1)
    cores = os.cpu_count() or 1
    agents_per_env = a / 5.0
    envs_per_core = max(1, int(target_s / (per_agent_step * steps * agents_per_env)))
    envs_per_core = min(envs_per_core, max(1, wl["n_envs"] // cores))
    shards = [(wl_name, np.arange(i * envs_per_core, (i + 1) * envs_per_core, dtype=np.uint32), steps)
              for i in range(cores)]
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_shard, shards)
    wall = time.perf_counter() - t0
    total = sum(r[0] for r in res)
    # one process alone: the mean of the processes' own rates
    single = float(np.mean([r[0] / r[1] for r in res]))
    sample = (f"{cores} processes x {envs_per_core} envs x {steps} steps of the workload "
              f"({total} agent-steps, FP64 C oracle, {wall:.1f} s wall; "
              f"{single:.0f} agent-steps/s per process)")
    return total / wall, cores, sample, wall, single, steps


# ----------------------------------------------------------------- GPU leg
def run_gpu(args, wl, world, rank, local):
    import torch
    from paper_2408_00930_gb300 import warpsci as W
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    env_base, _ = shard_of(wl["n_envs"], world, rank)
    kw = dict(chunk_steps=CHUNK, param_seed=1, env_base=env_base)
    if wl["env"] == 2:
        # the FORCE field only adds ring memory; the roll-out kernels ignore it
        kw.update(dim=wl["dim"], n_gauss=wl["n_gauss"], flags=W.WS_FLAG_FORCE)
    path = W.WS_PATH_BATCHED_BF16
    cfg, _ = W.make_config(wl["env"], path, wl["n_envs"], wl["horizon"], wl["limit"], *wl["h"],
                           **kw)
    if W.ws_query_bytes(cfg)[0] != W.WS_OK:
        path = W.WS_PATH_BATCHED_FP32
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def one_path(path, steps, warmup, measure_kernel):
        with torch.cuda.stream(stream):
            r = W.Rollout(wl["env"], path, wl["n_envs"], wl["horizon"], wl["limit"], *wl["h"],
                          device=dev, stream=stream, **kw)
        H = wl["horizon"]
        n_chunks = (H + CHUNK - 1) // CHUNK
        agent_steps = r.n_slots * H
        launch = None
        if measure_kernel and not args.no_tune:
            # autotune the launch configuration (outside the timed region; the
            # trials end with a reset) over one 50-step roll-out per candidate
            launch, _ = r.tune(min(CHUNK, H))
        elif measure_kernel:
            launch = r.launch().as_dict()
        if measure_kernel and args.launch:
            # fixed launch fields (k=v,...), e.g. to profile one kernel choice
            kv = dict(item.split("=") for item in args.launch.split(","))
            r.set_launch(**{k: int(v) for k, v in kv.items()})
            launch = r.launch().as_dict()

        def bench_step(i, evs=None):
            r.reset(1000 + i)
            if evs is not None:
                evs[0].record(stream)
            for c in range(n_chunks):
                r.rollout(min(CHUNK, H - c * CHUNK))
                if evs is not None:
                    evs[1 + c].record(stream)
            r.returns(H)
            if evs is not None:
                evs[-1].record(stream)

        for i in range(warmup):
            bench_step(i)
        torch.cuda.synchronize(dev)
        times, chunk_ms, roll_ms = [], [], []
        clocks = Clocks(local)
        barrier(world)
        torch.cuda.synchronize(dev)
        clocks.start()
        time.sleep(0.3)  # let the sampler start before the timed region
        for i in range(steps):
            flush.zero_()                      # L2 flush between timed steps
            torch.cuda.synchronize(dev)
            e_start = torch.cuda.Event(enable_timing=True)
            evs = [torch.cuda.Event(enable_timing=True) for _ in range(n_chunks + 2)]
            e_start.record(stream)
            bench_step(warmup + i, evs)
            torch.cuda.synchronize(dev)
            times.append(e_start.elapsed_time(evs[-1]))
            roll_ms.append(evs[0].elapsed_time(evs[n_chunks]))
            for c in range(n_chunks):
                chunk_ms.append(evs[c].elapsed_time(evs[c + 1]))
        torch.cuda.synchronize(dev)
        clk = clocks.stop()
        barrier(world)
        total_ms = max_over_ranks(sum(times), world)
        ret_ms = [t - rm for t, rm in zip(times, roll_ms)]
        force_ms = None
        if wl["env"] == 2 and measure_kernel:
            # ws_forces over the last 50-step chunk (outside the timed step; the
            # force is an optional output), L2 flushed before each launch
            force_ms = []
            for _ in range(3):
                flush.zero_()
                torch.cuda.synchronize(dev)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                r.forces(min(CHUNK, H))
                e1.record(stream)
                torch.cuda.synchronize(dev)
                force_ms.append(e0.elapsed_time(e1))
        res = dict(agent_steps=agent_steps, total_ms=total_ms, times=times, chunk_ms=chunk_ms,
                   force_ms=force_ms,
                   roll_ms=roll_ms, ret_ms=ret_ms, clocks=clk, n_chunks=n_chunks, rollout=r,
                   launch=launch)
        return res

    sfu_rates = None
    if path == W.WS_PATH_BATCHED_BF16:
        sfu_rates = probe_rates(local, ops=("tanh.approx.f32", "ex2.approx.ftz.f32",
                                            "sin.approx.ftz.f32", "lg2.approx.ftz.f32",
                                            "rsqrt.approx.ftz.f32", "fma.rn.f32"))
    main = one_path(path, args.steps, args.warmup, True)
    main["sfu_rates"] = sfu_rates
    r = main["rollout"]
    n_steps_total = args.steps
    value = job_throughput(main["agent_steps"], n_steps_total, world, main["total_ms"])
    # plain FP32 path beside it (fewer steps: it is the slow baseline)
    plain = None
    if not args.no_plain:
        pk = one_path(W.WS_PATH_PLAIN_FP32, max(1, min(args.steps, 2)), 1, False)
        plain = dict(value=pk["agent_steps"] * len(pk["times"]) * world / (pk["total_ms"] / 1e3),
                     unit="agent-steps/s", ms_per_step=pk["total_ms"] / len(pk["times"]),
                     path="plain_fp32 (one launch per sub-step per step, FP32 SIMT)",
                     us_per_env_step=pk["total_ms"] / len(pk["times"]) * 1e3 / wl["horizon"])
        pk["rollout"].close()
        if wl["n_envs"] <= 10000:
            # small configs are launch-bound: the same FP32 kernels captured in
            # CUDA graphs (the batched FP32 path) beside the per-step launches
            gk = one_path(W.WS_PATH_BATCHED_FP32, max(1, min(args.steps, 5)), 1, False)
            plain["batched_fp32_graphs"] = dict(
                value=gk["agent_steps"] * len(gk["times"]) * world / (gk["total_ms"] / 1e3),
                unit="agent-steps/s",
                us_per_env_step=gk["total_ms"] / len(gk["times"]) * 1e3 / wl["horizon"])
            gk["rollout"].close()
    # end to end through the C ABI with host buffers: policy weights H2D from
    # pinned host memory, the roll-out, returns, and the per-env return at t=0 D2H.
    par_bytes = r.fetch_raw(W.WS_F_PARAMS, _param_bytes(wl)).copy()
    host_par = torch.from_numpy(par_bytes).pin_memory()
    host_ret = torch.empty(r.n_slots * 4, dtype=torch.uint8).pin_memory()
    H = wl["horizon"]
    e2e_t = []
    for i in range(max(2, min(args.steps, 5))):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        st = W.ws_load(r.ctx, W.WS_F_PARAMS, host_par.data_ptr(), host_par.numel(), 0,
                       2**64 - 1)
        assert st == W.WS_OK, W.ws_last_error(r.ctx)
        r.reset(5000 + i)
        for c in range(main["n_chunks"]):
            r.rollout(min(CHUNK, H - c * CHUNK))
        r.returns(H)
        st = W.ws_fetch(r.ctx, W.WS_F_RETURN, 0, 1, host_ret.data_ptr(), host_ret.numel(), 0)
        assert st == W.WS_OK, W.ws_last_error(r.ctx)
        e2e_t.append(time.perf_counter() - t0)
    e2e_s = max_over_ranks(sum(e2e_t), world)
    e2e = {"value": main["agent_steps"] * len(e2e_t) * world / e2e_s, "unit": "agent-steps/s",
           "h2d_bytes_per_step": int(host_par.numel()), "d2h_bytes_per_step": int(host_ret.numel())}
    r.close()
    return path, value, main, plain, e2e


def run_a2c(wl, local):
    """One actor-critic update (ws_a2c_update) over the last 50 steps of a
    roll-out of the workload, then the PPO advantages (ws_advantages) and one
    PPO epoch (ws_ppo_update) over the same rows, each timed with CUDA events
    on the context's stream (L2 flushed before each; three measured rounds
    after one untimed).  FP32 SIMT GEMMs: algorithmic flops per row of an
    update = forward of policy and critic, their weight gradients (same count)
    and the data gradients of the two hidden layers; of the advantages, the
    critic's forward."""
    import torch
    from paper_2408_00930_gb300 import warpsci as W
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    T = min(CHUNK, wl["horizon"])
    with torch.cuda.stream(stream):
        r = W.Rollout(wl["env"], W.WS_PATH_BATCHED_BF16, wl["n_envs"], T, wl["limit"], *wl["h"],
                      device=dev, stream=stream, chunk_steps=CHUNK, flags=W.WS_FLAG_TRAIN)
    od, na = (4, 2) if wl["env"] == 0 else (6, 3)
    h0, h1 = wl["h"]
    fwd = lambda n_out: 2 * (od * h0 + h0 * h1 + h1 * n_out)
    flops_row = 2 * (fwd(na) + fwd(1)) + 2 * 2 * (h1 * na + h0 * h1 + h1 + h0 * h1)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def timed(fn):
        flush.zero_()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        assert st == W.WS_OK, st
        return e0.elapsed_time(e1)

    ms, ms_adv, ms_ppo = [], [], []
    for i in range(4):
        r.reset(77 + i)
        r.rollout(T)
        t_a2c = timed(lambda: W.ws_a2c_update(r.ctx, T, 1e-3, 0.5, 0.01, None))
        t_adv = timed(lambda: W.ws_advantages(r.ctx, T))
        t_ppo = timed(lambda: W.ws_ppo_update(r.ctx, T, 1e-3, 0.2, 0.5, 0.01, None))
        if i:
            ms.append(t_a2c)
            ms_adv.append(t_adv)
            ms_ppo.append(t_ppo)
    r.close()
    rows = T * wl["n_envs"]
    t = statistics.median(ms)
    hbm, bf16_burst, bf16_sus, peak_src = load_peaks()
    n_sms = torch.cuda.get_device_properties(local).multi_processor_count
    peak = 2 * 128 * n_sms * 2070e6 / 1e12   # FP32 FMA: 128 lanes / SM / clock
    achieved = flops_row * rows / (t * 1e-3) / 1e12
    return {"rows": rows, "ms": t, "rows_per_s": rows / (t * 1e-3), "unit": "rows/s",
            "roofline": {"bound": "fp32", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak,
                         "note": "FP32-equivalent flops of the update over the FP32 CUDA-core "
                                 "peak; the wide layers run on tcgen05 (three BF16 products "
                                 "per FP32 product)",
                         "peak_source": f"128 FP32 lanes x 2 flops / clock / SM x {n_sms} SMs x "
                                        "2070 MHz"},
            "kernels": "k_a2c_gather, k_gemm_tc (forward, weight and data gradients of the "
                       "wide layers on tcgen05, FP32 operands split into BF16 hi + lo), "
                       "k_fwd_thin, k_fwd_thin_k, k_dgrad_thin_k, k_wgrad_thin_n/_m, "
                       "k_colsum_slices, k_reduce_slices, k_a2c_head, k_sgd",
            "ppo": {"advantages_ms": statistics.median(ms_adv),
                    "epoch_ms": statistics.median(ms_ppo),
                    "epoch_rows_per_s": rows / (statistics.median(ms_ppo) * 1e-3),
                    "epoch_frac_fp32": flops_row * rows / (statistics.median(ms_ppo) * 1e-3) / 1e12
                    / peak,
                    "advantages_tflops": fwd(1) * rows / (statistics.median(ms_adv) * 1e-3) / 1e12,
                    "kernels": "ws_advantages: k_a2c_gather, the critic's forward, k_adv_store; "
                               "ws_ppo_update: as the A2C update with k_ppo_head"}}


def serve_mix(args, n_requests, rank, local):
    """Serving mix: Poisson arrivals (200 req/s) of requests across the three env
    types, admitted under a 150 GB budget, delivered in chunks of 50 steps; once
    on the BF16 paths (served) and once on the plain FP32 path."""
    import torch
    from paper_2408_00930_gb300 import serving_mix
    from paper_2408_00930_gb300 import warpsci as W
    torch.cuda.set_device(local)
    budget = int(args.serve_budget_gb * (1 << 30))
    stream = list(serving_mix.request_stream(1234 + rank, n_requests, rate=200.0))
    out = {}
    for label, bf16 in (("served", True), ("plain_fp32", False)):
        if not bf16 and args.no_plain:
            continue
        srv = W.Server(budget)
        t0 = time.perf_counter()
        keep = []
        rejected = 0
        for r in stream:
            dt = r["t_arrival"] - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            if bf16:
                path = W.WS_PATH_BATCHED_BF16
            else:
                path = W.WS_PATH_PLAIN_FP32
            q, k = W.make_request(r["env"], path, r["n_envs"], r["horizon"], CHUNK,
                                  r["episode_limit"], *r["hidden"], dim=r["dim"],
                                  n_gauss=r["n_gauss"], seed=r["seed"],
                                  flags=W.WS_REQ_CONSUME_ON_READY)
            keep.append(k)
            st, _ = srv.submit(q)
            if st != W.WS_OK:
                rejected += 1
        while True:
            s_ = srv.stats()
            if s_["completed"] + s_["rejected"] + s_["failed"] >= len(stream):
                break
            if time.perf_counter() - t0 > args.serve_timeout_s:
                break
            time.sleep(0.005)
        wall = time.perf_counter() - t0
        s_ = srv.stats()
        srv.close()
        out[label] = {"value": s_["agent_steps"] / wall, "unit": "agent-steps/s",
                      "p50_ms": s_["p50_ms"], "p99_ms": s_["p99_ms"], "wall_s": wall,
                      "requests": len(stream), "rejected": rejected, "failed": s_["failed"],
                      "completed": s_["completed"], "chunks": s_["chunks"],
                      "peak_bytes": s_["peak_bytes"], "agent_steps": s_["agent_steps"]}
    return out


def probe_rates(local, iters=2048, ops=None):
    """Results per clock per SM of the probed operations (ws_probe_rate), each
    the best of three launches."""
    import torch
    from paper_2408_00930_gb300 import warpsci as W
    dev = torch.device("cuda", local)
    n_sms = torch.cuda.get_device_properties(local).multi_processor_count
    buf = torch.empty(n_sms * 4 * 16, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    out = {}
    for op, name in enumerate(W.PROBE_OPS):
        if ops is not None and name not in ops:
            continue
        best = 0.0
        for _ in range(3):
            st, v = W.ws_probe_rate(op, iters, buf.data_ptr(), buf.numel(), stream.cuda_stream)
            assert st == W.WS_OK, st
            best = max(best, v)
        out[name] = best
    return out


def run_peaks(args, local):
    """Measured rates of the SFU operations and the FMA pipe that the rooflines
    divide by (results per SM clock; x SMs x clock = the chip's rate)."""
    import torch
    torch.cuda.set_device(local)
    rates = probe_rates(local)
    n_sms = torch.cuda.get_device_properties(local).multi_processor_count
    print(json.dumps({"peaks": "results per clock per SM (4 blocks x 256 threads x 8 chains per SM, "
                               "clock64 spans, best of 3)", "n_sms": n_sms,
                      "gpu": torch.cuda.get_device_name(local), "rates": rates}), flush=True)


def run_serving(args, world, rank, local):
    out = serve_mix(args, args.serve_requests, rank, local)
    if rank == 0:
        sv = out["served"]
        print(json.dumps({
            "metric": METRIC, "value": sv["value"], "unit": "agent-steps/s", "n_gpus": world,
            "steps": args.serve_requests, "warmup": 0, "ms_per_step": sv["wall_s"] * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
            "data": "synthetic",
            "config": {"workload": "serving mix: Poisson 200 req/s across control / economy / "
                                   "landscape, 256-65,536 envs, horizons 100-1,000, chunks of 50, "
                                   f"{args.serve_budget_gb:g} GB admission budget",
                       "paths": "served: BF16 tensor-core paths (one fused persistent kernel per "
                                "chunk for each env type); plain_fp32: one launch per sub-step "
                                "per step"},
            "latency": {"chunk_steps": CHUNK, "p50_ms": sv["p50_ms"], "p99_ms": sv["p99_ms"]},
            "serving": out}), flush=True)


def _param_bytes(wl):
    if wl["env"] == 0:
        w = [4, *wl["h"], 2]
        extra = 0
    elif wl["env"] == 1:
        w = [16, *wl["h"], 20]
        pw = [16, *wl["h"], 10]
        extra = sum(a * b + b for a, b in zip(pw[:-1], pw[1:]))
    elif wl["env"] == 3:
        w = [6, *wl["h"], 3]
        extra = 0
    else:
        w = [wl["dim"], *wl["h"], 2 * wl["dim"]]
        extra = 0
    return 4 * (sum(a * b + b for a, b in zip(w[:-1], w[1:])) + extra)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="control_scale", choices=sorted(WORKLOADS) + ["serving"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP32 comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--a2c", action="store_true",
                    help="also time one actor-critic update (ws_a2c_update), the PPO advantages "
                         "and one PPO epoch over 50 steps "
                         "(control and acrobot workloads)")
    ap.add_argument("--launch", default="",
                    help="launch fields set after tuning, as k=v,... (ws_launch names)")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the default launch configuration (profiling captures)")
    ap.add_argument("--horizon", type=int, default=0,
                    help="override the horizon (smaller cases for profiling captures)")
    ap.add_argument("--n-envs", type=int, default=0, help="override the env count")
    ap.add_argument("--serve-requests", type=int, default=48)
    ap.add_argument("--serve-budget-gb", type=float, default=150.0)
    ap.add_argument("--serve-timeout-s", type=float, default=600.0)
    ap.add_argument("--peaks", action="store_true",
                    help="measure the SFU and FMA-pipe rates (ws_probe_rate) and exit")
    ap.add_argument("--serve-sub-requests", type=int, default=12,
                    help="requests of the serving mix timed after the main workload and "
                         "reported in its line's serving object (0: skip)")
    args = ap.parse_args()
    if args.peaks:
        _, _, local = dist_init()
        run_peaks(args, local)
        return
    if args.workload == "serving":
        world, rank, local = dist_init()
        run_serving(args, world, rank, local)
        return
    wl = dict(WORKLOADS[args.workload])
    if args.horizon:
        wl["horizon"] = args.horizon
        wl["desc"] += f" [horizon overridden to {args.horizon}]"
    if args.n_envs:
        wl["n_envs"] = args.n_envs
        wl["desc"] += f" [envs overridden to {args.n_envs}]"
    world, rank, local = dist_init()
    if args.impl == "reference":
        if rank == 0:
            # one timed sample: every process rolls its envs over `steps` env
            # steps; the line reports those steps and the wall time per step
            v, cores, sample, wall, single, steps = oracle_throughput(args.workload)
            print(json.dumps({
                "impl": "reference", "metric": METRIC, "value": v, "unit": "agent-steps/s",
                "n_gpus": args.gpus, "steps": steps, "warmup": 0,
                "ms_per_step": wall * 1e3 / steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": wl["desc"], "arm": "FP64 C oracle on host cores"},
                "cpu_baseline": {"value": v, "unit": "agent-steps/s", "cores": cores,
                                 "kind": "oracle", "sample": sample, "single_core_value": single},
                "e2e": {"value": v, "unit": "agent-steps/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}), flush=True)
        return
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        # before the first GPU call: the pool is spawned, never forked after CUDA init
        v, cores, sample, _, single, _ = oracle_throughput(args.workload)
        cpu = {"value": v, "unit": "agent-steps/s", "cores": cores, "kind": "oracle",
               "sample": sample, "single_core_value": single}
    path, value, main_res, plain, e2e = run_gpu(args, wl, world, rank, local)
    a2c = run_a2c(wl, local) if args.a2c and wl["env"] in (0, 3) and rank == 0 else None
    serving = None
    if args.serve_sub_requests > 0 and world == 1:
        sv = serve_mix(args, args.serve_sub_requests, rank, local)
        serving = {"workload": f"{args.serve_sub_requests} requests of the serving mix (Poisson "
                               "200 req/s across control / economy / landscape, 256-65,536 envs, "
                               "horizons 100-1,000, chunks of 50, "
                               f"{args.serve_budget_gb:g} GB admission budget)", **sv}
    if rank != 0:
        return
    from paper_2408_00930_gb300 import warpsci as W
    hbm, bf16_burst, bf16_sus, peak_src = load_peaks()
    n_chunks = main_res["n_chunks"]
    launch_ms = statistics.mean(main_res["chunk_ms"])
    launch_steps = min(CHUNK, wl["horizon"])
    flops_launch = flops_per_agent_step(wl) * (main_res["agent_steps"] / wl["horizon"]) * launch_steps
    bf16 = path == W.WS_PATH_BATCHED_BF16
    peak = bf16_sus if bf16 else bf16_sus / 4.0
    tensor = {"bound": "tensor", "achieved": flops_launch / (launch_ms * 1e-3) / 1e12,
              "peak": peak, "unit": "TFLOP/s", "frac": None,
              "peak_source": f"{peak_src} bf16 sustained" if bf16 else
              f"{peak_src} bf16 sustained / 4 (fp32 SIMT)"}
    tensor["frac"] = tensor["achieved"] / tensor["peak"]
    if bf16:
        # The fused kernels are bound by the SFU.  Its rates differ per
        # operation (ws_probe_rate, measured here before the timed region:
        # tanh, sin, lg2 ~16 results / clock / SM; ex2 ~32), so the work is
        # counted in tanh-equivalents: each operation weighted by
        # rate(tanh) / rate(op).  SFU operations per agent-step, from the
        # kernels' arithmetic (expf / logf each take one ex2 / lg2):
        #   control    H0 + H1 tanh; 2 ex2 and 1 lg2 (the two-way softmax)
        #   acrobot    H0 + H1 tanh; 3 ex2, 1 lg2; 22 sin / cos (the
        #              observation's two pairs, four RK4 stages of one pair and
        #              two sines, the terminal height's two cosines)
        #   economy    agent: H0 + H1 tanh, 20 ex2, 2 lg2 (log-probability and
        #              the wealth feature); planner: H0 + H1 tanh, 10 ex2, 1 lg2
        #   landscape  H0 + H1 tanh; M ex2 (one per Gaussian) + D ex2 (sigma);
        #              per coordinate half a Box-Muller pair (lg2, rsqrt, sin,
        #              cos) and one pair for the noise draw
        import torch
        n_sms = torch.cuda.get_device_properties(local).multi_processor_count
        clk = main_res["clocks"] or {}
        sm_mhz = clk.get("sm_mhz") or clk.get("sm_max_mhz") or 2070.0
        n_slots = main_res["agent_steps"] / wl["horizon"]
        H = sum(wl["h"])
        rates = main_res.get("sfu_rates") or {}
        r_t = rates.get("tanh.approx.f32", 16.0)
        w = {"tanh": 1.0, "ex2": r_t / rates.get("ex2.approx.ftz.f32", 16.0),
             "sin": r_t / rates.get("sin.approx.ftz.f32", 16.0),
             "lg2": r_t / rates.get("lg2.approx.ftz.f32", 16.0),
             "rsqrt": r_t / rates.get("rsqrt.approx.ftz.f32", 16.0)}

        def teq(**ops):
            return sum(n * w[k] for k, n in ops.items())
        lc = main_res.get("launch") or {}
        cc = wl["env"] in (0, 3) and lc.get("ctrl_envs_per_cta", 0)
        ctrl_kern = (f"ws_control_cc (CUDA cores, {lc.get('ctrl_envs_per_cta')} envs per CTA, "
                     f"{lc.get('ctrl_threads_per_env')} threads per env)" if cc else "ws_control_tc")
        if wl["env"] == 0:
            per_step = n_slots * teq(tanh=H, ex2=2, lg2=1)
            op, kern = "tanh (and the softmax's ex2, lg2) on the SFU", ctrl_kern
        elif wl["env"] == 3:
            per_step = n_slots * teq(tanh=H, ex2=3, lg2=1, sin=22)
            op, kern = "tanh, ex2, lg2, sin, cos on the SFU", ctrl_kern + " (acrobot)"
        elif wl["env"] == 1:
            n_pl = wl["n_envs"]
            per_step = ((n_slots - n_pl) * teq(tanh=H, ex2=20, lg2=2)
                        + n_pl * teq(tanh=H, ex2=10, lg2=1))
            op, kern = "tanh, ex2, lg2 on the SFU", "ws_econ_tc (work queue of env groups)"
        else:
            D = wl["dim"]
            per_step = n_slots * teq(tanh=H, ex2=wl["n_gauss"] + D, lg2=D / 2 + 1,
                                     rsqrt=D / 2 + 1, sin=D + 2)
            op, kern = "ex2 (energy), tanh and the normals' lg2 / rsqrt / sin / cos on the SFU", \
                "ws_land_tc (CTA-pair clusters)"
        sfu_launch = per_step * launch_steps
        src = ("measured by ws_probe_rate before the timed region" if rates else
               "nominal 16 / clock / SM for every SFU operation (probe unavailable)")
        roofline = {"bound": "alu", "op": op,
                    "achieved": sfu_launch / (launch_ms * 1e-3) / 1e12,
                    "peak": r_t * n_sms * sm_mhz * 1e6 / 1e12,
                    "unit": "T tanh-equivalent SFU results/s", "frac": None,
                    "traffic": None,
                    "kernel": kern + " (fused persistent, one launch per 50-step chunk)",
                    "peak_source": f"tanh.approx {r_t:.2f} results / clock / SM x {n_sms} SMs x "
                                   f"{sm_mhz:.0f} MHz (median sampled SM clock); rates {src}",
                    "sfu_rates_per_clk_per_sm": rates or None,
                    "tensor": {k: tensor[k] for k in ("achieved", "peak", "unit", "frac",
                                                      "peak_source")}}
        roofline["frac"] = roofline["achieved"] / roofline["peak"]
        if cc:
            # the CUDA-core kernel runs the policy GEMMs as FP32 FMAs: one per
            # multiply-add of the three layers, against the measured FMA rate
            r_f = rates.get("fma.rn.f32", 124.0) if rates else 124.0
            fma_launch = flops_per_agent_step(wl) / 2 * n_slots * launch_steps
            roofline["fma"] = {"achieved": fma_launch / (launch_ms * 1e-3) / 1e12,
                               "peak": r_f * n_sms * sm_mhz * 1e6 / 1e12, "unit": "T FMA/s",
                               "peak_source": f"fma.rn.f32 {r_f:.1f} / clock / SM x {n_sms} SMs x "
                                              f"{sm_mhz:.0f} MHz"}
            roofline["fma"]["frac"] = roofline["fma"]["achieved"] / roofline["fma"]["peak"]
            roofline.pop("tensor", None)
    else:
        roofline = dict(tensor, traffic=None, kernel="plain per-step kernels")
    if bf16 and not args.horizon and not args.n_envs:
        # DRAM bytes (read + write) of one 50-step launch of the fused kernel, from
        # the ncu captures summarised under profiles/ (*_ncu_full_*.md), beside the
        # algorithmic record bytes of the launch (control 29 B, economy 85 B,
        # landscape 205 B per agent-step)
        ncu_bytes = {"control_scale": (3.420672 + 135.461888) * 1e6,
                     "economy": 92.465664e6 + 1.185742e9,
                     "landscape": (1.850368 + 25.001216) * 1e6}
        rec_bytes = {0: 29.0, 1: 85.0, 2: 205.0, 3: 37.0}[wl["env"]]
        if args.workload in ncu_bytes:
            roofline["traffic"] = ncu_bytes[args.workload]
            roofline["traffic_algorithmic"] = (rec_bytes * main_res["agent_steps"] / wl["horizon"]
                                               * launch_steps)
    # S7 returns scan (k_returns, one launch per bench step over the whole
    # horizon): HBM-bound at 9 B per slot-step (reward and done read, return
    # written); its time is the gap between the roll-out's last event and the
    # step's end event, on the same stream
    ret_ms = statistics.mean(main_res["ret_ms"])
    ret_bytes = 9.0 * main_res["agent_steps"]
    returns_roofline = {"bound": "hbm", "kernel": "k_returns",
                        "achieved": ret_bytes / (ret_ms * 1e-3) / 1e9, "peak": hbm,
                        "unit": "GB/s", "frac": None, "ms": ret_ms,
                        "algorithmic_bytes": ret_bytes,
                        "traffic": RETURNS_NCU_BYTES_PER_SLOT_STEP * main_res["agent_steps"]
                        if RETURNS_NCU_BYTES_PER_SLOT_STEP and args.workload == "control_scale"
                        else None,
                        "peak_source": f"{peak_src} hbm_gbs"}
    returns_roofline["frac"] = returns_roofline["achieved"] / hbm
    force_roofline = None
    if main_res.get("force_ms"):
        import torch
        n_sms = torch.cuda.get_device_properties(local).multi_processor_count
        clk = (main_res["clocks"] or {}).get("sm_mhz") or 2070.0
        f_ms = statistics.median(main_res["force_ms"])
        pairs = wl["n_envs"] * min(CHUNK, wl["horizon"]) * wl["n_gauss"]
        if bf16:
            # k_force_tc: exponents and the force sums on tcgen05; the epilogue's
            # one ex2 per (row, Gaussian) pair on the SFU (measured rate) binds
            r_e = (main_res.get("sfu_rates") or {}).get("ex2.approx.ftz.f32", 16.0)
            force_roofline = {"bound": "alu", "kernel": "k_force_tc (ws_forces, 50 steps)",
                              "op": "ex2 on the SFU (one per env-Gaussian pair)",
                              "achieved": pairs / (f_ms * 1e-3) / 1e12,
                              "peak": r_e * n_sms * clk * 1e6 / 1e12, "unit": "Top/s"}
            src = f"ex2.approx {r_e:.2f} results / clock / SM x {n_sms} SMs x {clk:.0f} MHz"
        else:
            # k_force_f32 (FP32 SIMT, direct difference form): per pair D
            # subtractions, D FMAs for |y - c|^2 and D FMAs for the force sum on
            # the FP32 pipe (128 lanes / SM / clock), one exp
            force_roofline = {"bound": "alu", "kernel": "k_force_f32 (ws_forces, 50 steps)",
                              "op": "FP32 instructions (3 D per env-Gaussian pair)",
                              "achieved": 3 * wl["dim"] * pairs / (f_ms * 1e-3) / 1e12,
                              "peak": 128 * n_sms * clk * 1e6 / 1e12, "unit": "Tinst/s"}
            src = f"128 FP32 lanes / clock / SM x {n_sms} SMs x {clk:.0f} MHz"
        force_roofline.update(ms=f_ms, peak_source=src,
                              frac=force_roofline["achieved"] / force_roofline["peak"])
    lat = sorted(main_res["chunk_ms"])
    # kernels of ours per bench step: the reset (plus the landscape's energy of
    # the fresh state), per 50-step roll-out either the fused kernel and the
    # counter advance per launch chunk (BF16 paths) or the per-step kernels
    # and one advance per graph chunk (plain path), and the returns scan
    launch = main_res["launch"] or {}
    ch = int(launch.get("chunk_steps", CHUNK))
    lens = [min(CHUNK, wl["horizon"] - c * CHUNK) for c in range(n_chunks)]
    if bf16:
        per_roll = sum(-(-n // ch) * 2 for n in lens)
    else:
        per_step = {0: 6, 1: 14, 2: 9, 3: 6}[wl["env"]]
        per_roll = sum(per_step * n + -(-n // ch) for n in lens)
    per_launch = (3 if wl["env"] == 2 else 1) + per_roll + 1
    out = {
        "metric": METRIC, "value": value, "unit": "agent-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": main_res["total_ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16" if bf16 else "f32",
        "data": "synthetic",
        "config": {"workload": wl["desc"],
                   "path": "batched_bf16" if bf16 else "batched_fp32",
                   "bench_step": f"ws_reset + ws_rollout x {n_chunks} chunks of {CHUNK} + ws_returns",
                   "l2": "flushed between timed steps (256 MiB write)",
                   "launch": main_res["launch"],
                   "parallelism": f"{world} env shards (rank r: global env ids "
                                  f"[r n, (r + 1) n), n = {wl['n_envs']})" if world > 1
                                  else "single GPU"},
        "latency": {"chunk_steps": CHUNK, "p50_ms": float(np.percentile(lat, 50)),
                    "p99_ms": float(np.percentile(lat, 99))},
        # every timed step resets the envs under its own seed (1000 + warm-up
        # + step index): the spread of the step time over those seeds
        "seeds": {"reset_seeds": [1000 + args.warmup + i for i in range(args.steps)],
                  "ms_min": float(min(main_res["times"])),
                  "ms_median": float(statistics.median(main_res["times"])),
                  "ms_max": float(max(main_res["times"])),
                  "rel_spread": float((max(main_res["times"]) - min(main_res["times"]))
                                      / statistics.median(main_res["times"]))},
        "roofline": roofline,
        "roofline_returns": returns_roofline,
        "roofline_force": force_roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "plain_fp32": plain,
        "gpu_launches": per_launch * args.steps,
        "clocks": main_res["clocks"],
        "a2c_update": a2c,
        "serving": serving,
    }
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
