// ws_runtime.cu -- the C ABI (include/warpsci.h): context layout over the
// caller's buffers, parameter init, reset, step/rollout dispatch per path,
// CUDA-graph capture of the horizon loop, fetch/load, host-side waits.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "ws_kernels.cuh"

using namespace ws;

// A WS_FLAG_BOUNDS_CHECK canary: its byte offset in the state or ring buffer
// and the region it follows.
struct Canary {
  size_t off;
  const char *after;
};

struct ws_ctx {
  ws_config cfg;
  Layout L;
  Dev d;
  cudaStream_t stream = nullptr;    // caller's stream (borrowed)
  cudaStream_t capture = nullptr;   // private stream used only to capture graphs
  cudaEvent_t ev = nullptr;
  Branch br{nullptr, nullptr, nullptr};  // economy: planner branch
  char *state = nullptr;
  char *ring = nullptr;
  uint64_t k_host = 0;
  uint64_t ring_gen = 0;            // bumped whenever k moves (steps, reset, step load)
  uint64_t adv_gen = ~0ull;         // ring_gen when ws_advantages last ran
  uint32_t adv_n = 0;               // ... over this many last steps
  uint64_t seed = 0;
  std::vector<int32_t> agents;      // economy agent counts (host copy)
  std::map<uint32_t, cudaGraphExec_t> graphs;
  int tc_grid = 0;                  // fused control kernel: default persistent grid
  ws_launch lc{};                   // launch configuration (ws_get_launch / ws_tune)
  std::vector<int32_t> items;       // fused economy kernel: host copy of the work items
  std::vector<Canary> state_spots, ring_spots;  // WS_FLAG_BOUNDS_CHECK canaries
  ws_status err = WS_OK;
  std::string msg;
};

namespace {

constexpr size_t kAlign = 256;
constexpr size_t kCanary = 256;            // WS_FLAG_BOUNDS_CHECK canary after each region
constexpr unsigned char kCanaryByte = 0xA5;
inline size_t up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// The critic of WS_FLAG_TRAIN: the policy's widths with one output.
PolicyShape critic_shape(const PolicyShape &p) { return PolicyShape{{p.w[0], p.w[1], p.w[2], 1}}; }

ws_status fail(ws_ctx *c, ws_status s, const std::string &m) {
  if (c && c->err == WS_OK) {
    c->err = s;
    c->msg = m;
  }
  return s;
}

ws_status cuda_check(ws_ctx *c, cudaError_t e, const char *where) {
  if (e == cudaSuccess) return WS_OK;
  return fail(c, WS_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

ws_status validate(const ws_config *cfg) {
  if (!cfg || cfg->struct_size != sizeof(ws_config)) return WS_ERR_INVALID;
  if (cfg->env < WS_ENV_CONTROL || cfg->env > WS_ENV_ACROBOT) return WS_ERR_INVALID;
  if (cfg->path < WS_PATH_PLAIN_FP32 || cfg->path > WS_PATH_BATCHED_BF16) return WS_ERR_INVALID;
  if (cfg->n_envs < 1 || cfg->n_envs > (1u << 26)) return WS_ERR_INVALID;
  if ((uint64_t)cfg->env_base + cfg->n_envs > 0xFFFFFFFFull) return WS_ERR_INVALID;
  if (cfg->ring_steps < 1 || cfg->episode_limit < 1) return WS_ERR_INVALID;
  if (cfg->hidden0 < 1 || cfg->hidden0 > 4096 || cfg->hidden1 < 1 || cfg->hidden1 > 4096)
    return WS_ERR_INVALID;
  if (cfg->flags & ~(WS_FLAG_DEBUG_LOGITS | WS_FLAG_ENERGY_TARGET | WS_FLAG_FORCE | WS_FLAG_TRAIN |
                     WS_FLAG_BOUNDS_CHECK))
    return WS_ERR_INVALID;
  if ((cfg->flags & WS_FLAG_FORCE) && cfg->env != WS_ENV_LANDSCAPE) return WS_ERR_INVALID;
  if ((cfg->flags & WS_FLAG_ENERGY_TARGET) &&
      (cfg->env != WS_ENV_LANDSCAPE || !std::isfinite(cfg->energy_target)))
    return WS_ERR_INVALID;
  if (!(cfg->gamma >= 0.f && cfg->gamma <= 1.f)) return WS_ERR_INVALID;
  if (cfg->env == WS_ENV_LANDSCAPE) {
    if (cfg->dim < 1 || cfg->dim > 64 || cfg->n_gauss < 1 || cfg->n_gauss > (1u << 22))
      return WS_ERR_INVALID;
    if (!(cfg->step_clip > 0.f) || !(cfg->noise_sigma >= 0.f)) return WS_ERR_INVALID;
  }
  if (cfg->env == WS_ENV_ECONOMY && cfg->agents_per_env) {
    for (uint32_t e = 0; e < cfg->n_envs; ++e)
      if (cfg->agents_per_env[e] < 2 || cfg->agents_per_env[e] > 1024) return WS_ERR_INVALID;
  }
  return WS_OK;
}

// Agent counts U{8..256}: Philox(0, env, 0, ECON_INIT) word 0, multiply-shift.
void agent_counts(const ws_config *cfg, std::vector<int32_t> &out) {
  out.assign(cfg->n_envs, 1);
  if (cfg->env != WS_ENV_ECONOMY) return;
  for (uint32_t e = 0; e < cfg->n_envs; ++e) {
    if (cfg->agents_per_env) {
      out[e] = cfg->agents_per_env[e];
    } else {
      const uint4 r = draw(cfg->param_seed, 0, cfg->env_base + e, 0, kTagEconInit, 0);
      out[e] = 8 + (int32_t)bounded(r.x, 249u);
    }
  }
}

// The classic-control envs (control, acrobot) on BF16: the fused kernel of
// ws_control_tc.cu.
bool use_tc_control(const ws_config *cfg) {
  return (cfg->env == WS_ENV_CONTROL || cfg->env == WS_ENV_ACROBOT) &&
         cfg->path == WS_PATH_BATCHED_BF16;
}

// Economy / landscape on the BF16 path: per-layer tensor-core policy kernels.
bool use_tc_layers(const ws_config *cfg) {
  return !use_tc_control(cfg) && cfg->path == WS_PATH_BATCHED_BF16;
}

bool tc_layers_supported(const PolicyShape &p) {
  for (int l = 0; l < kMaxLayers; ++l)
    if (!dense_tc_supported(p.w[l], p.w[l + 1])) return false;
  return p.w[1] % 8 == 0 && p.w[2] % 8 == 0;
}

// The economy's policies fit the whole-MLP kernel (all three weight images in
// shared memory); the landscape's 256-wide layers run one layer per kernel.
bool use_mlp3(const ws_config *cfg, const PolicyShape &p, const PolicyShape &pp) {
  return use_tc_layers(cfg) && cfg->env == WS_ENV_ECONOMY && mlp3_tc_supported(p) &&
         mlp3_tc_supported(pp);
}

// Economy on the BF16 path: the fused persistent kernel when both policies
// have its shape (16-128-128-20 / -10) and every env fits one work item
// (at most three tiles of 128 agent rows).
constexpr int kEconMaxTiles = 3;
bool use_econ_fused(const ws_config *cfg, const PolicyShape &p, const PolicyShape &pp,
                    const std::vector<int32_t> &agents) {
  if (cfg->env != WS_ENV_ECONOMY || cfg->path != WS_PATH_BATCHED_BF16) return false;
  if (!econ_tc_supported(p, pp)) return false;
  for (int32_t a : agents)
    if (a > kEconMaxTiles * 128) return false;
  return true;
}

// Work items of the fused economy kernel: runs of consecutive envs with at most
// cap_rows agents and max_envs envs each, as {first agent slot, rows, first env,
// envs}; largest first when lpt (the queue then hands the long items out early).
std::vector<int32_t> econ_items(const std::vector<int32_t> &agents, int cap_rows, int max_envs,
                                bool lpt) {
  struct It { int32_t slot0, rows, env0, n; };
  std::vector<It> v;
  int32_t slot = 0;
  size_t e = 0;
  while (e < agents.size()) {
    It it{slot, 0, (int32_t)e, 0};
    while (e < agents.size() && it.n < max_envs && it.rows + agents[e] <= cap_rows) {
      it.rows += agents[e];
      slot += agents[e];
      ++it.n;
      ++e;
    }
    v.push_back(it);
  }
  if (lpt)
    std::stable_sort(v.begin(), v.end(), [](const It &a, const It &b) { return a.rows > b.rows; });
  std::vector<int32_t> out;
  out.reserve(v.size() * 4);
  for (const It &it : v) {
    out.push_back(it.slot0);
    out.push_back(it.rows);
    out.push_back(it.env0);
    out.push_back(it.n);
  }
  return out;
}

// Landscape on the BF16 path: the fused persistent kernel for the policy
// shapes it holds (D in {8, 16, 24}, D-256-256-2D); the per-step tensor-core
// kernels otherwise.  Resets still take the per-step energy kernel.
bool use_land_fused(const ws_config *cfg, const PolicyShape &p) {
  return cfg->env == WS_ENV_LANDSCAPE && cfg->path == WS_PATH_BATCHED_BF16 &&
         land_tc_supported((int)cfg->dim, (int)cfg->n_gauss, p) &&
         energy_tc_supported((int)cfg->dim, (int)cfg->n_gauss);
}

size_t tc_layers_bytes(const PolicyShape &p) {
  size_t n = 0;
  for (int l = 0; l < kMaxLayers; ++l) n += up(dense_tc_packed_bytes(p.w[l], p.w[l + 1]));
  return n;
}

Layout make_layout(const ws_config *cfg, const std::vector<int32_t> &agents,
                   std::vector<Canary> *state_spots = nullptr,
                   std::vector<Canary> *ring_spots = nullptr) {
  Layout L{};
  L.env = cfg->env;
  L.path = cfg->path;
  L.n_envs = cfg->n_envs;
  L.ring_steps = cfg->ring_steps;
  uint64_t sa = 0;
  for (int32_t a : agents) sa += (uint64_t)a;
  if (cfg->env == WS_ENV_ECONOMY) {
    L.n_agent_slots = (uint32_t)sa;
    L.n_slots = (uint32_t)sa + cfg->n_envs;
    L.obs_dim = kEconF;
    L.act_dim = 1;
    L.n_out = 20;
    L.n_out_planner = 10;
    L.pol = PolicyShape{{kEconF, (int)cfg->hidden0, (int)cfg->hidden1, 20}};
    L.pol_planner = PolicyShape{{kEconF, (int)cfg->hidden0, (int)cfg->hidden1, 10}};
  } else if (cfg->env == WS_ENV_CONTROL) {
    L.n_agent_slots = cfg->n_envs;
    L.n_slots = cfg->n_envs;
    L.obs_dim = 4;
    L.act_dim = 1;
    L.n_out = 2;
    L.pol = PolicyShape{{4, (int)cfg->hidden0, (int)cfg->hidden1, 2}};
    L.pol_planner = PolicyShape{{0, 0, 0, 0}};
  } else if (cfg->env == WS_ENV_ACROBOT) {
    L.n_agent_slots = cfg->n_envs;
    L.n_slots = cfg->n_envs;
    L.obs_dim = kAcroObs;
    L.act_dim = 1;
    L.n_out = 3;
    L.pol = PolicyShape{{kAcroObs, (int)cfg->hidden0, (int)cfg->hidden1, 3}};
    L.pol_planner = PolicyShape{{0, 0, 0, 0}};
  } else {
    L.n_agent_slots = cfg->n_envs;
    L.n_slots = cfg->n_envs;
    L.obs_dim = cfg->dim;
    L.act_dim = cfg->dim;
    L.n_out = 2 * cfg->dim;
    L.pol = PolicyShape{{(int)cfg->dim, (int)cfg->hidden0, (int)cfg->hidden1, (int)(2 * cfg->dim)}};
    L.pol_planner = PolicyShape{{0, 0, 0, 0}};
  }
  const size_t N = cfg->n_envs, S = L.n_slots, Sa = L.n_agent_slots, M = cfg->n_gauss,
               D = cfg->dim, R = cfg->ring_steps;
  // Regions are carved in order, each 256-byte aligned.  With
  // WS_FLAG_BOUNDS_CHECK each one is followed right at its end by a 256-byte
  // canary (recorded with the region's name), so that a kernel writing past one
  // field hits the canary before the next field.
  const bool check = (cfg->flags & WS_FLAG_BOUNDS_CHECK) != 0;
  auto carve = [&](size_t &o, size_t bytes, const char *name, std::vector<Canary> *spots) {
    const size_t at = o;
    o = at + bytes;
    if (check && bytes) {
      if (spots) spots->push_back(Canary{o, name});
      o += kCanary;
    }
    o = up(o);
    return at;
  };
  auto st = [&](size_t &o, size_t bytes, const char *name) { return carve(o, bytes, name, state_spots); };
  auto rg = [&](size_t &o, size_t bytes, const char *name) { return carve(o, bytes, name, ring_spots); };
  size_t o = 0;
  L.k_off = st(o, 8, "step counter");
  L.err_off = st(o, 8, "error flag");
  L.params_off = st(o, L.pol.count() * 4, "PARAMS");
  L.params_planner_off =
      st(o, cfg->env == WS_ENV_ECONOMY ? L.pol_planner.count() * 4 : 0, "planner PARAMS");
  L.econ_fused = use_econ_fused(cfg, L.pol, L.pol_planner, agents) ? 1 : 0;
  L.packed_bytes = use_tc_control(cfg) ? control_tc_packed_bytes(L.pol) : 0;
  if (use_tc_layers(cfg))
    L.packed_bytes = tc_layers_bytes(L.pol) +
                     (cfg->env == WS_ENV_ECONOMY ? tc_layers_bytes(L.pol_planner) : 0);
  if (use_mlp3(cfg, L.pol, L.pol_planner))
    L.packed_bytes = up(mlp3_tc_packed_bytes(L.pol)) + up(mlp3_tc_packed_bytes(L.pol_planner));
  if (L.econ_fused) L.packed_bytes = econ_tc_packed_bytes();
  L.land_fused = use_land_fused(cfg, L.pol) ? 1 : 0;
  if (L.land_fused) L.packed_bytes = land_tc_policy_bytes();
  L.packed_off = st(o, L.packed_bytes, "BF16 operand images");
  size_t env_params = 0;
  if (cfg->env == WS_ENV_LANDSCAPE) env_params = up(M * D * 4) + up(M * 4) + up(M * 4);
  if (cfg->env == WS_ENV_ECONOMY) env_params = up(N * 4);
  L.env_params_off = st(o, env_params, "ENV_PARAMS");
  // landscape tables: |c|^2 and the exponent coefficients, the BF16 centre
  // image, the fused kernel's energy image and its force image
  L.env_derived_bytes = cfg->env == WS_ENV_LANDSCAPE ? up(M * 4) + up(M * 4) : 0;
  if (cfg->env == WS_ENV_LANDSCAPE && cfg->path == WS_PATH_BATCHED_BF16)
    L.env_derived_bytes += up(energy_tc_bytes((int)D, (int)M));
  const size_t land_energy_rel = L.env_derived_bytes;
  if (L.land_fused) L.env_derived_bytes += up(land_tc_energy_bytes((int)M));
  const size_t force_img_rel = L.env_derived_bytes;
  if (L.land_fused && (cfg->flags & WS_FLAG_FORCE)) L.env_derived_bytes += up(force_tc_bytes((int)M));
  L.env_derived_off = st(o, L.env_derived_bytes, "landscape tables");
  L.land_energy_off = L.env_derived_off + land_energy_rel;
  L.force_img_off = L.env_derived_off + force_img_rel;
  size_t state = 0;
  if (cfg->env == WS_ENV_CONTROL || cfg->env == WS_ENV_ACROBOT) state = up(4 * N * 4);
  if (cfg->env == WS_ENV_ECONOMY) state = up(Sa * 8) + up(kEconF * Sa * 4);
  if (cfg->env == WS_ENV_LANDSCAPE) state = up(D * N * 4) + up(N * 4) + up(N);
  L.state_off = st(o, state, "STATE");
  L.t_off = st(o, N * 4, "episode counters");
  L.aux_off = st(o, cfg->env == WS_ENV_ECONOMY ? up((N + 1) * 4) + up(Sa * 4) : 0,
                 "agent offsets");
  L.items_off = st(o, L.econ_fused ? N * 16 : 0, "work items");
  L.queue_off = st(o, L.econ_fused ? 8 : 0, "work queue");
  L.scratch_off = o;
  const bool plain_scratch = !use_tc_control(cfg) && !L.econ_fused;
  if (L.econ_fused && (cfg->flags & WS_FLAG_DEBUG_LOGITS)) {
    L.scratch_out_off = st(o, Sa * L.n_out * 4, "LOGITS");
    L.scratch_pout_off = st(o, N * 10 * 4, "planner LOGITS");
  }
  if (plain_scratch) {
    L.scratch_h0_off = st(o, S * cfg->hidden0 * 4, "hidden 0");
    L.scratch_h1_off = st(o, S * cfg->hidden1 * 4, "hidden 1");
    L.scratch_out_off = st(o, S * L.n_out * 4, "LOGITS");
    if (cfg->env == WS_ENV_ECONOMY) {
      L.scratch_pobs_off = st(o, N * kEconF * 4, "planner observation");
      L.scratch_ph0_off = st(o, N * cfg->hidden0 * 4, "planner hidden 0");
      L.scratch_ph1_off = st(o, N * cfg->hidden1 * 4, "planner hidden 1");
      L.scratch_pout_off = st(o, N * 10 * 4, "planner LOGITS");
      L.scratch_income_off = st(o, Sa * 8, "income");
    }
    if (cfg->env == WS_ENV_LANDSCAPE)  // energy partials
      L.scratch_income_off = st(o, (size_t)kEnergyChunks * 2 * N * 4, "energy partials");
    if (cfg->env == WS_ENV_ACROBOT)    // the policy's input
      L.scratch_pobs_off = st(o, (size_t)kAcroObs * N * 4, "acrobot observation");
  }
  L.critic_off = L.train_off = o;
  if (cfg->flags & WS_FLAG_TRAIN) {
    // critics: the policy's (agents'), then the planner's
    size_t cb = up(critic_shape(L.pol).count() * 4);
    if (cfg->env == WS_ENV_ECONOMY) cb += up(critic_shape(L.pol_planner).count() * 4);
    L.critic_off = st(o, cb, "CRITIC");
    L.train_off = st(o, train_scratch_bytes(L.pol), "update scratch");
  }
  L.state_bytes = o;
  size_t r = 0;
  L.ring_obs = rg(r, R * L.obs_dim * S * 4, "OBS");
  L.ring_act = rg(r, R * L.act_dim * S * 4, "ACTION");
  L.ring_logp = rg(r, R * S * 4, "LOGP");
  L.ring_rew = rg(r, R * S * 4, "REWARD");
  L.ring_done = rg(r, R * S, "DONE");
  L.ring_ret = rg(r, R * S * 4, "RETURN");
  L.ring_wealth = rg(r, cfg->env == WS_ENV_ECONOMY ? R * S * 8 : 0, "WEALTH");
  L.ring_energy = rg(r, cfg->env == WS_ENV_LANDSCAPE ? R * S * 4 : 0, "ENERGY");
  L.ring_force = rg(r, cfg->env == WS_ENV_LANDSCAPE && (cfg->flags & WS_FLAG_FORCE)
                           ? R * (size_t)cfg->dim * S * 4 : 0, "FORCE");
  L.ring_adv = rg(r, (cfg->flags & WS_FLAG_TRAIN) ? R * S * 4 : 0, "ADVANTAGE");
  L.ring_sample = rg(r, cfg->env == WS_ENV_LANDSCAPE && (cfg->flags & WS_FLAG_TRAIN)
                            ? R * (size_t)cfg->dim * S * 4 : 0, "SAMPLE");
  L.ring_pout = rg(r, (cfg->flags & WS_FLAG_DEBUG_LOGITS) ? R * (size_t)L.n_out * S * 4 : 0,
                   "POLICY_OUT");
  L.ring_bytes = r;
  return L;
}

void make_dev(ws_ctx *c) {
  const Layout &L = c->L;
  const ws_config &cfg = c->cfg;
  Dev &d = c->d;
  std::memset(&d, 0, sizeof(d));
  char *S = c->state, *R = c->ring;
  d.env = cfg.env;
  d.n_envs = L.n_envs;
  d.n_slots = L.n_slots;
  d.n_agent_slots = L.n_agent_slots;
  d.ring_steps = L.ring_steps;
  d.episode_limit = cfg.episode_limit;
  d.dim = cfg.dim;
  d.n_gauss = cfg.n_gauss;
  d.n_out = L.n_out;
  d.n_out_planner = L.n_out_planner;
  d.noise_sigma = cfg.noise_sigma;
  d.energy_target = (cfg.flags & WS_FLAG_ENERGY_TARGET) ? cfg.energy_target : -INFINITY;
  d.step_clip = cfg.step_clip;
  d.gamma = cfg.gamma;
  d.seed = c->seed;
  d.env_base = cfg.env_base;
  d.k = (uint64_t *)(S + L.k_off);
  d.err = (uint32_t *)(S + L.err_off);
  d.params = (const float *)(S + L.params_off);
  d.params_planner = (const float *)(S + L.params_planner_off);
  d.pol = L.pol;
  d.pol_planner = L.pol_planner;
  const size_t N = L.n_envs, Sa = L.n_agent_slots, M = cfg.n_gauss, D = cfg.dim;
  if (cfg.env == WS_ENV_LANDSCAPE) {
    d.centres = (float *)(S + L.env_params_off);
    d.widths = (float *)(S + L.env_params_off + up(M * D * 4));
    d.amps = (float *)(S + L.env_params_off + up(M * D * 4) + up(M * 4));
    d.cnorm = (float *)(S + L.env_derived_off);
    d.coef = (float *)(S + L.env_derived_off + up(M * 4));
    if (cfg.path == WS_PATH_BATCHED_BF16)
      d.eimg = (const uint8_t *)(S + L.env_derived_off + up(M * 4) + up(M * 4));
    d.s = (float *)(S + L.state_off);
    d.eobs = (float *)(S + L.state_off + up(D * N * 4));
    d.needs_energy = (uint8_t *)(S + L.state_off + up(D * N * 4) + up(N * 4));
  } else if (cfg.env == WS_ENV_CONTROL) {
    d.s = (float *)(S + L.state_off);
  } else if (cfg.env == WS_ENV_ACROBOT) {
    d.s = (float *)(S + L.state_off);
    if (!use_tc_control(&cfg)) d.pobs = (float *)(S + L.scratch_pobs_off);
  } else {
    d.wealth = (int64_t *)(S + L.state_off);
    d.feat = (float *)(S + L.state_off + up(Sa * 8));
    d.agent_off = (const int32_t *)(S + L.aux_off);
    d.slot_env = (const int32_t *)(S + L.aux_off + up((N + 1) * 4));
  }
  d.t = (int32_t *)(S + L.t_off);
  if (L.econ_fused) {
    d.items = (const int32_t *)(S + L.items_off);
    d.queue = (uint32_t *)(S + L.queue_off);
    d.n_items = (uint32_t)(c->items.size() / 4);
    d.dbg_logits = (cfg.flags & WS_FLAG_DEBUG_LOGITS) ? 1 : 0;
    if (d.dbg_logits) {
      d.out = (float *)(S + L.scratch_out_off);
      d.pout = (float *)(S + L.scratch_pout_off);
    }
  } else if (L.land_fused) {
    d.dbg_logits = (cfg.flags & WS_FLAG_DEBUG_LOGITS) ? 1 : 0;
    d.limg = (const uint8_t *)(S + L.land_energy_off);
    if (cfg.flags & WS_FLAG_FORCE) d.fimg = (const uint8_t *)(S + L.force_img_off);
  } else if (use_mlp3(&cfg, L.pol, L.pol_planner)) {
    d.tc_mlp = 1;
    d.mlp3 = 1;
    d.pk[0][0] = (const uint8_t *)(S + L.packed_off);
    d.pk[1][0] = (const uint8_t *)(S + L.packed_off + up(mlp3_tc_packed_bytes(L.pol)));
  } else if (use_tc_layers(&cfg)) {
    d.tc_mlp = 1;
    size_t o = L.packed_off;
    for (int pid = 0; pid < (cfg.env == WS_ENV_ECONOMY ? 2 : 1); ++pid) {
      const PolicyShape &p = pid ? L.pol_planner : L.pol;
      for (int l = 0; l < kMaxLayers; ++l) {
        d.pk[pid][l] = (const uint8_t *)(S + o);
        o += up(dense_tc_packed_bytes(p.w[l], p.w[l + 1]));
      }
    }
  }
  if (!use_tc_control(&cfg) && !L.econ_fused) {
    d.h0 = (float *)(S + L.scratch_h0_off);
    d.h1 = (float *)(S + L.scratch_h1_off);
    d.out = (float *)(S + L.scratch_out_off);
    if (cfg.env == WS_ENV_ECONOMY) {
      d.pobs = (float *)(S + L.scratch_pobs_off);
      d.ph0 = (float *)(S + L.scratch_ph0_off);
      d.ph1 = (float *)(S + L.scratch_ph1_off);
      d.pout = (float *)(S + L.scratch_pout_off);
      d.income = (int64_t *)(S + L.scratch_income_off);
    }
    if (cfg.env == WS_ENV_LANDSCAPE) d.epart = (float *)(S + L.scratch_income_off);
  }
  d.r_obs = (float *)(R + L.ring_obs);
  d.r_act = (void *)(R + L.ring_act);
  d.r_logp = (float *)(R + L.ring_logp);
  d.r_rew = (float *)(R + L.ring_rew);
  d.r_done = (uint8_t *)(R + L.ring_done);
  d.r_ret = (float *)(R + L.ring_ret);
  d.r_wealth = cfg.env == WS_ENV_ECONOMY ? (int64_t *)(R + L.ring_wealth) : nullptr;
  d.r_energy = cfg.env == WS_ENV_LANDSCAPE ? (float *)(R + L.ring_energy) : nullptr;
  d.r_force = (cfg.flags & WS_FLAG_FORCE) ? (float *)(R + L.ring_force) : nullptr;
  d.r_adv = (cfg.flags & WS_FLAG_TRAIN) ? (float *)(R + L.ring_adv) : nullptr;
  d.r_sample = (cfg.env == WS_ENV_LANDSCAPE && (cfg.flags & WS_FLAG_TRAIN))
                   ? (float *)(R + L.ring_sample)
                   : nullptr;
  d.r_pout = (cfg.flags & WS_FLAG_DEBUG_LOGITS) ? (float *)(R + L.ring_pout) : nullptr;
}

void drop_graphs(ws_ctx *c) {
  for (auto &kv : c->graphs) cudaGraphExecDestroy(kv.second);
  c->graphs.clear();
}

// Paths whose chunks run as one persistent kernel launch each.
bool fused(const ws_ctx *c) { return use_tc_control(&c->cfg) || c->L.econ_fused || c->L.land_fused; }

uint32_t chunk_of(const ws_ctx *c) { return c->lc.chunk_steps; }

int sm_count() {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

int max_agents(const ws_ctx *c) {
  int m = 1;
  for (int32_t a : c->agents) m = a > m ? a : m;
  return m;
}

// Defaults of a fresh context.
void default_launch(ws_ctx *c) {
  ws_launch &l = c->lc;
  l = ws_launch{};
  l.struct_size = sizeof(ws_launch);
  l.chunk_steps = c->cfg.chunk_steps ? c->cfg.chunk_steps : (fused(c) ? 100u : 25u);
  l.grid = 0;
  l.econ_tiles = 3;
  l.econ_lpt = 1;
  l.energy_chunks = 2;
  l.env_threads = 256;
  // fused landscape: a CTA pair per tile while the pairs fit the SMs at once
  const uint32_t tiles = (c->L.n_envs + 127) / 128;
  l.tile_ctas = 2 * tiles <= (uint32_t)sm_count() ? 2u : 1u;
  l.ctrl_envs_per_cta = 0;  // the tensor-core kernel
  l.ctrl_threads_per_env = 8;
}

// The fused kernels' device-wait limit of a launch configuration (0 = 2 s).
uint64_t device_wait_ns(const ws_launch &l) { return l.wait_ns ? l.wait_ns : 2000000000ull; }

int econ_grid(const ws_ctx *c) {
  const int sms = sm_count();
  const int n = (int)c->d.n_items;
  return n < sms ? n : sms;
}

// (Re)build the fused economy kernel's work items for the context's tile count
// and upload them (stream-ordered; the host copy lives in the context).
ws_status set_econ_items(ws_ctx *c) {
  c->items = econ_items(c->agents, (int)c->lc.econ_tiles * 128, econ_tc_max_envs_per_item(),
                        c->lc.econ_lpt != 0);
  c->d.n_items = (uint32_t)(c->items.size() / 4);
  cudaError_t e = cudaMemcpyAsync((void *)c->d.items, c->items.data(), c->items.size() * 4,
                                  cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d.queue, 0, 8, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return cuda_check(c, e, "upload work items");
}

// Enqueue `n` steps on stream st (used directly and under capture).
ws_status enqueue_steps(ws_ctx *c, uint32_t n, cudaStream_t st) {
  if (use_tc_control(&c->cfg)) {
    const uint32_t chunk = chunk_of(c);
    for (uint32_t done = 0; done < n;) {
      const uint32_t m = (n - done) < chunk ? (n - done) : chunk;
      cudaError_t e;
      if (c->lc.ctrl_envs_per_cta) {
        e = launch_control_cc(c->d, m, (int)c->lc.ctrl_envs_per_cta,
                              (int)c->lc.ctrl_threads_per_env, st);
      } else {
        const int grid = c->lc.grid ? (int)c->lc.grid : c->tc_grid;
        e = launch_control_tc(c->d, c->state + c->L.packed_off, m, grid, st);
      }
      if (e != cudaSuccess) return cuda_check(c, e, "control kernel launch");
      launch_advance(c->d, m, st);
      done += m;
    }
  } else if (c->L.land_fused) {
    const uint32_t chunk = chunk_of(c);
    for (uint32_t done = 0; done < n;) {
      const uint32_t m = (n - done) < chunk ? (n - done) : chunk;
      cudaError_t e = launch_land_tc(c->d, c->state + c->L.packed_off, c->state + c->L.land_energy_off,
                                     m, (int)c->lc.tile_ctas, st);
      if (e != cudaSuccess) return cuda_check(c, e, "land_tc launch");
      launch_advance(c->d, m, st);
      done += m;
    }
  } else if (c->L.econ_fused) {
    const uint32_t chunk = chunk_of(c);
    const int grid = econ_grid(c);
    for (uint32_t done = 0; done < n;) {
      const uint32_t m = (n - done) < chunk ? (n - done) : chunk;
      cudaError_t e =
          launch_econ_tc(c->d, c->state + c->L.packed_off, m, (int)c->lc.econ_tiles, grid, st);
      if (e != cudaSuccess) return cuda_check(c, e, "econ_tc launch");
      launch_advance(c->d, m, st);
      done += m;
    }
  } else {
    const Branch *br = c->br.aux ? &c->br : nullptr;
    for (uint32_t i = 0; i < n; ++i) launch_plain_step(c->d, i, st, br);
    launch_advance(c->d, n, st);
  }
  return cuda_check(c, cudaGetLastError(), "step launch");
}

ws_status graph_for(ws_ctx *c, uint32_t n, cudaGraphExec_t *out) {
  auto it = c->graphs.find(n);
  if (it != c->graphs.end()) {
    *out = it->second;
    return WS_OK;
  }
  cudaError_t e = cudaStreamBeginCapture(c->capture, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_check(c, e, "begin capture");
  ws_status s = enqueue_steps(c, n, c->capture);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(c->capture, &g);
  if (s != WS_OK) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  if (e != cudaSuccess) return cuda_check(c, e, "end capture");
  cudaGraphExec_t ex = nullptr;
  e = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_check(c, e, "graph instantiate");
  c->graphs[n] = ex;
  *out = ex;
  return WS_OK;
}

size_t ring_field_step_bytes(const ws_ctx *c, ws_field f, size_t *field_off) {
  const Layout &L = c->L;
  const size_t S = L.n_slots;
  switch (f) {
    case WS_F_OBS: *field_off = L.ring_obs; return (size_t)L.obs_dim * S * 4;
    case WS_F_ACTION: *field_off = L.ring_act; return (size_t)L.act_dim * S * 4;
    case WS_F_LOGP: *field_off = L.ring_logp; return S * 4;
    case WS_F_REWARD: *field_off = L.ring_rew; return S * 4;
    case WS_F_DONE: *field_off = L.ring_done; return S;
    case WS_F_RETURN: *field_off = L.ring_ret; return S * 4;
    case WS_F_WEALTH:
      if (L.env != WS_ENV_ECONOMY) return 0;
      *field_off = L.ring_wealth; return S * 8;
    case WS_F_ENERGY:
      if (L.env != WS_ENV_LANDSCAPE) return 0;
      *field_off = L.ring_energy; return S * 4;
    case WS_F_FORCE:
      if (!(c->cfg.flags & WS_FLAG_FORCE)) return 0;
      *field_off = L.ring_force; return (size_t)c->cfg.dim * S * 4;
    case WS_F_ADVANTAGE:
      if (!(c->cfg.flags & WS_FLAG_TRAIN)) return 0;
      *field_off = L.ring_adv; return S * 4;
    case WS_F_SAMPLE:
      if (L.env != WS_ENV_LANDSCAPE || !(c->cfg.flags & WS_FLAG_TRAIN)) return 0;
      *field_off = L.ring_sample; return (size_t)c->cfg.dim * S * 4;
    case WS_F_POLICY_OUT:
      if (!(c->cfg.flags & WS_FLAG_DEBUG_LOGITS)) return 0;
      *field_off = L.ring_pout; return (size_t)L.n_out * S * 4;
    default: return 0;
  }
}

// (device pointer, bytes) pieces of a state-like field, in ABI order.
struct Piece { char *p; size_t n; };
std::vector<Piece> state_pieces(ws_ctx *c, ws_field f) {
  const Layout &L = c->L;
  const size_t N = L.n_envs, Sa = L.n_agent_slots, D = c->cfg.dim, M = c->cfg.n_gauss;
  char *S = c->state;
  std::vector<Piece> v;
  if (f == WS_F_STATE) {
    if (L.env == WS_ENV_CONTROL || L.env == WS_ENV_ACROBOT) {
      v.push_back({S + L.state_off, 4 * N * 4});
    } else if (L.env == WS_ENV_ECONOMY) {
      v.push_back({S + L.state_off, Sa * 8});
      v.push_back({S + L.state_off + up(Sa * 8), kEconF * Sa * 4});
    } else {
      v.push_back({S + L.state_off, D * N * 4});
      v.push_back({S + L.state_off + up(D * N * 4), N * 4});
    }
    v.push_back({S + L.t_off, N * 4});
  } else if (f == WS_F_CRITIC) {
    if (c->cfg.flags & WS_FLAG_TRAIN) {
      v.push_back({S + L.critic_off, critic_shape(L.pol).count() * 4});
      if (L.env == WS_ENV_ECONOMY)
        v.push_back({S + L.critic_off + up(critic_shape(L.pol).count() * 4),
                     critic_shape(L.pol_planner).count() * 4});
    }
  } else if (f == WS_F_PARAMS) {
    v.push_back({S + L.params_off, L.pol.count() * 4});
    if (L.env == WS_ENV_ECONOMY) v.push_back({S + L.params_planner_off, L.pol_planner.count() * 4});
  } else if (f == WS_F_ENV_PARAMS) {
    if (L.env == WS_ENV_LANDSCAPE) {
      v.push_back({S + L.env_params_off, M * D * 4});
      v.push_back({S + L.env_params_off + up(M * D * 4), M * 4});
      v.push_back({S + L.env_params_off + up(M * D * 4) + up(M * 4), M * 4});
    } else if (L.env == WS_ENV_ECONOMY) {
      v.push_back({S + L.env_params_off, N * 4});
    }
  } else if (f == WS_F_LOGITS) {
    if (use_tc_control(&c->cfg)) return v;
    if ((L.econ_fused || L.land_fused) && !c->d.dbg_logits) return v;
    v.push_back({S + L.scratch_out_off, (size_t)L.n_agent_slots * L.n_out * 4});
    if (L.env == WS_ENV_ECONOMY) v.push_back({S + L.scratch_pout_off, N * 10 * 4});
  }
  return v;
}

ws_status after_params_changed(ws_ctx *c) {
  if (c->cfg.env == WS_ENV_LANDSCAPE) launch_landscape_derive(c->d, c->stream);
  if (c->d.eimg) launch_energy_tc_pack(c->d, (void *)c->d.eimg, c->stream);
  if (use_tc_control(&c->cfg)) launch_control_tc_pack(c->d, c->state + c->L.packed_off, c->stream);
  if (c->L.econ_fused) {
    launch_econ_tc_pack(c->d.params, c->d.params_planner, c->state + c->L.packed_off, c->stream);
  } else if (c->L.land_fused) {
    launch_land_tc_pack(c->d, c->state + c->L.packed_off, c->state + c->L.land_energy_off, c->stream);
    if (c->d.fimg) launch_force_tc_pack(c->d, c->d.limg, (void *)c->d.fimg, c->stream);
  } else if (c->d.mlp3) {
    launch_mlp3_tc_pack(c->d.params, c->L.pol, (void *)c->d.pk[0][0], c->stream);
    launch_mlp3_tc_pack(c->d.params_planner, c->L.pol_planner, (void *)c->d.pk[1][0], c->stream);
  } else if (use_tc_layers(&c->cfg)) {
    for (int pid = 0; pid < (c->cfg.env == WS_ENV_ECONOMY ? 2 : 1); ++pid) {
      const PolicyShape &p = pid ? c->L.pol_planner : c->L.pol;
      const float *par = pid ? c->d.params_planner : c->d.params;
      for (int l = 0; l < kMaxLayers; ++l) {
        const float *W = par + p.layer_offset(l);
        launch_dense_tc_pack(W, W + (size_t)p.w[l] * p.w[l + 1], p.w[l], p.w[l + 1],
                             (void *)c->d.pk[pid][l], c->stream);
      }
    }
  }
  return cuda_check(c, cudaGetLastError(), "param derive");
}

// The update's policy / critic pairs: one over every slot, or the economy's
// agents on slots [0, Sa) and planners on [Sa, S).
int train_groups(const ws_ctx *c, TrainGroup (&g)[2]) {
  const Layout &L = c->L;
  float *crit0 = (float *)(c->state + L.critic_off);
  g[0] = TrainGroup{(float *)c->d.params, crit0, L.pol, critic_shape(L.pol), 0u, L.n_agent_slots};
  if (L.env != WS_ENV_ECONOMY) return 1;
  g[1] = TrainGroup{(float *)c->d.params_planner,
                    (float *)(c->state + L.critic_off + up(critic_shape(L.pol).count() * 4)),
                    L.pol_planner, critic_shape(L.pol_planner), L.n_agent_slots, L.n_envs};
  return 2;
}

// After an update: repack the BF16 images, then (stats != NULL) wait and
// return the loss sums as means over the n x n_slots rows.
ws_status finish_update(ws_ctx *c, const TrainBufs &tb, uint32_t n, double *stats, int n_stats,
                        const char *what) {
  ws_status s = cuda_check(c, cudaGetLastError(), what);
  if (s == WS_OK) s = after_params_changed(c);
  if (s == WS_OK && stats) {
    double h[4];
    s = cuda_check(c, cudaMemcpyAsync(h, tb.stats, 8 * n_stats, cudaMemcpyDeviceToHost, c->stream),
                   "update stats");
    if (s == WS_OK) s = cuda_check(c, cudaStreamSynchronize(c->stream), "update stats sync");
    const double R = (double)n * c->L.n_slots;
    if (s == WS_OK)
      for (int i = 0; i < n_stats; ++i) stats[i] = h[i] / R;
  }
  return s;
}

}  // namespace

extern "C" {

ws_status ws_query_bytes(const ws_config *cfg, size_t *state_bytes, size_t *ring_bytes,
                         uint32_t *n_slots) {
  ws_status s = validate(cfg);
  if (s != WS_OK) return s;
  if (use_tc_control(cfg) && !control_tc_supported(PolicyShape{{4, (int)cfg->hidden0, (int)cfg->hidden1, 2}}))
    return WS_ERR_UNSUPPORTED;
  std::vector<int32_t> agents;
  agent_counts(cfg, agents);
  const Layout L = make_layout(cfg, agents);
  if (use_tc_layers(cfg) &&
      !(tc_layers_supported(L.pol) && (cfg->env != WS_ENV_ECONOMY || tc_layers_supported(L.pol_planner))))
    return WS_ERR_UNSUPPORTED;
  if (use_tc_layers(cfg) && cfg->env == WS_ENV_LANDSCAPE &&
      !energy_tc_supported((int)cfg->dim, (int)cfg->n_gauss))
    return WS_ERR_UNSUPPORTED;
  if (state_bytes) *state_bytes = L.state_bytes;
  if (ring_bytes) *ring_bytes = L.ring_bytes;
  if (n_slots) *n_slots = L.n_slots;
  return WS_OK;
}

ws_status ws_create(const ws_config *cfg, void *state_buf, size_t state_bytes, void *ring_buf,
                    size_t ring_bytes, void *cuda_stream, ws_ctx **out) {
  if (!out) return WS_ERR_INVALID;
  *out = nullptr;
  size_t need_s = 0, need_r = 0;
  ws_status s = ws_query_bytes(cfg, &need_s, &need_r, nullptr);
  if (s != WS_OK) return s;
  if (!state_buf || !ring_buf) return WS_ERR_INVALID;
  if (((uintptr_t)state_buf | (uintptr_t)ring_buf) % kAlign) return WS_ERR_INVALID;
  if (state_bytes < need_s || ring_bytes < need_r) return WS_ERR_NOMEM;
  ws_ctx *c = new ws_ctx();
  c->cfg = *cfg;
  c->cfg.agents_per_env = nullptr;  // host array is copied, never kept
  agent_counts(cfg, c->agents);
  c->L = make_layout(cfg, c->agents, &c->state_spots, &c->ring_spots);
  c->stream = (cudaStream_t)cuda_stream;
  c->state = (char *)state_buf;
  c->ring = (char *)ring_buf;
  c->seed = cfg->param_seed;
  make_dev(c);
  default_launch(c);
  c->d.env_threads = (int)c->lc.env_threads;
  c->d.update_simt = (int)c->lc.update_gemm;
  c->d.energy_chunks = (int)c->lc.energy_chunks;
  c->d.wait_ns = device_wait_ns(c->lc);
  cudaError_t e = cudaStreamCreateWithFlags(&c->capture, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev, cudaEventDisableTiming);
  if (e == cudaSuccess && cfg->env == WS_ENV_ECONOMY) {
    e = cudaStreamCreateWithFlags(&c->br.aux, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->br.fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->br.join, cudaEventDisableTiming);
  }
  for (const Canary &k : c->state_spots)
    if (e == cudaSuccess) e = cudaMemsetAsync(c->state + k.off, kCanaryByte, kCanary, c->stream);
  for (const Canary &k : c->ring_spots)
    if (e == cudaSuccess) e = cudaMemsetAsync(c->ring + k.off, kCanaryByte, kCanary, c->stream);
  if (e != cudaSuccess) {
    cuda_check(c, e, "stream/event create");
    ws_status r = c->err;
    ws_destroy(c);
    return r;
  }
  cudaMemsetAsync(c->d.err, 0, 8, c->stream);
  if (cfg->env == WS_ENV_ECONOMY) {
    const size_t N = c->L.n_envs, Sa = c->L.n_agent_slots;
    std::vector<int32_t> off(N + 1, 0), slot_env(Sa, 0);
    for (size_t i = 0; i < N; ++i) {
      off[i + 1] = off[i] + c->agents[i];
      for (int32_t a = 0; a < c->agents[i]; ++a) slot_env[off[i] + a] = (int32_t)i;
    }
    cudaMemcpyAsync(c->state + c->L.env_params_off, c->agents.data(), N * 4, cudaMemcpyHostToDevice,
                    c->stream);
    cudaMemcpyAsync((void *)c->d.agent_off, off.data(), (N + 1) * 4, cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync((void *)c->d.slot_env, slot_env.data(), Sa * 4, cudaMemcpyHostToDevice, c->stream);
    e = cudaStreamSynchronize(c->stream);  // host staging vectors end here
    if (e == cudaSuccess && c->L.econ_fused) {
      econ_tc_init();
      if (set_econ_items(c) != WS_OK) {
        ws_status r = c->err;
        ws_destroy(c);
        return r;
      }
    }
    if (e != cudaSuccess) {
      cuda_check(c, e, "upload agent counts");
      ws_status r = c->err;
      ws_destroy(c);
      return r;
    }
  }
  launch_init_policy((float *)c->d.params, c->L.pol, cfg->param_seed, 0, c->stream);
  if (cfg->flags & WS_FLAG_TRAIN) {  // the critics: policy ids 2 (and 3, the planner's)
    launch_init_policy((float *)(c->state + c->L.critic_off), critic_shape(c->L.pol),
                       cfg->param_seed, 2, c->stream);
    if (cfg->env == WS_ENV_ECONOMY)
      launch_init_policy((float *)(c->state + c->L.critic_off + up(critic_shape(c->L.pol).count() * 4)),
                         critic_shape(c->L.pol_planner), cfg->param_seed, 3, c->stream);
  }
  if (cfg->env == WS_ENV_ECONOMY)
    launch_init_policy((float *)c->d.params_planner, c->L.pol_planner, cfg->param_seed, 1, c->stream);
  if (cfg->env == WS_ENV_LANDSCAPE) launch_init_landscape(c->d, cfg->param_seed, c->stream);
  if (use_tc_control(cfg)) c->tc_grid = control_tc_default_grid(c->d);
  if (use_tc_layers(cfg)) dense_tc_init();
  if (c->d.mlp3) mlp3_tc_init();
  if (use_tc_layers(cfg) && cfg->env == WS_ENV_LANDSCAPE) energy_tc_init((int)cfg->n_gauss);
  if (c->L.land_fused) land_tc_init();
  s = after_params_changed(c);
  if (s == WS_OK) s = ws_reset(c, cfg->param_seed);
  if (s == WS_OK) s = cuda_check(c, cudaStreamSynchronize(c->stream), "create sync");
  if (s != WS_OK) {
    ws_destroy(c);
    return s;
  }
  *out = c;
  return WS_OK;
}

ws_status ws_reset(ws_ctx *c, uint64_t seed) {
  if (!c) return WS_ERR_INVALID;
  if (c->err != WS_OK) return c->err;
  if (seed != c->seed) drop_graphs(c);  // graphs bake the key into their launches
  c->seed = seed;
  c->d.seed = seed;
  cudaMemsetAsync(c->d.k, 0, 8, c->stream);
  // the economy's per-step income accumulator must start at zero (every step
  // clears it after use; a fresh caller buffer holds arbitrary bytes)
  if (c->d.income) cudaMemsetAsync(c->d.income, 0, (size_t)c->L.n_agent_slots * 8, c->stream);
  // landscape energy partials: the tensor-core path fills only the first slots
  if (c->d.epart)
    cudaMemsetAsync(c->d.epart, 0, (size_t)kEnergyChunks * 2 * c->L.n_envs * 4, c->stream);
  launch_reset(c->d, c->stream);
  c->k_host = 0;
  c->ring_gen += 1;
  return cuda_check(c, cudaGetLastError(), "reset");
}

ws_status ws_step(ws_ctx *c) {
  if (!c) return WS_ERR_INVALID;
  if (c->err != WS_OK) return c->err;
  ws_status s = enqueue_steps(c, 1, c->stream);
  c->ring_gen += 1;
  if (s == WS_OK) c->k_host += 1;
  return s;
}

ws_status ws_rollout(ws_ctx *c, uint32_t n) {
  if (!c) return WS_ERR_INVALID;
  if (c->err != WS_OK) return c->err;
  if (n == 0) return WS_OK;
  ws_status s = WS_OK;
  if (c->cfg.path == WS_PATH_PLAIN_FP32) {
    for (uint32_t i = 0; i < n && s == WS_OK; ++i) s = enqueue_steps(c, 1, c->stream);
  } else if (fused(c)) {
    cudaGraphExec_t g;
    s = graph_for(c, n, &g);
    if (s == WS_OK) s = cuda_check(c, cudaGraphLaunch(g, c->stream), "graph launch");
  } else {
    const uint32_t chunk = chunk_of(c);
    const uint32_t full = n / chunk, rem = n % chunk;
    cudaGraphExec_t g;
    if (full) {
      s = graph_for(c, chunk, &g);
      for (uint32_t i = 0; i < full && s == WS_OK; ++i)
        s = cuda_check(c, cudaGraphLaunch(g, c->stream), "graph launch");
    }
    if (rem && s == WS_OK) {
      s = graph_for(c, rem, &g);
      if (s == WS_OK) s = cuda_check(c, cudaGraphLaunch(g, c->stream), "graph launch");
    }
  }
  c->ring_gen += 1;
  if (s == WS_OK) c->k_host += n;
  return s;
}

ws_status ws_returns(ws_ctx *c, uint32_t n) {
  if (!c) return WS_ERR_INVALID;
  if (c->err != WS_OK) return c->err;
  if (n == 0 || n > c->k_host || n > c->L.ring_steps) return WS_ERR_RANGE;
  launch_returns(c->d, n, c->stream);
  return cuda_check(c, cudaGetLastError(), "returns");
}

ws_status ws_a2c_update(ws_ctx *c, uint32_t n, float lr, float c_v, float c_e, double *stats) {
  if (!c) return WS_ERR_INVALID;
  if (c->err != WS_OK) return c->err;
  if (!(c->cfg.flags & WS_FLAG_TRAIN)) return WS_ERR_STATE;
  if (n == 0 || n > c->k_host || n > c->L.ring_steps) return WS_ERR_RANGE;
  if (!std::isfinite(lr) || !std::isfinite(c_v) || !std::isfinite(c_e)) return WS_ERR_INVALID;
  const TrainBufs tb = train_bufs((uint8_t *)c->state + c->L.train_off, c->L.pol);
  TrainGroup g[2];
  const int ng = train_groups(c, g);
  launch_returns(c->d, n, c->stream);
  launch_a2c_update(c->d, tb, g, ng, n, lr, c_v, c_e, c->stream);
  return finish_update(c, tb, n, stats, 3, "a2c update");
}

ws_status ws_advantages(ws_ctx *c, uint32_t n) {
  if (!c) return WS_ERR_INVALID;
  if (c->err != WS_OK) return c->err;
  if (!(c->cfg.flags & WS_FLAG_TRAIN)) return WS_ERR_STATE;
  if (n == 0 || n > c->k_host || n > c->L.ring_steps) return WS_ERR_RANGE;
  const TrainBufs tb = train_bufs((uint8_t *)c->state + c->L.train_off, c->L.pol);
  TrainGroup g[2];
  const int ng = train_groups(c, g);
  launch_returns(c->d, n, c->stream);
  launch_advantages(c->d, tb, g, ng, n, c->stream);
  ws_status s = cuda_check(c, cudaGetLastError(), "advantages");
  if (s == WS_OK) {
    c->adv_gen = c->ring_gen;
    c->adv_n = n;
  }
  return s;
}

ws_status ws_ppo_update(ws_ctx *c, uint32_t n, float lr, float eps, float c_v, float c_e,
                        double *stats) {
  if (!c) return WS_ERR_INVALID;
  if (c->err != WS_OK) return c->err;
  if (!(c->cfg.flags & WS_FLAG_TRAIN)) return WS_ERR_STATE;
  if (!std::isfinite(lr) || !std::isfinite(c_v) || !std::isfinite(c_e) || !std::isfinite(eps) ||
      !(eps > 0.f))
    return WS_ERR_INVALID;
  if (n == 0 || n > c->k_host || n > c->L.ring_steps) return WS_ERR_RANGE;
  if (c->adv_gen != c->ring_gen || n > c->adv_n) return WS_ERR_STATE;
  const TrainBufs tb = train_bufs((uint8_t *)c->state + c->L.train_off, c->L.pol);
  TrainGroup g[2];
  const int ng = train_groups(c, g);
  launch_ppo_update(c->d, tb, g, ng, n, lr, eps, c_v, c_e, c->stream);
  return finish_update(c, tb, n, stats, 4, "ppo update");
}

ws_status ws_forces(ws_ctx *c, uint32_t n) {
  if (!c) return WS_ERR_INVALID;
  if (c->err != WS_OK) return c->err;
  if (!(c->cfg.flags & WS_FLAG_FORCE)) return WS_ERR_STATE;
  if (n == 0 || n > c->k_host || n > c->L.ring_steps) return WS_ERR_RANGE;
  launch_forces(c->d, n, c->stream);
  return cuda_check(c, cudaGetLastError(), "forces");
}

}  // extern "C"

// Bytes per step of a ring field (0 if the context has no such field).
size_t ws_field_step_bytes(const ws_ctx *c, ws_field f) {
  size_t off = 0;
  return c ? ring_field_step_bytes(c, f, &off) : 0;
}

// Fetch on an explicit stream, without waiting (the copy is ordered after the
// work already enqueued on that stream only).
ws_status ws_fetch_async(ws_ctx *c, ws_field f, uint64_t t0, uint32_t n, void *dst,
                         size_t dst_bytes, int on_dev, cudaStream_t st) {
  if (!c || (!dst && dst_bytes)) return WS_ERR_INVALID;
  if (c->err != WS_OK) return c->err;
  const cudaMemcpyKind kind = on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (f == WS_F_STATE || f == WS_F_PARAMS || f == WS_F_ENV_PARAMS || f == WS_F_LOGITS ||
      f == WS_F_CRITIC) {
    if (t0 != 0 || n != 0) return WS_ERR_INVALID;
    if (f == WS_F_LOGITS &&
        (use_tc_control(&c->cfg) || ((c->L.econ_fused || c->L.land_fused) && !c->d.dbg_logits)))
      return WS_ERR_UNSUPPORTED;
    std::vector<Piece> v = state_pieces(c, f);
    if (v.empty()) return WS_ERR_INVALID;
    size_t tot = 0;
    for (auto &p : v) tot += p.n;
    if (dst_bytes < tot) return WS_ERR_NOMEM;
    char *o = (char *)dst;
    for (auto &p : v) {
      ws_status s = cuda_check(c, cudaMemcpyAsync(o, p.p, p.n, kind, st), "fetch copy");
      if (s != WS_OK) return s;
      o += p.n;
    }
    return WS_OK;
  }
  size_t foff = 0;
  const size_t per = ring_field_step_bytes(c, f, &foff);
  if (per == 0) return WS_ERR_INVALID;
  if (n == 0) return WS_OK;
  const uint64_t R = c->L.ring_steps;
  const uint64_t lo = c->k_host > R ? c->k_host - R : 0;
  if (t0 < lo || t0 + n > c->k_host) return WS_ERR_RANGE;
  if (dst_bytes < per * n) return WS_ERR_NOMEM;
  char *o = (char *)dst;
  uint64_t t = t0;
  uint32_t left = n;
  while (left) {
    const uint64_t row = t % R;
    const uint32_t run = (uint32_t)((R - row) < left ? (R - row) : left);
    ws_status s = cuda_check(
        c, cudaMemcpyAsync(o, c->ring + foff + row * per, per * run, kind, st), "fetch copy");
    if (s != WS_OK) return s;
    o += per * run;
    t += run;
    left -= run;
  }
  return WS_OK;
}

extern "C" {

ws_status ws_fetch(ws_ctx *c, ws_field f, uint64_t t0, uint32_t n, void *dst, size_t dst_bytes,
                   int on_dev) {
  if (!c) return WS_ERR_INVALID;
  ws_status s = ws_fetch_async(c, f, t0, n, dst, dst_bytes, on_dev, c->stream);
  if (s != WS_OK) return s;
  if (!on_dev) return cuda_check(c, cudaStreamSynchronize(c->stream), "fetch sync");
  return WS_OK;
}

ws_status ws_load(ws_ctx *c, ws_field f, const void *src, size_t src_bytes, int on_dev, uint64_t k) {
  if (!c || !src) return WS_ERR_INVALID;
  if (c->err != WS_OK) return c->err;
  if (f != WS_F_STATE && f != WS_F_PARAMS && f != WS_F_ENV_PARAMS && f != WS_F_CRITIC)
    return WS_ERR_INVALID;
  if (f == WS_F_ENV_PARAMS && c->cfg.env != WS_ENV_LANDSCAPE) return WS_ERR_INVALID;
  if (f == WS_F_CRITIC && !(c->cfg.flags & WS_FLAG_TRAIN)) return WS_ERR_INVALID;
  if (f == WS_F_STATE && k == UINT64_MAX) return WS_ERR_INVALID;
  std::vector<Piece> v = state_pieces(c, f);
  size_t tot = 0;
  for (auto &p : v) tot += p.n;
  if (src_bytes != tot) return WS_ERR_INVALID;
  const cudaMemcpyKind kind = on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const char *i = (const char *)src;
  for (auto &p : v) {
    ws_status s = cuda_check(c, cudaMemcpyAsync(p.p, i, p.n, kind, c->stream), "load copy");
    if (s != WS_OK) return s;
    i += p.n;
  }
  if (f == WS_F_STATE && c->cfg.env == WS_ENV_LANDSCAPE)
    cudaMemsetAsync(c->d.needs_energy, 0, c->L.n_envs, c->stream);
  if (f != WS_F_STATE) {
    ws_status s = after_params_changed(c);
    if (s != WS_OK) return s;
  }
  if (k != UINT64_MAX) {
    ws_status s = cuda_check(c, cudaMemcpyAsync(c->d.k, &k, 8, cudaMemcpyHostToDevice, c->stream),
                             "load step");
    if (s != WS_OK) return s;
    c->k_host = k;
    c->ring_gen += 1;
  }
  // pageable host sources are consumed before return
  if (!on_dev || k != UINT64_MAX) return cuda_check(c, cudaStreamSynchronize(c->stream), "load sync");
  return WS_OK;
}

ws_status ws_get_step(const ws_ctx *c, uint64_t *k) {
  if (!c || !k) return WS_ERR_INVALID;
  *k = c->k_host;
  return WS_OK;
}

ws_status ws_sync(ws_ctx *c, uint32_t timeout_ms) {
  if (!c) return WS_ERR_INVALID;
  if (c->err != WS_OK) return c->err;
  ws_status s = cuda_check(c, cudaEventRecord(c->ev, c->stream), "sync record");
  if (s != WS_OK) return s;
  const auto t_end = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
  for (;;) {
    cudaError_t e = cudaEventQuery(c->ev);
    if (e == cudaSuccess) break;
    if (e != cudaErrorNotReady) return cuda_check(c, e, "sync query");
    if (timeout_ms && std::chrono::steady_clock::now() >= t_end) return WS_ERR_TIMEOUT;
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  uint32_t flag[2] = {0, 0};
  s = cuda_check(c, cudaMemcpy(flag, c->d.err, 8, cudaMemcpyDeviceToHost), "sync flag");
  if (s != WS_OK) return s;
  if (flag[0]) {
    char buf[96];
    std::snprintf(buf, sizeof buf, "device wait ran out (site %u)", flag[1]);
    return fail(c, WS_ERR_TIMEOUT, buf);
  }
  // WS_FLAG_BOUNDS_CHECK: every region's canary must still hold its fill byte
  for (int b = 0; b < 2; ++b) {
    const std::vector<Canary> &spots = b ? c->ring_spots : c->state_spots;
    const char *base = b ? c->ring : c->state;
    for (const Canary &k : spots) {
      unsigned char tail[kCanary];
      s = cuda_check(c, cudaMemcpy(tail, base + k.off, kCanary, cudaMemcpyDeviceToHost), "canary");
      if (s != WS_OK) return s;
      for (size_t i = 0; i < kCanary; ++i)
        if (tail[i] != kCanaryByte) {
          char buf[160];
          std::snprintf(buf, sizeof buf,
                        "canary overwritten (%s buffer, canary after %s at byte %zu, offset %zu)",
                        b ? "ring" : "state", k.after, k.off + i, i);
          return fail(c, WS_ERR_CUDA, buf);
        }
    }
  }
  return WS_OK;
}

const char *ws_last_error(const ws_ctx *c) { return c ? c->msg.c_str() : "null context"; }

ws_status ws_get_launch(const ws_ctx *c, ws_launch *out) {
  if (!c || !out) return WS_ERR_INVALID;
  *out = c->lc;
  return WS_OK;
}

ws_status ws_set_launch(ws_ctx *c, const ws_launch *l) {
  if (!c || !l || l->struct_size != sizeof(ws_launch)) return WS_ERR_INVALID;
  if (c->err != WS_OK) return c->err;
  if (l->chunk_steps < 1 || (c->cfg.chunk_steps && l->chunk_steps != c->cfg.chunk_steps))
    return WS_ERR_INVALID;
  if (l->grid > 65535 || l->econ_tiles < 1 || l->econ_tiles > 3 || l->econ_lpt > 1)
    return WS_ERR_INVALID;
  if (c->L.econ_fused && (int)l->econ_tiles * 128 < max_agents(c)) return WS_ERR_INVALID;
  if (l->energy_chunks != 1 && l->energy_chunks != 2 && l->energy_chunks != 4) return WS_ERR_INVALID;
  if (c->d.eimg && !energy_tc_chunks_ok((int)c->cfg.n_gauss, (int)l->energy_chunks))
    return WS_ERR_INVALID;
  if (l->env_threads < 64 || l->env_threads > 1024 || l->env_threads % 32) return WS_ERR_INVALID;
  if (l->tile_ctas != 1 && l->tile_ctas != 2) return WS_ERR_INVALID;
  const uint32_t tpe = l->ctrl_threads_per_env;
  if (tpe != 4 && tpe != 8 && tpe != 16 && tpe != 64) return WS_ERR_INVALID;
  if (l->ctrl_envs_per_cta > 32 || l->update_gemm > 1) return WS_ERR_INVALID;
  if (l->ctrl_envs_per_cta && use_tc_control(&c->cfg) &&
      (!control_cc_supported(c->L.pol) ||
       !control_cc_tile_ok(c->L.pol, (int)l->ctrl_envs_per_cta, (int)tpe)))
    return WS_ERR_INVALID;
  const ws_launch old = c->lc;
  c->lc = *l;
  drop_graphs(c);  // graphs bake the launch parameters in
  c->d.env_threads = (int)l->env_threads;
  c->d.energy_chunks = (int)l->energy_chunks;
  c->d.update_simt = (int)l->update_gemm;
  c->d.wait_ns = device_wait_ns(*l);
  if (c->L.econ_fused && (old.econ_tiles != l->econ_tiles || old.econ_lpt != l->econ_lpt)) {
    ws_status s = set_econ_items(c);
    if (s != WS_OK) return s;
  }
  if (c->d.epart && old.energy_chunks != l->energy_chunks)  // unused partial slots read as zero
    return cuda_check(c, cudaMemsetAsync(c->d.epart, 0, (size_t)kEnergyChunks * 2 * c->L.n_envs * 4,
                                         c->stream), "launch change");
  return WS_OK;
}

}  // extern "C"

namespace {

// Process-wide cache of tuned launch configurations, keyed by the shape of the
// configuration (everything that changes speed, nothing that changes results'
// identity such as seeds).
std::mutex g_tune_mu;
std::map<std::string, std::pair<ws_launch, float>> g_tune_cache;

std::string tune_key(const ws_ctx *c) {
  int dev = 0;
  cudaGetDevice(&dev);
  uint64_t h = 1469598103934665603ull;  // FNV-1a over the agent counts
  for (int32_t a : c->agents) {
    h ^= (uint32_t)a;
    h *= 1099511628211ull;
  }
  char buf[256];
  std::snprintf(buf, sizeof buf, "%d/%d/%u/%u/%u/%u/%u/%u/%u/%llx/%d/%d", c->cfg.env, c->cfg.path,
                c->cfg.n_envs, c->cfg.hidden0, c->cfg.hidden1, c->cfg.dim, c->cfg.n_gauss,
                c->cfg.chunk_steps, c->cfg.flags, (unsigned long long)h, dev, sm_count());
  return buf;
}

// Candidate launch configurations of the context's path (cartesian product of
// the knobs the path has; chunk lengths above the trial length are pointless).
std::vector<ws_launch> tune_candidates(const ws_ctx *c, uint32_t trial) {
  std::vector<uint32_t> chunks;
  if (c->cfg.chunk_steps) {
    chunks.push_back(c->cfg.chunk_steps);
  } else if (c->cfg.path == WS_PATH_PLAIN_FP32) {
    chunks.push_back(c->lc.chunk_steps);
  } else {
    const uint32_t opts_f[] = {25u, 50u, 100u, 200u}, opts_s[] = {10u, 25u, 50u};
    const uint32_t *o = fused(c) ? opts_f : opts_s;
    const int no = fused(c) ? 4 : 3;
    for (int i = 0; i < no; ++i)
      if (o[i] <= trial) chunks.push_back(o[i]);
    if (chunks.empty()) chunks.push_back(trial);
  }
  std::vector<uint32_t> grids{0u}, tiles{c->lc.econ_tiles}, lpts{c->lc.econ_lpt},
      echunks{c->lc.energy_chunks}, threads{c->lc.env_threads}, tctas{c->lc.tile_ctas};
  if (c->L.land_fused) tctas = {1u, 2u};
  if (use_tc_control(&c->cfg)) {
    const uint32_t n_tiles = (c->L.n_envs + 127) / 128, half = (n_tiles + 1) / 2;
    if (half >= 1 && half < (uint32_t)c->tc_grid) grids.push_back(half);
  }
  if (c->L.econ_fused) {
    tiles.clear();
    for (uint32_t t = (uint32_t)((max_agents(c) + 127) / 128); t <= 3; ++t) tiles.push_back(t);
    lpts = {1u, 0u};
  }
  if (c->d.eimg && !c->L.land_fused) {
    echunks.clear();
    for (uint32_t e : {1u, 2u, 4u})
      if (energy_tc_chunks_ok((int)c->cfg.n_gauss, (int)e)) echunks.push_back(e);
  }
  if (!fused(c)) threads = {128u, 256u, 512u};
  // classic-control kernel choice: {0, -} the tensor-core tiles, else the
  // CUDA-core kernel's (envs per CTA, envs per thread); offered while 128-env
  // tiles would leave most SMs idle
  std::vector<std::pair<uint32_t, uint32_t>> ctrl{{0u, c->lc.ctrl_threads_per_env}};
  if (use_tc_control(&c->cfg) && control_cc_supported(c->L.pol) &&
      c->L.n_envs <= 256u * (uint32_t)sm_count())
    for (uint32_t ne : {1u, 2u, 4u, 8u, 16u, 32u})
      for (uint32_t tpe : {4u, 8u, 16u, 64u})
        if (control_cc_tile_ok(c->L.pol, (int)ne, (int)tpe)) ctrl.push_back({ne, tpe});
  std::vector<ws_launch> v;
  for (uint32_t ch : chunks)
    for (uint32_t g : grids)
      for (uint32_t t : tiles)
        for (uint32_t lp : lpts)
          for (uint32_t ec : echunks)
            for (uint32_t th : threads)
              for (uint32_t tcs : tctas) {
              ws_launch l = c->lc;
              l.tile_ctas = tcs;
              l.chunk_steps = ch;
              l.grid = g;
              l.econ_tiles = t;
              l.econ_lpt = lp;
              l.energy_chunks = ec;
              l.env_threads = th;
              for (const auto &cc : ctrl) {
                if (cc.first && g) continue;  // the CUDA-core kernel has no grid knob
                l.ctrl_envs_per_cta = cc.first;
                l.ctrl_threads_per_env = cc.second;
                v.push_back(l);
              }
            }
  return v;
}

}  // namespace

extern "C" {

ws_status ws_tune(ws_ctx *c, uint32_t trial_steps, ws_launch *chosen, float *ms_per_step) {
  if (!c || trial_steps == 0) return WS_ERR_INVALID;
  if (c->err != WS_OK) return c->err;
  const std::string key = tune_key(c);
  ws_launch best = c->lc;
  float best_ms = -1.f;
  {
    std::lock_guard<std::mutex> g(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      best = it->second.first;
      best_ms = it->second.second;
    }
  }
  if (best_ms < 0.f) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ws_status s = cuda_check(c, cudaEventCreate(&e0), "tune event");
    if (s == WS_OK) s = cuda_check(c, cudaEventCreate(&e1), "tune event");
    for (const ws_launch &cand : tune_candidates(c, trial_steps)) {
      if (s != WS_OK) break;
      s = ws_set_launch(c, &cand);
      if (s == WS_OK) s = ws_rollout(c, trial_steps);  // untimed: graph capture, warm caches
      // the best of three timed trials (a short trial's single time is noisy)
      float ms = -1.f;
      for (int rep = 0; rep < 3 && s == WS_OK; ++rep) {
        s = cuda_check(c, cudaEventRecord(e0, c->stream), "tune record");
        if (s == WS_OK) s = ws_rollout(c, trial_steps);
        if (s == WS_OK) s = cuda_check(c, cudaEventRecord(e1, c->stream), "tune record");
        if (s == WS_OK) s = cuda_check(c, cudaEventSynchronize(e1), "tune sync");
        if (s == WS_OK) s = ws_sync(c, 0);  // surfaces a device-side failure of the trial
        float t = 0.f;
        if (s == WS_OK) s = cuda_check(c, cudaEventElapsedTime(&t, e0, e1), "tune time");
        if (s == WS_OK && (ms < 0.f || t < ms)) ms = t;
      }
      if (s == WS_OK && (best_ms < 0.f || ms < best_ms)) {
        best_ms = ms;
        best = cand;
      }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s != WS_OK) return s;
    best_ms /= (float)trial_steps;
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune_cache[key] = {best, best_ms};
  }
  ws_status s = ws_set_launch(c, &best);
  if (s == WS_OK) s = ws_reset(c, c->seed);
  if (s == WS_OK) s = cuda_check(c, cudaStreamSynchronize(c->stream), "tune reset");
  if (s != WS_OK) return s;
  if (chosen) *chosen = best;
  if (ms_per_step) *ms_per_step = best_ms;
  return WS_OK;
}

void ws_destroy(ws_ctx *c) {
  if (!c) return;
  if (c->stream || c->ev) cudaStreamSynchronize(c->stream);
  drop_graphs(c);
  if (c->br.aux) cudaStreamSynchronize(c->br.aux);
  if (c->br.fork) cudaEventDestroy(c->br.fork);
  if (c->br.join) cudaEventDestroy(c->br.join);
  if (c->br.aux) cudaStreamDestroy(c->br.aux);
  if (c->ev) cudaEventDestroy(c->ev);
  if (c->capture) cudaStreamDestroy(c->capture);
  delete c;
}

}  // extern "C"
