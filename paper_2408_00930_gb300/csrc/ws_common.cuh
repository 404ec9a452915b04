// ws_common.cuh -- shared device/host pieces of the roll-out engine:
// Philox4x32-10, the variate maps, the draw tags, and the context layout.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/warpsci.h"

#define WS_HD __host__ __device__ __forceinline__

namespace ws {

// Counter-based generator of Salmon, Moraes, Dror, Shaw (SC'11, Sec. 5):
// ten rounds of two 32x32->64 products whose halves are XOR-ed into the other
// counter words with the round key; the key advances by the Weyl increments.
struct Philox {
  static constexpr uint32_t kMulA = 0xD2511F53u, kMulB = 0xCD9E8D57u;
  static constexpr uint32_t kWeylA = 0x9E3779B9u, kWeylB = 0xBB67AE85u;
};

WS_HD uint32_t mul_hi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
  return __umulhi(a, b);
#else
  return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
}

WS_HD uint4 philox10(uint4 c, uint32_t key_lo, uint32_t key_hi) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t a_hi = mul_hi32(Philox::kMulA, c.x), a_lo = Philox::kMulA * c.x;
    const uint32_t b_hi = mul_hi32(Philox::kMulB, c.z), b_lo = Philox::kMulB * c.z;
    c = make_uint4(b_hi ^ c.y ^ key_lo, b_lo, a_hi ^ c.w ^ key_hi, a_lo);
    key_lo += Philox::kWeylA;
    key_hi += Philox::kWeylB;
  }
  return c;
}

enum Tag : uint32_t {
  kTagAction = 0,
  kTagReset = 1,
  kTagPartner = 2,
  kTagNoise = 3,
  kTagPolicyInit = 4,
  kTagLandscapeInit = 5,
  kTagEconInit = 6
};
constexpr uint32_t kPlannerId = 0xFFFFFFFFu;
constexpr uint32_t kStepInit = 0xFFFFFFFFu;  // the draw of a full reset ("step -1")

WS_HD uint4 draw(uint64_t seed, uint32_t c0, uint32_t env, uint32_t agent, uint32_t tag,
                 uint32_t sub) {
  return philox10(make_uint4(c0, env, agent, (tag << 24) | (sub & 0xFFFFFFu)), (uint32_t)seed,
                  (uint32_t)(seed >> 32));
}

// Top 24 bits as a float in [0, 1); exact.
WS_HD float u01(uint32_t w) { return (float)(w >> 8) * 0x1p-24f; }

// U(a, b) := fmaf(b - a, u, a), one rounding.
WS_HD float uniform(uint32_t w, float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(b - a, u01(w), a);
#else
  return fmaf(b - a, u01(w), a);
#endif
}

// Box-Muller on a word pair: u1 in (0, 1], u2 in [0, 1).
__device__ __forceinline__ float2 box_muller(uint32_t w0, uint32_t w1) {
  const float u1 = (float)((w0 >> 8) + 1u) * 0x1p-24f;
  const float u2 = (float)(w1 >> 8) * 0x1p-24f;
  const float rho = sqrtf(-2.0f * logf(u1));
  float s, c;
  sincospif(2.0f * u2, &s, &c);
  return make_float2(rho * c, rho * s);
}

WS_HD uint32_t bounded(uint32_t w, uint32_t n) { return mul_hi32(w, n); }

// ------------------------------------------------------------------------
// Context layout: byte offsets into the caller's state and ring buffers.
// ------------------------------------------------------------------------
constexpr int kEconF = 16;
constexpr int kAcroObs = 6;  // acrobot observation: cos/sin of both angles, both velocities
constexpr int kMaxLayers = 3;

struct PolicyShape {
  int w[kMaxLayers + 1];  // widths in -> h0 -> h1 -> out
  WS_HD size_t count() const {
    size_t n = 0;
    for (int l = 0; l < kMaxLayers; ++l) n += (size_t)w[l] * w[l + 1] + w[l + 1];
    return n;
  }
  WS_HD size_t layer_offset(int l) const {
    size_t n = 0;
    for (int i = 0; i < l; ++i) n += (size_t)w[i] * w[i + 1] + w[i + 1];
    return n;
  }
};

struct Layout {
  int env, path;
  uint32_t n_envs, n_slots, n_agent_slots, ring_steps, obs_dim, act_dim, n_out, n_out_planner;
  PolicyShape pol, pol_planner;
  // state buffer
  size_t k_off;            // u64 step counter
  size_t err_off;          // u32 device error flag + u32 where
  size_t params_off;       // f32 policy params (agent)
  size_t params_planner_off;
  size_t packed_off;       // bf16 tensor-core operand images of the policy
  size_t packed_bytes;
  size_t env_params_off;   // landscape centres/widths/amps (+ derived), econ counts
  size_t env_derived_off;  // landscape: cnorm[M], coef[M], bf16 hi/lo centre images
  size_t env_derived_bytes;
  size_t state_off;        // env state
  size_t t_off;            // i32 episode step per env
  size_t aux_off;          // economy: agent offsets [n_envs+1] and slot->env map
  size_t items_off;        // economy, fused kernel: work items [n_envs][4] i32
  size_t queue_off;        // economy, fused kernel: work-queue counters (2 x u32)
  int econ_fused;          // economy on the fused persistent kernel
  int land_fused;          // landscape on the fused persistent kernel
  size_t land_energy_off;
  size_t force_img_off;     // landscape, fused kernel with WS_FLAG_FORCE: the force image
  size_t critic_off, train_off;  // WS_FLAG_TRAIN: critic parameters, update scratch
  size_t scratch_off;      // plain-path activations
  size_t scratch_h0_off, scratch_h1_off, scratch_out_off;
  size_t scratch_pobs_off, scratch_ph0_off, scratch_ph1_off, scratch_pout_off;
  size_t scratch_income_off;
  size_t state_bytes;
  // ring buffer: per field, [ring_steps][...]
  size_t ring_obs, ring_act, ring_logp, ring_rew, ring_done, ring_ret, ring_wealth, ring_energy;
  size_t ring_force;  // landscape with WS_FLAG_FORCE
  size_t ring_adv;    // WS_FLAG_TRAIN: advantages of ws_advantages
  size_t ring_sample; // landscape with WS_FLAG_TRAIN: behaviour samples of ws_advantages
  size_t ring_pout;   // WS_FLAG_DEBUG_LOGITS: every step's policy outputs
  size_t ring_bytes;
};

}  // namespace ws
