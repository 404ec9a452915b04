// ws_control_cc.cu -- fused persistent CUDA-core roll-out kernels of the
// classic-control envs (the control env and the acrobot, paper App. C) for env
// counts too small to fill the GPU with 128-env tensor-core tiles.
//
// Paper grounding: Sec. 2 / App. B keep the env step, the policy forward, the
// sampling and the in-place store on the GPU with no host round-trip; the envs
// are independent.  The tensor-core kernel (ws_control_tc.cu) gives each SM a
// 128-env tile and runs one step of a tile as a serial chain (layer-1 MMA, tanh,
// layer-2 MMAs, tanh, sampling, env step); with 1,000 envs only 8 SMs work and a
// step costs that whole chain (~3.4 K cycles, most of it MMA round trips and the
// SFU work of 128 rows on one SM).  Here a CTA serves NE envs on the CUDA cores
// instead, so that the envs spread over many SMs; a step is three phases
// between CTA barriers:
//   P2  layer 1: z1 = b1 + o W1 in FP32, h1 = tanh(z1) on the SFU's packed
//       bf16x2 form (the operand precision of the tensor-core path), h1 to
//       shared memory [env][unit]
//   P3  layer 2: z2 = b2 + h1 W2 with W2 rounded to BF16 (as the tensor-core
//       path's operands) and FP32 accumulation, h2 = tanh(z2) in FP32, then the
//       layer-3 partial dot products h2 W3
//   P4  one thread per env ("env lane"): logits + b3, categorical inverse-CDF
//       draw, env step, reward, done, auto-reset, the time-major record write
//       and the next observation; meanwhile two threads per env of another warp
//       draw the next step's action uniform and reset words (Philox, double-
//       buffered by step parity) and, for the control env, take sin / cos of the
//       next pole angle (the Euler step of the angle does not depend on the
//       action), so that neither is on the env lanes' chain.
// Two work splits ("threads per env", a launch parameter):
//   tiled (4, 8 or 16 threads per env)  16 unit groups of H / 16 consecutive
//       hidden units times NE / RE env groups of RE = 16 / threads-per-env envs;
//       thread t owns unit group t % 16 of env group t / 16 (a half-warp per env
//       group), W2 in shared memory; the layer-3 partials of the 16 unit groups
//       meet in a butterfly of warp shuffles (partner g ^ 1, then g ^ 2, g ^ 4,
//       g ^ 8)
//   unit per thread (64 threads per env, H = 64)  thread u of an env owns hidden
//       unit u with its W2 column in registers (h1 read as shared-memory
//       broadcasts), for the smallest env counts where the step's latency, not
//       the SM's throughput, decides; the first lane of each group of four units
//       forms the group's partial, the butterfly runs over those lanes inside
//       each of the env's two warps, and the env lane adds the two warps' sums
// Both run every accumulation in one fixed order: z1 from b1 over the inputs in
// order; z2 as two chains in k order (from b2 over the first half of k, from
// zero over the second) added; per unit group of H / 16 units the layer-3
// partial as an FMA chain over its units from zero; the 16 group partials summed
// in the butterfly's pairing (group g with g ^ 1, then g ^ 2, g ^ 4, g ^ 8).
// Every split and every NE therefore gives bit-identical records.  No device
// waits beyond the CTA barriers.
#include "ws_acrobot.cuh"
#include "ws_kernels.cuh"
#include "ws_tc.cuh"

namespace ws {

namespace {

constexpr int kUG = 16;  // unit groups of the layer-3 partials

struct CcCart {
  static constexpr int OBS = 4, NA = 2;
};
struct CcAcro {
  static constexpr int OBS = 6, NA = 3;
};

// State of an env lane and its observation.
template <typename E>
struct Lane {
  float x = 0.f, v = 0.f, th = 0.f, w = 0.f;  // acrobot: (th1, th2, w1, w2)
  int tep = 0;
  bool fresh = true;  // the state is not the Euler step of the last one (start, reset)
  float ob[E::OBS] = {};
};

template <typename E>
__device__ __forceinline__ void lane_load(const Dev &d, Lane<E> &s, uint32_t e) {
  const uint32_t N = d.n_envs;
  s.x = d.s[e];
  s.v = d.s[N + e];
  s.th = d.s[2 * N + e];
  s.w = d.s[3 * N + e];
  s.tep = d.t[e];
}
template <typename E>
__device__ __forceinline__ void lane_store(const Dev &d, const Lane<E> &s, uint32_t e) {
  const uint32_t N = d.n_envs;
  d.s[e] = s.x;
  d.s[N + e] = s.v;
  d.s[2 * N + e] = s.th;
  d.s[3 * N + e] = s.w;
  d.t[e] = s.tep;
}

// The observation of the lane's state into ob and into xo[i * stride].
template <typename E>
__device__ __forceinline__ void lane_observe(Lane<E> &s, float *xo, int stride) {
  if constexpr (E::NA == 3) {
    acro_sincos<true>(s.x, &s.ob[1], &s.ob[0]);
    acro_sincos<true>(s.v, &s.ob[3], &s.ob[2]);
    s.ob[4] = s.th;
    s.ob[5] = s.w;
  } else {
    s.ob[0] = s.x;
    s.ob[1] = s.v;
    s.ob[2] = s.th;
    s.ob[3] = s.w;
  }
#pragma unroll
  for (int i = 0; i < E::OBS; ++i) xo[i * stride] = s.ob[i];
}

// P4 of an env lane: the draw from the logits (b3 included), the env step, the
// records of step row, the auto-reset from the reset words rr[0], rr[rs], ...
// (control: sin / cos of the pole angle precomputed).
template <typename E>
__device__ __forceinline__ void lane_step(const Dev &d, Lane<E> &s, float l0, float l1v, float l2,
                                          float u, const uint32_t *rr, int rs, float sin_th,
                                          float cos_th, bool valid, uint32_t e, uint32_t row) {
  constexpr bool ACRO = E::NA == 3;
  const uint32_t S = d.n_slots;
  // categorical draw by inverse CDF: a = min{ i : u S < C_i } (C_i running sums
  // of exp(l - max), S the total)
  int a;
  float m, Ssum, la;
  if constexpr (ACRO) {
    m = fmaxf(fmaxf(l0, l1v), l2);
    const float e0 = expf(l0 - m), e1 = expf(l1v - m), e2 = expf(l2 - m);
    Ssum = (e0 + e1) + e2;
    const float thr = u * Ssum;
    a = thr < e0 ? 0 : (thr < e0 + e1 ? 1 : 2);
    la = a == 0 ? l0 : (a == 1 ? l1v : l2);
  } else {
    m = fmaxf(l0, l1v);
    const float e0 = expf(l0 - m), e1 = expf(l1v - m);
    Ssum = e0 + e1;
    a = (u * Ssum < e0) ? 0 : 1;
    la = a ? l1v : l0;
  }
  float ns[4];
  float rew;
  bool done;
  const int t2 = s.tep + 1;
  if constexpr (ACRO) {
    // RK4 of the two-link dynamics, dt = 0.2, torque a - 1
    ns[0] = s.x;
    ns[1] = s.v;
    ns[2] = s.th;
    ns[3] = s.w;
    acro_step<true>(ns, (float)(a - 1), 0.2f);
    const bool term = acro_terminal<true>(ns);
    rew = term ? 0.0f : -1.0f;
    done = term || t2 >= (int)d.episode_limit;
  } else {
    // explicit Euler, dt = 0.02
    const float uf = a ? 10.0f : -10.0f;
    const float xacc = uf - 0.5f * s.x - 0.1f * s.v;
    const float thacc = 9.8f * sin_th - 0.3f * cos_th * uf;
    ns[0] = s.x + 0.02f * s.v;
    ns[1] = s.v + 0.02f * xacc;
    ns[2] = __fmaf_rn(0.02f, s.w, s.th);  // the draw lanes predict sin / cos of this
    ns[3] = s.w + 0.02f * thacc;
    rew = 1.0f;
    done = fabsf(ns[0]) > 2.4f || fabsf(ns[2]) > 0.21f || t2 >= (int)d.episode_limit;
  }
  if (valid) {
    const float lp = (la - m) - logf(Ssum);
    const size_t o = (size_t)row * S + e;
    float *obr = d.r_obs + (size_t)row * E::OBS * S + e;
#pragma unroll
    for (int i = 0; i < E::OBS; ++i) obr[(size_t)i * S] = s.ob[i];
    ((int32_t *)d.r_act)[o] = a;
    d.r_logp[o] = lp;
    d.r_rew[o] = rew;
    d.r_done[o] = (uint8_t)done;
    if (d.r_pout) {  // the FP32 logits the draw read
      float *po = d.r_pout + (size_t)row * E::NA * S + e;
      po[0] = l0;
      po[S] = l1v;
      if (ACRO) po[2 * (size_t)S] = l2;
    }
  }
  s.fresh = done;
  if (done) {
    const float lim = ACRO ? 0.1f : 0.05f;
    s.x = uniform(rr[0], -lim, lim);
    s.v = uniform(rr[rs], -lim, lim);
    s.th = uniform(rr[2 * rs], -lim, lim);
    s.w = uniform(rr[3 * rs], -lim, lim);
    s.tep = 0;
  } else {
    s.x = ns[0];
    s.v = ns[1];
    s.th = ns[2];
    s.w = ns[3];
    s.tep = t2;
  }
}

// First thread of the draw lanes: the warp after the env lanes' (threads
// 0 .. NE - 1), so that their Philox rounds run beside the env lanes' P4.
__host__ __device__ constexpr int draw_lane0(int ne) { return 32 * ((ne + 31) / 32); }

// Draw lane i = slot - draw_lane0(NE) < 2 NE: the action uniform (i < NE) or the
// reset words (i >= NE) of step k for env base + i % NE, one Philox block each
// (the same instructions on every lane of the warp).  For the control env the
// lanes also take sin / cos of the next pole angle th + 0.02 w (the Euler step
// does not depend on the action; (th, w) read during P3), into sc[0 .. 2 NE):
// the env lane uses them unless its env was reset.
__device__ __forceinline__ void draw_lanes(const Dev &d, int slot, int NE, uint32_t base, uint32_t k,
                                           float *us, uint32_t *rrs, bool trig = false,
                                           float th = 0.f, float w = 0.f, float *sc = nullptr) {
  const int i = slot - draw_lane0(NE);
  if (i < 0 || i >= 2 * NE) return;
  const bool act = i < NE;
  const int q = act ? i : i - NE;
  const uint4 r = draw(d.seed, k, d.env_base + base + (uint32_t)q, 0, act ? kTagAction : kTagReset, 0);
  float sn = 0.f, cs = 0.f;
  if (trig) {
    const float th1 = __fmaf_rn(0.02f, w, th);
    sn = sinf(th1);
    cs = cosf(th1);
  }
  if (act) {
    us[q] = u01(r.x);
    if (trig) {
      sc[q] = sn;
      sc[NE + q] = cs;
    }
  } else {
    uint32_t *o = rrs + q;
    o[0] = r.x;
    o[NE] = r.y;
    o[2 * NE] = r.z;
    o[3 * NE] = r.w;
  }
}

// The pole angle and velocity of a draw lane's env (control env; read during
// P3, while xo holds this step's observations).
template <typename E>
__device__ __forceinline__ void draw_lane_state(int slot, int NE, const float *xo, float &th,
                                                float &w) {
  th = w = 0.f;
  const int i = slot - draw_lane0(NE);
  if (E::NA == 3 || i < 0 || i >= 2 * NE) return;
  const int q = i < NE ? i : i - NE;
  th = xo[2 * NE + q];
  w = xo[3 * NE + q];
}

// sin / cos of the env lane's pole angle: the draw lanes' prediction, or its
// own after a start or a reset.
template <typename E>
__device__ __forceinline__ void lane_trig(const Lane<E> &s, const float *sc, int NE, int q,
                                          float &sn, float &cs) {
  sn = cs = 0.f;
  if constexpr (E::NA == 2) {
    if (s.fresh) {
      sn = sinf(s.th);
      cs = cosf(s.th);
    } else {
      sn = sc[q];
      cs = sc[NE + q];
    }
  }
}

// ------------------------------------------------------------------ tiled
template <typename E, int H, int NE, int RE>
struct CtrlCc {
  static_assert(H == 64 || H == 128, "hidden width 64 or 128");
  static_assert(RE == 1 || RE == 2 || RE == 4, "envs per thread 1, 2 or 4");
  static_assert(NE % RE == 0 && NE % 4 == 0, "envs per CTA");
  static constexpr int RU = H / kUG;          // hidden units per thread (4 or 8)
  static constexpr int EG = NE / RE;          // env groups
  static constexpr int THREADS = kUG * EG;
  static constexpr int HP = H + 4;            // h1 row stride (floats)
  // shared memory, in floats; every array starts on a 16-byte boundary
  static constexpr int S_W1 = 0;                       // [OBS][H] FP32
  static constexpr int S_B1 = S_W1 + E::OBS * H;       // [H]
  static constexpr int S_W2 = S_B1 + H;                // [H][H] BF16-rounded, [k][unit]
  static constexpr int S_B2 = S_W2 + H * H;            // [H]
  static constexpr int S_W3 = S_B2 + H;                // [H][4] FP32, W3[u][0..NA-1] padded
  static constexpr int S_B3 = S_W3 + H * 4;            // [4]
  static constexpr int S_XO = S_B3 + 4;                // [OBS][NE] this step's observations
  static constexpr int S_H1 = S_XO + E::OBS * NE;      // [NE][HP] h1 (BF16 values)
  static constexpr int S_LG = S_H1 + NE * HP;          // [4][NE] logit sums without b3
  static constexpr int S_U = S_LG + 4 * NE;            // [2][NE] action uniforms (step parity)
  static constexpr int S_RR = S_U + 2 * NE;            // [2][4][NE] reset words (step parity)
  static constexpr int S_SC = S_RR + 8 * NE;           // [2][2][NE] predicted sin, cos (parity)
  static constexpr int FLOATS = S_SC + 4 * NE;
  static constexpr int SMEM = FLOATS * 4;
  static_assert(S_W2 % 4 == 0 && S_H1 % 4 == 0 && S_W3 % 4 == 0 && HP % 4 == 0, "alignment");
  static_assert(draw_lane0(NE) + 2 * NE <= THREADS, "env lanes, then the draw lanes' warps");
};

template <typename E, int H, int NE, int RE>
__global__ void __launch_bounds__(CtrlCc<E, H, NE, RE>::THREADS)
    k_ctrl_cc(Dev d, uint32_t n_steps) {
  using C = CtrlCc<E, H, NE, RE>;
  constexpr int OBS = E::OBS, NA = E::NA, RU = C::RU;
  constexpr bool ACRO = NA == 3;
  extern __shared__ float4 smem4[];
  float *sm = (float *)smem4;
  const int tid = threadIdx.x;
  const int ug = tid % kUG, eg = tid / kUG;

  // Stage the policy: W1, b1, W2 (rounded to BF16), b2, W3, b3 from the FP32
  // parameters [W1 (OBS x H) | b1 | W2 (H x H) | b2 | W3 (H x NA) | b3].
  {
    const float *p = d.params;
    for (int i = tid; i < OBS * H + H; i += C::THREADS) sm[C::S_W1 + i] = p[i];
    const float4 *W2 = (const float4 *)(p + OBS * H + H);  // 16-byte aligned: OBS H + H = 4 k
#pragma unroll 4
    for (int i = tid; i < H * H / 4; i += C::THREADS) {
      const float4 q = __ldg(W2 + i);
      *(float4 *)(sm + C::S_W2 + 4 * i) =
          make_float4(tc::bf16_lo(tc::pack_bf16x2(q.x, 0.f)), tc::bf16_lo(tc::pack_bf16x2(q.y, 0.f)),
                      tc::bf16_lo(tc::pack_bf16x2(q.z, 0.f)), tc::bf16_lo(tc::pack_bf16x2(q.w, 0.f)));
    }
    const float *b2 = p + OBS * H + H + H * H, *W3 = b2 + H, *b3 = W3 + H * NA;
    for (int i = tid; i < H; i += C::THREADS) sm[C::S_B2 + i] = b2[i];
    for (int i = tid; i < H * 4; i += C::THREADS) {
      const int u = i / 4, a = i % 4;
      sm[C::S_W3 + i] = a < NA ? W3[u * NA + a] : 0.f;
    }
    if (tid < 4) sm[C::S_B3 + tid] = tid < NA ? b3[tid] : 0.f;
  }

  const uint64_t k0 = d.k[0];
  const uint32_t R = d.ring_steps, N = d.n_envs;
  const uint32_t row0 = (uint32_t)(k0 % R);
  const int n_tiles = (int)((N + NE - 1) / NE);
  float *xo = sm + C::S_XO, *h1s = sm + C::S_H1, *lg = sm + C::S_LG, *sc = sm + C::S_SC;
  float *us = sm + C::S_U;
  uint32_t *rrs = (uint32_t *)(sm + C::S_RR);

  for (int tile = (int)blockIdx.x; tile < n_tiles; tile += (int)gridDim.x) {
    const uint32_t base = (uint32_t)tile * NE;
    const uint32_t e = base + (uint32_t)tid;
    const bool lane_env = tid < NE;
    const bool valid = lane_env && e < N;
    Lane<E> s;
    __syncthreads();  // the previous tile's last reads of xo / draws are done
    if (valid) lane_load(d, s, e);
    if (lane_env) lane_observe(s, xo + tid, NE);
    draw_lanes(d, tid, NE, base, (uint32_t)k0, us, rrs);

    uint32_t row = row0;
    for (uint32_t j = 0; j < n_steps; ++j) {
      const uint32_t k = (uint32_t)(k0 + j);
      const int par = (int)(j & 1u);
      __syncthreads();  // observations and draws of step k ready; last step's logits read
      // ---- P2: layer 1 and act 1 (h1 = tanh(z1) on the packed BF16 form)
      {
        float ov[RE][OBS];
#pragma unroll
        for (int r = 0; r < RE; ++r)
#pragma unroll
          for (int i = 0; i < OBS; ++i) ov[r][i] = xo[i * NE + eg * RE + r];
#pragma unroll
        for (int c = 0; c < RU; c += 4) {
          const int u0 = ug * RU + c;
          const float4 b = *(const float4 *)(sm + C::S_B1 + u0);
          float4 wv[OBS];
#pragma unroll
          for (int i = 0; i < OBS; ++i) wv[i] = *(const float4 *)(sm + C::S_W1 + i * H + u0);
#pragma unroll
          for (int r = 0; r < RE; ++r) {
            float z0 = b.x, z1 = b.y, z2 = b.z, z3 = b.w;
#pragma unroll
            for (int i = 0; i < OBS; ++i) {
              z0 = __fmaf_rn(ov[r][i], wv[i].x, z0);
              z1 = __fmaf_rn(ov[r][i], wv[i].y, z1);
              z2 = __fmaf_rn(ov[r][i], wv[i].z, z2);
              z3 = __fmaf_rn(ov[r][i], wv[i].w, z3);
            }
            const uint32_t t01 = tc::tanh_bf16x2(tc::pack_bf16x2(z0, z1));
            const uint32_t t23 = tc::tanh_bf16x2(tc::pack_bf16x2(z2, z3));
            *(float4 *)(h1s + (eg * RE + r) * C::HP + u0) =
                make_float4(tc::bf16_lo(t01), tc::bf16_hi(t01), tc::bf16_lo(t23), tc::bf16_hi(t23));
          }
        }
      }
      __syncthreads();  // h1 complete
      // ---- P3: layer 2, act 2, layer-3 partials
      float pth, pw;
      draw_lane_state<E>(tid, NE, xo, pth, pw);
      {
        // z2 = (b2 + sum_{k < H/2} h1_k W2_k) + sum_{k >= H/2} h1_k W2_k: two
        // chains in k order, added at the end
        float acc[RE][RU], acc2[RE][RU];
#pragma unroll
        for (int c = 0; c < RU; c += 4) {
          const float4 b = *(const float4 *)(sm + C::S_B2 + ug * RU + c);
#pragma unroll
          for (int r = 0; r < RE; ++r) {
            acc[r][c] = b.x;
            acc[r][c + 1] = b.y;
            acc[r][c + 2] = b.z;
            acc[r][c + 3] = b.w;
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) acc2[r][c + cc] = 0.f;
          }
        }
        const float *w2 = sm + C::S_W2 + ug * RU;
        const float *hr = h1s + eg * RE * C::HP;
        auto chain = [&](float (&a)[RE][RU], int k4) {
          float4 hv[RE];
#pragma unroll
          for (int r = 0; r < RE; ++r) hv[r] = *(const float4 *)(hr + r * C::HP + k4);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            float wk[RU];
#pragma unroll
            for (int c = 0; c < RU; c += 4) {
              const float4 q = *(const float4 *)(w2 + (k4 + kk) * H + c);
              wk[c] = q.x;
              wk[c + 1] = q.y;
              wk[c + 2] = q.z;
              wk[c + 3] = q.w;
            }
#pragma unroll
            for (int r = 0; r < RE; ++r) {
              const float hk = kk == 0 ? hv[r].x : kk == 1 ? hv[r].y : kk == 2 ? hv[r].z : hv[r].w;
#pragma unroll
              for (int c = 0; c < RU; ++c) a[r][c] = __fmaf_rn(hk, wk[c], a[r][c]);
            }
          }
        };
#pragma unroll 2
        for (int k4 = 0; k4 < H / 2; k4 += 4) {
          chain(acc, k4);
          chain(acc2, k4 + H / 2);
        }
#pragma unroll
        for (int r = 0; r < RE; ++r)
#pragma unroll
          for (int c = 0; c < RU; ++c) acc[r][c] = acc[r][c] + acc2[r][c];
        // h2 = tanh(z2) (FP32) and this thread's layer-3 partial sums, units in order
        float pl[RE][NA];
#pragma unroll
        for (int r = 0; r < RE; ++r)
#pragma unroll
          for (int a = 0; a < NA; ++a) pl[r][a] = 0.f;
#pragma unroll
        for (int c = 0; c < RU; ++c) {
          const float4 w3 = *(const float4 *)(sm + C::S_W3 + (ug * RU + c) * 4);
#pragma unroll
          for (int r = 0; r < RE; ++r) {
            const float h2 = tc::tanh_fast(acc[r][c]);
            pl[r][0] = __fmaf_rn(h2, w3.x, pl[r][0]);
            pl[r][1] = __fmaf_rn(h2, w3.y, pl[r][1]);
            if (NA == 3) pl[r][NA - 1] = __fmaf_rn(h2, w3.z, pl[r][NA - 1]);
          }
        }
        // butterfly over the 16 unit groups (lanes of one half-warp): every lane
        // ends with the same sum, since each level adds the same two values
#pragma unroll
        for (int m = 1; m < kUG; m <<= 1)
#pragma unroll
          for (int r = 0; r < RE; ++r)
#pragma unroll
            for (int a = 0; a < NA; ++a)
              pl[r][a] += __shfl_xor_sync(0xffffffffu, pl[r][a], m);
        if (ug == 0)
#pragma unroll
          for (int r = 0; r < RE; ++r)
#pragma unroll
            for (int a = 0; a < NA; ++a) lg[a * NE + eg * RE + r] = pl[r][a];
      }
      __syncthreads();  // logits complete
      // ---- P4: sampling, env step, records (env lanes); next step's draws
      if (lane_env) {
        float sin_th, cos_th;
        lane_trig(s, sc + par * 2 * NE, NE, tid, sin_th, cos_th);
        const float l0 = lg[tid] + sm[C::S_B3], l1v = lg[NE + tid] + sm[C::S_B3 + 1];
        const float l2 = ACRO ? lg[2 * NE + tid] + sm[C::S_B3 + 2] : 0.f;
        lane_step(d, s, l0, l1v, l2, us[par * NE + tid], rrs + par * 4 * NE + tid, NE, sin_th,
                  cos_th, valid, e, row);
        lane_observe(s, xo + tid, NE);
      } else if (j + 1 < n_steps) {
        const int np = par ^ 1;
        draw_lanes(d, tid, NE, base, k + 1, us + np * NE, rrs + np * 4 * NE, !ACRO, pth, pw,
                   sc + np * 2 * NE);
      }
      row = (row + 1 == R) ? 0 : row + 1;
    }
    if (valid) lane_store(d, s, e);
  }
}

// ------------------------------------------------------------ unit per thread
template <typename E, int NE>
struct CtrlCu {
  static constexpr int H = 64;  // four units per layer-3 group (H / 16)
  static constexpr int THREADS = H * NE;
  static constexpr int HP = H + 4;
  static constexpr int S_XO = 0;                       // [OBS][NE]
  static constexpr int S_H1 = 4 * ((E::OBS * NE + 3) / 4);  // [NE][HP]
  static constexpr int S_PT = S_H1 + NE * HP;          // [NA][NE][2] per-warp partial sums
  static constexpr int S_U = S_PT + 3 * NE * 2;        // [2][NE]
  static constexpr int S_RR = S_U + 2 * NE;            // [2][4][NE]
  static constexpr int S_SC = S_RR + 8 * NE;           // [2][2][NE] predicted sin, cos
  static constexpr int FLOATS = S_SC + 4 * NE;
  static constexpr int SMEM = FLOATS * 4;
  static_assert(S_H1 % 4 == 0 && HP % 4 == 0, "alignment");
  static_assert(NE <= 32 && draw_lane0(NE) + 2 * NE <= THREADS, "env lanes, then draw lanes");
};

template <typename E, int NE>
__global__ void __launch_bounds__(CtrlCu<E, NE>::THREADS)
    k_ctrl_cu(Dev d, uint32_t n_steps) {
  using C = CtrlCu<E, NE>;
  constexpr int OBS = E::OBS, NA = E::NA, H = C::H;
  constexpr bool ACRO = NA == 3;
  extern __shared__ float4 smem4[];
  float *sm = (float *)smem4;
  const int tid = threadIdx.x;
  const int q = tid / H, u = tid % H, lane = tid & 31;

  // this thread's unit: W1 column, b1, W2 column (BF16-rounded), b2, and the W3
  // rows of the four units of its layer-3 group
  const float *p = d.params;
  float w1c[OBS], w2c[H], w3g[4][NA];
#pragma unroll
  for (int i = 0; i < OBS; ++i) w1c[i] = p[i * H + u];
  const float b1u = p[OBS * H + u];
  const float *W2 = p + OBS * H + H;
#pragma unroll
  for (int k = 0; k < H; ++k) w2c[k] = tc::bf16_lo(tc::pack_bf16x2(__ldg(W2 + k * H + u), 0.f));
  const float *b2 = W2 + H * H, *W3 = b2 + H, *b3 = W3 + H * NA;
  const float b2u = b2[u];
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int a = 0; a < NA; ++a) w3g[c][a] = W3[((u & ~3) + c) * NA + a];
  const float b30 = b3[0], b31 = b3[1], b32 = NA == 3 ? b3[NA - 1] : 0.f;

  const uint64_t k0 = d.k[0];
  const uint32_t R = d.ring_steps, N = d.n_envs;
  const uint32_t row0 = (uint32_t)(k0 % R);
  const int n_tiles = (int)((N + NE - 1) / NE);
  float *xo = sm + C::S_XO, *h1s = sm + C::S_H1, *pt = sm + C::S_PT, *sc = sm + C::S_SC;
  float *us = sm + C::S_U;
  uint32_t *rrs = (uint32_t *)(sm + C::S_RR);

  for (int tile = (int)blockIdx.x; tile < n_tiles; tile += (int)gridDim.x) {
    const uint32_t base = (uint32_t)tile * NE;
    const uint32_t e = base + (uint32_t)tid;
    const bool lane_env = tid < NE;
    const bool valid = lane_env && e < N;
    Lane<E> s;
    __syncthreads();
    if (valid) lane_load(d, s, e);
    if (lane_env) lane_observe(s, xo + tid, NE);
    draw_lanes(d, tid, NE, base, (uint32_t)k0, us, rrs);

    uint32_t row = row0;
    for (uint32_t j = 0; j < n_steps; ++j) {
      const uint32_t k = (uint32_t)(k0 + j);
      const int par = (int)(j & 1u);
      __syncthreads();  // observations and draws of step k ready
      // ---- P2: layer 1 and act 1 of unit u of env q
      {
        float z = b1u;
#pragma unroll
        for (int i = 0; i < OBS; ++i) z = __fmaf_rn(xo[i * NE + q], w1c[i], z);
        h1s[q * C::HP + u] = tc::bf16_lo(tc::tanh_bf16x2(tc::pack_bf16x2(z, 0.f)));
      }
      __syncthreads();  // h1 complete
      // ---- P3: layer 2 of unit u (two chains in k order: from b2 over the first
      // half of k, from zero over the second, added), act 2, layer-3 partials
      float pth, pw;
      draw_lane_state<E>(tid, NE, xo, pth, pw);
      {
        float za = b2u, zb = 0.f;
        const float *hr = h1s + q * C::HP;
#pragma unroll
        for (int k4 = 0; k4 < H / 2; k4 += 4) {
          const float4 ha = *(const float4 *)(hr + k4);
          const float4 hb = *(const float4 *)(hr + k4 + H / 2);
          za = __fmaf_rn(ha.x, w2c[k4], za);
          zb = __fmaf_rn(hb.x, w2c[k4 + H / 2], zb);
          za = __fmaf_rn(ha.y, w2c[k4 + 1], za);
          zb = __fmaf_rn(hb.y, w2c[k4 + H / 2 + 1], zb);
          za = __fmaf_rn(ha.z, w2c[k4 + 2], za);
          zb = __fmaf_rn(hb.z, w2c[k4 + H / 2 + 2], zb);
          za = __fmaf_rn(ha.w, w2c[k4 + 3], za);
          zb = __fmaf_rn(hb.w, w2c[k4 + H / 2 + 3], zb);
        }
        const float h2 = tc::tanh_fast(za + zb);
        // the group of units 4g .. 4g + 3 (four lanes of one warp): each of its
        // lanes forms the group's FMA chain over the four from zero
        float hg[4];
        hg[0] = h2;
#pragma unroll
        for (int c = 1; c < 4; ++c) hg[c] = __shfl_sync(0xffffffffu, h2, (lane & ~3) + c);
        float pa[NA];
#pragma unroll
        for (int a = 0; a < NA; ++a) pa[a] = 0.f;
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
          for (int a = 0; a < NA; ++a) pa[a] = __fmaf_rn(hg[c], w3g[c][a], pa[a]);
        // butterfly over the warp's eight groups (every lane of a group holds its
        // partial; partners g ^ 1, g ^ 2, g ^ 4 sit at lane distance 4, 8, 16)
#pragma unroll
        for (int m = 4; m < 32; m <<= 1)
#pragma unroll
          for (int a = 0; a < NA; ++a) pa[a] += __shfl_xor_sync(0xffffffffu, pa[a], m);
        if (lane == 0)
#pragma unroll
          for (int a = 0; a < NA; ++a) pt[(a * NE + q) * 2 + (u >> 5)] = pa[a];
      }
      __syncthreads();  // group partials complete
      // ---- P4: sampling, env step, records (env lanes); next step's draws
      if (lane_env) {
        float sin_th, cos_th;
        lane_trig(s, sc + par * 2 * NE, NE, tid, sin_th, cos_th);
        // the last butterfly level: the env's two warps (groups g and g ^ 8)
        const float l0 = (pt[tid * 2] + pt[tid * 2 + 1]) + b30;
        const float l1v = (pt[(NE + tid) * 2] + pt[(NE + tid) * 2 + 1]) + b31;
        const float l2 = ACRO ? (pt[(2 * NE + tid) * 2] + pt[(2 * NE + tid) * 2 + 1]) + b32 : 0.f;
        lane_step(d, s, l0, l1v, l2, us[par * NE + tid], rrs + par * 4 * NE + tid, NE, sin_th,
                  cos_th, valid, e, row);
        lane_observe(s, xo + tid, NE);
      } else if (j + 1 < n_steps) {
        const int np = par ^ 1;
        draw_lanes(d, tid, NE, base, k + 1, us + np * NE, rrs + np * 4 * NE, !ACRO, pth, pw,
                   sc + np * 2 * NE);
      }
      row = (row + 1 == R) ? 0 : row + 1;
    }
    if (valid) lane_store(d, s, e);
  }
}

// The dynamic shared-memory limit of one kernel, raised once per device; Tag
// makes the flags per kernel (the attribute call is idempotent, so a race on
// them is benign).
template <typename Tag, typename K>
cudaError_t set_smem_once(K kernel, int smem) {
  static bool attr_set[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && attr_set[dev]) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess && dev >= 0 && dev < 64) attr_set[dev] = true;
  return e;
}

int cc_grid(uint32_t n_envs, int ne) {
  const int n_tiles = (int)((n_envs + (uint32_t)ne - 1) / (uint32_t)ne);
  return n_tiles < 65535 ? n_tiles : 65535;
}

template <typename E, int H, int NE, int RE>
cudaError_t run_cc(const Dev &d, uint32_t n_steps, cudaStream_t st) {
  using C = CtrlCc<E, H, NE, RE>;
  cudaError_t e = set_smem_once<C>(k_ctrl_cc<E, H, NE, RE>, C::SMEM);
  if (e != cudaSuccess) return e;
  k_ctrl_cc<E, H, NE, RE><<<cc_grid(d.n_envs, NE), C::THREADS, C::SMEM, st>>>(d, n_steps);
  return cudaGetLastError();
}

template <typename E, int NE>
cudaError_t run_cu(const Dev &d, uint32_t n_steps, cudaStream_t st) {
  using C = CtrlCu<E, NE>;
  cudaError_t e = set_smem_once<C>(k_ctrl_cu<E, NE>, C::SMEM);
  if (e != cudaSuccess) return e;
  k_ctrl_cu<E, NE><<<cc_grid(d.n_envs, NE), C::THREADS, C::SMEM, st>>>(d, n_steps);
  return cudaGetLastError();
}

template <typename E, int H>
cudaError_t run_cc_h(const Dev &d, uint32_t n_steps, int ne, int tpe, cudaStream_t st) {
  switch (ne * 128 + tpe) {
    case 4 * 128 + 16: return run_cc<E, H, 4, 1>(d, n_steps, st);
    case 8 * 128 + 16: return run_cc<E, H, 8, 1>(d, n_steps, st);
    case 8 * 128 + 8: return run_cc<E, H, 8, 2>(d, n_steps, st);
    case 16 * 128 + 16: return run_cc<E, H, 16, 1>(d, n_steps, st);
    case 16 * 128 + 8: return run_cc<E, H, 16, 2>(d, n_steps, st);
    case 16 * 128 + 4: return run_cc<E, H, 16, 4>(d, n_steps, st);
    case 32 * 128 + 16: return run_cc<E, H, 32, 1>(d, n_steps, st);
    case 32 * 128 + 8: return run_cc<E, H, 32, 2>(d, n_steps, st);
    case 32 * 128 + 4: return run_cc<E, H, 32, 4>(d, n_steps, st);
    default: break;
  }
  if constexpr (H == 64) {
    switch (ne * 128 + tpe) {
      case 1 * 128 + 64: return run_cu<E, 1>(d, n_steps, st);
      case 2 * 128 + 64: return run_cu<E, 2>(d, n_steps, st);
      case 4 * 128 + 64: return run_cu<E, 4>(d, n_steps, st);
      case 8 * 128 + 64: return run_cu<E, 8>(d, n_steps, st);
      default: break;
    }
  }
  return cudaErrorInvalidValue;
}

template <typename E>
cudaError_t run_cc_env(const Dev &d, uint32_t n_steps, int ne, int tpe, cudaStream_t st) {
  if (d.pol.w[1] == 64) return run_cc_h<E, 64>(d, n_steps, ne, tpe, st);
  return run_cc_h<E, 128>(d, n_steps, ne, tpe, st);
}

}  // namespace

bool control_cc_supported(const PolicyShape &sh) {
  const bool cart = sh.w[0] == CcCart::OBS && sh.w[3] == CcCart::NA;
  const bool acro = sh.w[0] == CcAcro::OBS && sh.w[3] == CcAcro::NA;
  return (cart || acro) && sh.w[1] == sh.w[2] && (sh.w[1] == 64 || sh.w[1] == 128);
}

bool control_cc_tile_ok(const PolicyShape &sh, int envs_per_cta, int threads_per_env) {
  const int ne = envs_per_cta, tpe = threads_per_env;
  if (tpe == 64)  // unit per thread: hidden width 64, 64 .. 512 threads
    return sh.w[1] == 64 && (ne == 1 || ne == 2 || ne == 4 || ne == 8);
  if (ne != 4 && ne != 8 && ne != 16 && ne != 32) return false;
  if (tpe != 4 && tpe != 8 && tpe != 16) return false;
  const int threads = ne * tpe;
  return threads >= 64 && threads <= 512;
}

cudaError_t launch_control_cc(const Dev &d, uint32_t n_steps, int envs_per_cta, int threads_per_env,
                              cudaStream_t st) {
  if (!control_cc_supported(d.pol) || !control_cc_tile_ok(d.pol, envs_per_cta, threads_per_env))
    return cudaErrorInvalidValue;
  if (d.pol.w[3] == CcAcro::NA)
    return run_cc_env<CcAcro>(d, n_steps, envs_per_cta, threads_per_env, st);
  return run_cc_env<CcCart>(d, n_steps, envs_per_cta, threads_per_env, st);
}

}  // namespace ws
