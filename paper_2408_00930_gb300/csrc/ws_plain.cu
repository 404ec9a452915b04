// ws_plain.cu -- parameter init (S0), full reset, the plain FP32 per-sub-step
// kernels (S1-S6: observe/store, policy layers, sampling, env steps with
// auto-reset) and the discounted-return scan (S7).
//
// Every kernel here is one launch per sub-step per step: this is the
// one-launch-per-step FP32 baseline (and, captured in a CUDA graph, the
// batched-FP32 path).  The fused tensor-core path lives in ws_control_tc.cu.
#include <math.h>

#include "ws_acrobot.cuh"
#include "ws_kernels.cuh"

namespace ws {

namespace {

__device__ __forceinline__ uint64_t step_k(const Dev &d, uint32_t off) { return d.k[0] + off; }
__device__ __forceinline__ uint32_t ring_row(const Dev &d, uint64_t k) {
  return (uint32_t)(k % d.ring_steps);
}
__device__ __forceinline__ uint32_t word(const uint4 &r, int i) {
  return i == 0 ? r.x : i == 1 ? r.y : i == 2 ? r.z : r.w;
}

// ---------------------------------------------------------------- S0 init
// Policy weights and biases of layer l: U(-1/sqrt(n_in), 1/sqrt(n_in)); element
// i takes word i&3 of Philox(i>>2, l, policy, POLICY_INIT) under param_seed.
__global__ void k_init_policy(float *p, PolicyShape sh, uint64_t seed, uint32_t pid) {
  const size_t total = sh.count();
  for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += (size_t)gridDim.x * blockDim.x) {
    int l = 0;
    size_t base = 0;
    while (l < kMaxLayers - 1) {
      const size_t c = (size_t)sh.w[l] * sh.w[l + 1] + sh.w[l + 1];
      if (g < base + c) break;
      base += c;
      ++l;
    }
    const size_t i = g - base;
    const float bound = __fdiv_rn(1.0f, __fsqrt_rn((float)sh.w[l]));
    const uint4 r = draw(seed, (uint32_t)(i >> 2), (uint32_t)l, pid, kTagPolicyInit, 0);
    p[g] = uniform(word(r, (int)(i & 3)), -bound, bound);
  }
}

// Landscape: centre coordinates U[-3,3] (4 per draw, subs 0..), width
// exp(0.3 z) and amplitude z from sub 64 (cos branches of the two pairs).
__global__ void k_init_landscape(float *c, float *wd, float *am, int D, int M, uint64_t seed) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  for (int j = 0; j < D; j += 4) {
    const uint4 r = draw(seed, (uint32_t)m, 0, 0, kTagLandscapeInit, (uint32_t)(j >> 2));
    for (int i = 0; i < 4 && j + i < D; ++i) c[(size_t)m * D + j + i] = uniform(word(r, i), -3.0f, 3.0f);
  }
  const uint4 r = draw(seed, (uint32_t)m, 0, 0, kTagLandscapeInit, 64);
  const float z0 = box_muller(r.x, r.y).x;
  const float z2 = box_muller(r.z, r.w).x;
  wd[m] = expf(0.3f * z0);
  am[m] = z2;
}

// |c_m|^2 and 1/(2 w_m^2) for the plain energy loop.
__global__ void k_landscape_derive(Dev d) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= (int)d.n_gauss) return;
  float s = 0.f;
  for (int j = 0; j < (int)d.dim; ++j) {
    const float v = d.centres[(size_t)m * d.dim + j];
    s = fmaf(v, v, s);
  }
  d.cnorm[m] = s;
  const float w = d.widths[m];
  d.coef[m] = 0.5f / (w * w);
}

// ---------------------------------------------------------------- resets
__device__ void control_reset_env(const Dev &d, uint32_t k, uint32_t e) {
  const uint4 r = draw(d.seed, k, d.env_base + e, 0, kTagReset, 0);
  d.s[0 * d.n_envs + e] = uniform(r.x, -0.05f, 0.05f);
  d.s[1 * d.n_envs + e] = uniform(r.y, -0.05f, 0.05f);
  d.s[2 * d.n_envs + e] = uniform(r.z, -0.05f, 0.05f);
  d.s[3 * d.n_envs + e] = uniform(r.w, -0.05f, 0.05f);
}

// Acrobot: (th1, th2, w1, w2) from the four words of RESET(k, env), U(-0.1, 0.1).
__device__ void acrobot_reset_env(const Dev &d, uint32_t k, uint32_t e) {
  const uint4 r = draw(d.seed, k, d.env_base + e, 0, kTagReset, 0);
  d.s[0 * d.n_envs + e] = uniform(r.x, -0.1f, 0.1f);
  d.s[1 * d.n_envs + e] = uniform(r.y, -0.1f, 0.1f);
  d.s[2 * d.n_envs + e] = uniform(r.z, -0.1f, 0.1f);
  d.s[3 * d.n_envs + e] = uniform(r.w, -0.1f, 0.1f);
}

// Economy agent redraw: wealth 1e4 + (64-bit word) mod 990001, features N(0,1).
__device__ void econ_reset_agent(const Dev &d, uint32_t k, uint32_t env, uint32_t agent,
                                 uint32_t slot) {
  uint4 r = draw(d.seed, k, d.env_base + env, agent, kTagReset, 0);
  const uint64_t big = ((uint64_t)r.y << 32) | (uint64_t)r.x;
  d.wealth[slot] = 10000 + (int64_t)(big % 990001ull);
  for (int j = 0; j < 4; ++j) {
    r = draw(d.seed, k, d.env_base + env, agent, kTagReset, 1 + j);
    const float2 a = box_muller(r.x, r.y), b = box_muller(r.z, r.w);
    d.feat[(size_t)(4 * j + 0) * d.n_agent_slots + slot] = a.x;
    d.feat[(size_t)(4 * j + 1) * d.n_agent_slots + slot] = a.y;
    d.feat[(size_t)(4 * j + 2) * d.n_agent_slots + slot] = b.x;
    d.feat[(size_t)(4 * j + 3) * d.n_agent_slots + slot] = b.y;
  }
}

__device__ void landscape_reset_env(const Dev &d, uint32_t k, uint32_t e) {
  for (int j = 0; j < (int)d.dim; j += 4) {
    const uint4 r = draw(d.seed, k, d.env_base + e, 0, kTagReset, (uint32_t)(j >> 2));
    for (int i = 0; i < 4 && j + i < (int)d.dim; ++i)
      d.s[(size_t)(j + i) * d.n_envs + e] = uniform(word(r, i), -3.0f, 3.0f);
  }
  d.needs_energy[e] = 1;
}

__global__ void k_reset(Dev d) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (d.env == WS_ENV_CONTROL) {
    if (i < d.n_envs) {
      control_reset_env(d, kStepInit, i);
      d.t[i] = 0;
    }
  } else if (d.env == WS_ENV_ACROBOT) {
    if (i < d.n_envs) {
      acrobot_reset_env(d, kStepInit, i);
      d.t[i] = 0;
    }
  } else if (d.env == WS_ENV_ECONOMY) {
    if (i < d.n_agent_slots) {
      const uint32_t env = (uint32_t)d.slot_env[i];
      econ_reset_agent(d, kStepInit, env, i - (uint32_t)d.agent_off[env], i);
    }
    if (i < d.n_envs) d.t[i] = 0;
  } else {
    if (i < d.n_envs) {
      landscape_reset_env(d, kStepInit, i);
      d.t[i] = 0;
    }
  }
}

// -------------------------------------------------------- S2 policy layers
// Y[M][N] = act(X W + b), X addressed as X[r * ldr + c * ldc] (SoA env state
// or a row-major activation), W [K][N] row-major.  64x64 tiles, 4x4 per
// thread, K staged 16 at a time through shared memory.
constexpr int kBM = 64, kBN = 64, kBK = 16, kTM = 4, kTN = 4;
constexpr int kDenseThreads = (kBM / kTM) * (kBN / kTN);

__global__ __launch_bounds__(kDenseThreads) void k_dense_fp32(const float *__restrict__ X,
                                                               long ldr, long ldc,
                                                               const float *__restrict__ W,
                                                               const float *__restrict__ b,
                                                               float *__restrict__ Y, int M, int K,
                                                               int N, int act) {
  __shared__ float As[kBK][kBM + 4];
  __shared__ float Ws[kBK][kBN + 4];
  const int tid = threadIdx.x;
  const int tx = tid % (kBN / kTN), ty = tid / (kBN / kTN);
  const long row0 = (long)blockIdx.x * kBM;
  const int col0 = blockIdx.y * kBN;
  float acc[kTM][kTN];
#pragma unroll
  for (int i = 0; i < kTM; ++i)
#pragma unroll
    for (int j = 0; j < kTN; ++j) acc[i][j] = 0.f;
  for (int k0 = 0; k0 < K; k0 += kBK) {
    if (ldc == 1) {  // row-major rows: walk k fastest
      for (int idx = tid; idx < kBM * kBK; idx += kDenseThreads) {
        const int kk = idx % kBK, r = idx / kBK;
        const long gr = row0 + r;
        const int gk = k0 + kk;
        As[kk][r] = (gr < M && gk < K) ? X[gr * ldr + gk] : 0.f;
      }
    } else {  // SoA: walk rows fastest
      for (int idx = tid; idx < kBM * kBK; idx += kDenseThreads) {
        const int r = idx % kBM, kk = idx / kBM;
        const long gr = row0 + r;
        const int gk = k0 + kk;
        As[kk][r] = (gr < M && gk < K) ? X[gr * ldr + (long)gk * ldc] : 0.f;
      }
    }
    for (int idx = tid; idx < kBK * kBN; idx += kDenseThreads) {
      const int c = idx % kBN, kk = idx / kBN;
      const int gc = col0 + c, gk = k0 + kk;
      Ws[kk][c] = (gc < N && gk < K) ? W[(long)gk * N + gc] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kBK; ++kk) {
      float a[kTM], w[kTN];
#pragma unroll
      for (int i = 0; i < kTM; ++i) a[i] = As[kk][ty * kTM + i];
#pragma unroll
      for (int j = 0; j < kTN; ++j) w[j] = Ws[kk][tx * kTN + j];
#pragma unroll
      for (int i = 0; i < kTM; ++i)
#pragma unroll
        for (int j = 0; j < kTN; ++j) acc[i][j] = fmaf(a[i], w[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < kTM; ++i) {
    const long r = row0 + ty * kTM + i;
    if (r >= M) continue;
#pragma unroll
    for (int j = 0; j < kTN; ++j) {
      const int c = col0 + tx * kTN + j;
      if (c >= N) continue;
      const float v = acc[i][j] + b[c];
      Y[r * N + c] = act ? tanhf(v) : v;
    }
  }
}

void dense(const float *X, long ldr, long ldc, const float *W, const float *b, float *Y, int M,
           int K, int N, int act, cudaStream_t st) {
  if (M <= 0) return;
  dim3 grid((unsigned)((M + kBM - 1) / kBM), (unsigned)((N + kBN - 1) / kBN));
  k_dense_fp32<<<grid, kDenseThreads, 0, st>>>(X, ldr, ldc, W, b, Y, M, K, N, act);
}

// Three layers: tanh, tanh, linear.  Paper App. B: inference runs on the
// policy held in global memory, referenced by every block.
void mlp3(const float *X, long ldr, long ldc, const float *params, const PolicyShape &sh,
          float *h0, float *h1, float *out, int M, cudaStream_t st) {
  const float *W0 = params + sh.layer_offset(0);
  const float *W1 = params + sh.layer_offset(1);
  const float *W2 = params + sh.layer_offset(2);
  dense(X, ldr, ldc, W0, W0 + (size_t)sh.w[0] * sh.w[1], h0, M, sh.w[0], sh.w[1], 1, st);
  dense(h0, sh.w[1], 1, W1, W1 + (size_t)sh.w[1] * sh.w[2], h1, M, sh.w[1], sh.w[2], 1, st);
  dense(h1, sh.w[2], 1, W2, W2 + (size_t)sh.w[2] * sh.w[3], out, M, sh.w[2], sh.w[3], 0, st);
}

// BF16 tensor-core variant: hidden activations in BF16 row-major, logits FP32.
void tc_mlp3(const Dev &d, const float *X, long ldr, long ldc, const PolicyShape &sh, int pid,
             void *h0, void *h1, float *out, long M, cudaStream_t st) {
  launch_dense_tc(X, ldr, ldc, 0, sh.w[0], d.pk[pid][0], sh.w[1], h0, 1, 1, M, d.err, st);
  launch_dense_tc(h0, 0, 0, 1, sh.w[1], d.pk[pid][1], sh.w[2], h1, 1, 1, M, d.err, st);
  launch_dense_tc(h1, 0, 0, 1, sh.w[2], d.pk[pid][2], sh.w[3], out, 0, 0, M, d.err, st);
}

void policy(const Dev &d, const float *X, long ldr, long ldc, const float *params,
            const PolicyShape &sh, int pid, float *h0, float *h1, float *out, int M,
            cudaStream_t st) {
  if (d.mlp3)
    launch_mlp3_tc(X, ldr, ldc, d.pk[pid][0], sh, out, M, d.err, st);
  else if (d.tc_mlp)
    tc_mlp3(d, X, ldr, ldc, sh, pid, h0, h1, out, M, st);
  else
    mlp3(X, ldr, ldc, params, sh, h0, h1, out, M, st);
}

// ------------------------------------------------- S1/S6 observation store
// ring.obs[row][j][slot_base + i] = src[j * ld + i]
__global__ void k_store_obs(Dev d, uint32_t off, const float *src, int dim, uint32_t n, size_t ld,
                            uint32_t slot_base) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t row = ring_row(d, step_k(d, off));
  float *dst = d.r_obs + (size_t)row * dim * d.n_slots;
  for (int j = 0; j < dim; ++j) dst[(size_t)j * d.n_slots + slot_base + i] = src[(size_t)j * ld + i];
}

// ------------------------------------------------------------ S3 sampling
// Categorical by inverse CDF in FP32: a = min{ i : u S < C_i }, C_i the
// running sum of exp(l - max), S the total; logp = (l_a - max) - log S.
// mode 0: control (env = row), 1: economy agents, 2: economy planner.
__global__ void k_sample_cat(Dev d, uint32_t off, const float *logits, int n_cls, int mode,
                             uint32_t n_rows, uint32_t slot_base) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_rows) return;
  const uint64_t k = step_k(d, off);
  uint32_t env = i, agent = 0;
  if (mode == 1) {
    env = (uint32_t)d.slot_env[i];
    agent = i - (uint32_t)d.agent_off[env];
  } else if (mode == 2) {
    agent = kPlannerId;
  }
  const float u = u01(draw(d.seed, (uint32_t)k, d.env_base + env, agent, kTagAction, 0).x);
  const float *l = logits + (size_t)i * n_cls;
  float m = l[0];
  for (int c = 1; c < n_cls; ++c) m = fmaxf(m, l[c]);
  float S = 0.f;
  for (int c = 0; c < n_cls; ++c) S += expf(l[c] - m);
  const float thr = u * S;
  float C = 0.f;
  int a = n_cls - 1;
  for (int c = 0; c < n_cls; ++c) {
    C += expf(l[c] - m);
    if (thr < C) {
      a = c;
      break;
    }
  }
  const uint32_t row = ring_row(d, k);
  const size_t o = (size_t)row * d.n_slots + slot_base + i;
  ((int32_t *)d.r_act)[o] = a;
  d.r_logp[o] = (l[a] - m) - logf(S);
  if (d.r_pout) {  // the logits this draw read (a planner's rows past its 10 are zero)
    float *po = d.r_pout + (size_t)row * d.n_out * d.n_slots + slot_base + i;
    for (int c = 0; c < (int)d.n_out; ++c) po[(size_t)c * d.n_slots] = c < n_cls ? l[c] : 0.f;
  }
}

// Diagonal Gaussian head: mean out[0:D], log sigma clamp(out[D:2D], -5, 2);
// dx = clip(mean + sigma z, +-clip); logp of the unclipped sample.
__global__ void k_sample_gauss(Dev d, uint32_t off) {
  const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d.n_envs) return;
  const uint64_t k = step_k(d, off);
  const uint32_t row = ring_row(d, k);
  const int D = (int)d.dim;
  const float *o = d.out + (size_t)e * 2 * D;
  float *act = (float *)d.r_act + (size_t)row * D * d.n_slots;
  float lp = 0.f;
  const float half_log_2pi = 0.91893853320467274f;
  for (int j = 0; j < D; j += 4) {
    const uint4 r = draw(d.seed, (uint32_t)k, d.env_base + e, 0, kTagAction, (uint32_t)(j >> 2));
    const float2 p = box_muller(r.x, r.y), q = box_muller(r.z, r.w);
    const float z4[4] = {p.x, p.y, q.x, q.y};
    for (int i = 0; i < 4 && j + i < D; ++i) {
      const float z = z4[i];
      const float ls = fminf(fmaxf(o[D + j + i], -5.0f), 2.0f);
      const float smp = o[j + i] + expf(ls) * z;
      act[(size_t)(j + i) * d.n_slots + e] = fminf(fmaxf(smp, -d.step_clip), d.step_clip);
      lp += -0.5f * z * z - ls - half_log_2pi;
    }
  }
  d.r_logp[(size_t)row * d.n_slots + e] = lp;
  if (d.r_pout) {
    float *po = d.r_pout + (size_t)row * 2 * D * d.n_slots + e;
    for (int c = 0; c < 2 * D; ++c) po[(size_t)c * d.n_slots] = o[c];
  }
}

// ----------------------------------------------------- S4/S5 control env
__global__ void k_control_step(Dev d, uint32_t off) {
  const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d.n_envs) return;
  const uint64_t k = step_k(d, off);
  const uint32_t row = ring_row(d, k);
  const size_t o = (size_t)row * d.n_slots + e;
  const int a = ((const int32_t *)d.r_act)[o];
  const float x = d.s[e], v = d.s[d.n_envs + e], th = d.s[2 * d.n_envs + e],
              w = d.s[3 * d.n_envs + e];
  const float u = a ? 10.0f : -10.0f;
  const float xacc = u - 0.5f * x - 0.1f * v;
  const float thacc = 9.8f * sinf(th) - 0.3f * cosf(th) * u;
  const float x2 = x + 0.02f * v, v2 = v + 0.02f * xacc;
  const float th2 = th + 0.02f * w, w2 = w + 0.02f * thacc;
  const int t2 = d.t[e] + 1;
  const bool done = fabsf(x2) > 2.4f || fabsf(th2) > 0.21f || t2 >= (int)d.episode_limit;
  d.r_rew[o] = 1.0f;
  d.r_done[o] = (uint8_t)done;
  if (done) {
    control_reset_env(d, (uint32_t)k, e);
    d.t[e] = 0;
  } else {
    d.s[e] = x2;
    d.s[d.n_envs + e] = v2;
    d.s[2 * d.n_envs + e] = th2;
    d.s[3 * d.n_envs + e] = w2;
    d.t[e] = t2;
  }
}

// ----------------------------------------------------- acrobot (S1, S4/S5)
// The physics (acro_step) is in ws_acrobot.cuh, shared with the fused kernel.
// Observation (cos th1, sin th1, cos th2, sin th2, w1, w2): into the policy's
// input [6][N] and the ring.
__global__ void k_acrobot_observe(Dev d, uint32_t off) {
  const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d.n_envs) return;
  const size_t N = d.n_envs;
  const float th1 = d.s[e], th2 = d.s[N + e];
  float o[kAcroObs];
  sincosf(th1, &o[1], &o[0]);
  sincosf(th2, &o[3], &o[2]);
  o[4] = d.s[2 * N + e];
  o[5] = d.s[3 * N + e];
  const uint32_t row = ring_row(d, step_k(d, off));
  float *dst = d.r_obs + (size_t)row * kAcroObs * d.n_slots + e;
#pragma unroll
  for (int j = 0; j < kAcroObs; ++j) {
    d.pobs[(size_t)j * N + e] = o[j];
    dst[(size_t)j * d.n_slots] = o[j];
  }
}

__global__ void k_acrobot_step(Dev d, uint32_t off) {
  const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d.n_envs) return;
  const uint64_t k = step_k(d, off);
  const uint32_t row = ring_row(d, k);
  const size_t o = (size_t)row * d.n_slots + e, N = d.n_envs;
  const int a = ((const int32_t *)d.r_act)[o];
  float s[4] = {d.s[e], d.s[N + e], d.s[2 * N + e], d.s[3 * N + e]};
  acro_step<false>(s, (float)(a - 1), 0.2f);
  const bool term = acro_terminal<false>(s);
  const int t2 = d.t[e] + 1;
  const bool done = term || t2 >= (int)d.episode_limit;
  d.r_rew[o] = term ? 0.0f : -1.0f;
  d.r_done[o] = (uint8_t)done;
  if (done) {
    acrobot_reset_env(d, (uint32_t)k, e);
    d.t[e] = 0;
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) d.s[i * N + e] = s[i];
    d.t[e] = t2;
  }
}

// -------------------------------------------------------- economy (S1..S5)
// Fixed-order block reduction: xor-shuffle tree inside each warp, then the
// warp partials summed in warp order by every thread (deterministic for floats).
template <typename T>
__device__ T block_sum(T v, T *sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  T r = sh[0];
  for (int i = 1; i < nw; ++i) r += sh[i];
  __syncthreads();
  return r;
}

constexpr int kEconThreads = 128;

// Per env: planner observation = mean agent features; store agent and
// planner observations and pre-step wealth (planner slot: env total).
__global__ __launch_bounds__(kEconThreads) void k_econ_observe(Dev d, uint32_t off) {
  __shared__ float shf[kEconF][kEconThreads / 32];
  __shared__ long long shi[kEconThreads / 32];
  const uint32_t e = blockIdx.x;
  const int a0 = d.agent_off[e], n = d.agent_off[e + 1] - a0;
  const uint32_t row = ring_row(d, step_k(d, off));
  float *obs = d.r_obs + (size_t)row * kEconF * d.n_slots;
  const uint32_t ps = d.n_agent_slots + e;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  float s[kEconF];
#pragma unroll
  for (int j = 0; j < kEconF; ++j) s[j] = 0.f;
  long long ws = 0;
  int64_t *wrec = d.r_wealth + (size_t)row * d.n_slots;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
#pragma unroll
    for (int j = 0; j < kEconF; ++j) {
      const float f = d.feat[(size_t)j * d.n_agent_slots + a0 + i];
      s[j] += f;
      obs[(size_t)j * d.n_slots + a0 + i] = f;
    }
    const int64_t w = d.wealth[a0 + i];
    wrec[a0 + i] = w;
    ws += w;
  }
#pragma unroll
  for (int j = 0; j < kEconF; ++j) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s[j] += __shfl_xor_sync(0xffffffffu, s[j], o);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ws += __shfl_xor_sync(0xffffffffu, ws, o);
  if (lane == 0) {
#pragma unroll
    for (int j = 0; j < kEconF; ++j) shf[j][wid] = s[j];
    shi[wid] = ws;
  }
  __syncthreads();
  if (threadIdx.x < kEconF) {
    const int j = threadIdx.x;
    float tot = shf[j][0];
    for (int q = 1; q < kEconThreads / 32; ++q) tot += shf[j][q];
    const float mean = tot / (float)n;
    d.pobs[(size_t)e * kEconF + j] = mean;
    obs[(size_t)j * d.n_slots + ps] = mean;
  }
  if (threadIdx.x == 32) {
    long long tot = shi[0];
    for (int q = 1; q < kEconThreads / 32; ++q) tot += shi[q];
    wrec[ps] = tot;
  }
}

// Transfers t_i = floor(w_i a_i / 400) from pre-step wealth to partner
// p_i = (i + 1 + floor(r (n-1) / 2^32)) mod n; integer atomics commute, so
// the result is exact and order-free.
__global__ void k_econ_transfer(Dev d, uint32_t off) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n_agent_slots) return;
  const uint64_t k = step_k(d, off);
  const uint32_t row = ring_row(d, k);
  const uint32_t env = (uint32_t)d.slot_env[i];
  const int a0 = d.agent_off[env], n = d.agent_off[env + 1] - a0;
  const uint32_t ai = i - (uint32_t)a0;
  const int64_t act = ((const int32_t *)d.r_act)[(size_t)row * d.n_slots + i];
  const int64_t w0 = d.r_wealth[(size_t)row * d.n_slots + i];
  const uint32_t r = draw(d.seed, (uint32_t)k, d.env_base + env, ai, kTagPartner, 0).x;
  const uint32_t p = (ai + 1u + bounded(r, (uint32_t)(n - 1))) % (uint32_t)n;
  const int64_t amt = (w0 * act) / 400;
  atomicAdd((unsigned long long *)&d.wealth[i], (unsigned long long)(-amt));
  atomicAdd((unsigned long long *)&d.wealth[a0 + p], (unsigned long long)amt);
  atomicAdd((unsigned long long *)&d.income[a0 + p], (unsigned long long)amt);
}

// Per env: tax on income, even redistribution (remainder to low indices),
// feature drift, rewards, planner reward (mean), done and auto-reset.
__global__ __launch_bounds__(kEconThreads) void k_econ_finish(Dev d, uint32_t off) {
  __shared__ float shf[kEconThreads / 32];
  __shared__ long long shi[kEconThreads / 32];
  const uint32_t e = blockIdx.x;
  const uint64_t k = step_k(d, off);
  const uint32_t row = ring_row(d, k);
  const int a0 = d.agent_off[e], n = d.agent_off[e + 1] - a0;
  const uint32_t ps = d.n_agent_slots + e;
  const size_t rbase = (size_t)row * d.n_slots;
  const int64_t tau = ((const int32_t *)d.r_act)[rbase + ps];
  long long tsum = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int64_t tax = (d.income[a0 + i] * tau) / 20;
    d.wealth[a0 + i] -= tax;
    tsum += tax;
  }
  const long long T = block_sum(tsum, shi);
  // floor(T / n) and T - n floor(T / n) in [0, n), for a pool of either sign
  int64_t share = T / n, rem = T % n;
  if (rem < 0) {
    rem += n;
    share -= 1;
  }
  const int t2 = d.t[e] + 1;
  const bool done = t2 >= (int)d.episode_limit;
  const float inv_ln_1e6 = 0.0723824136505f;
  float rsum = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const uint32_t s = (uint32_t)(a0 + i);
    const int64_t w2 = d.wealth[s] + share + (i < rem ? 1 : 0);
    d.wealth[s] = w2;
    d.income[s] = 0;
    const int a = ((const int32_t *)d.r_act)[rbase + s];
    const float drive = ((float)a - 9.5f) / 9.5f;
    for (int j = 0; j < kEconF - 1; ++j) {
      float *f = &d.feat[(size_t)j * d.n_agent_slots + s];
      *f = 0.95f * *f + 0.05f * ((j & 1) ? -drive : drive);
    }
    d.feat[(size_t)(kEconF - 1) * d.n_agent_slots + s] = logf((float)w2) * inv_ln_1e6;
    const float r = (float)(w2 - d.r_wealth[rbase + s]) / 1e4f - 1e-3f * (float)(a * a);
    d.r_rew[rbase + s] = r;
    d.r_done[rbase + s] = (uint8_t)done;
    rsum += r;
    if (done) econ_reset_agent(d, (uint32_t)k, e, (uint32_t)i, s);
  }
  const float rtot = block_sum(rsum, shf);
  if (threadIdx.x == 0) {
    d.r_rew[rbase + ps] = rtot / (float)n;
    d.r_done[rbase + ps] = (uint8_t)done;
    d.t[e] = done ? 0 : t2;
  }
}

// ------------------------------------------------------ landscape (S4/S5)
// Partial energies of E(y) = sum_m a_m exp(-|y - c_m|^2 / (2 w_m^2)) over the
// Gaussians of chunk blockIdx.y, in FP32 with Kahan compensation.
// mode 0: y = x + dx (the post-step candidate); mode 1: y = x, only for envs
// flagged needs_energy (after a reset).
constexpr int kEnergyThreads = 128, kEnergyTileM = 64;

__global__ __launch_bounds__(kEnergyThreads) void k_energy_partial(Dev d, uint32_t off, int mode) {
  extern __shared__ float sm[];
  const int D = (int)d.dim;
  float *ys = sm;                                  // [D][kEnergyThreads]
  float *cs = ys + (size_t)D * kEnergyThreads;     // [kEnergyTileM][D]
  float *as = cs + (size_t)kEnergyTileM * D;       // [kEnergyTileM]
  float *qs = as + kEnergyTileM;                   // [kEnergyTileM]
  const uint32_t e = blockIdx.x * kEnergyThreads + threadIdx.x;
  const bool valid = e < d.n_envs;
  bool want = valid && (mode == 0 || d.needs_energy[e]);
  if (!__syncthreads_or(want)) return;
  const uint32_t row = ring_row(d, step_k(d, off));
  const float *act = (const float *)d.r_act + (size_t)row * D * d.n_slots;
  for (int j = 0; j < D; ++j) {
    float y = 0.f;
    if (valid) {
      y = d.s[(size_t)j * d.n_envs + e];
      if (mode == 0) y = y + act[(size_t)j * d.n_slots + e];
    }
    ys[j * kEnergyThreads + threadIdx.x] = y;
  }
  const int M = (int)d.n_gauss;
  const int per = (M + kEnergyChunks - 1) / kEnergyChunks;
  const int m_lo = blockIdx.y * per, m_hi = min(M, m_lo + per);
  float sum = 0.f, comp = 0.f;
  for (int t0 = m_lo; t0 < m_hi; t0 += kEnergyTileM) {
    const int nt = min(kEnergyTileM, m_hi - t0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < nt * D; idx += kEnergyThreads) cs[idx] = d.centres[(size_t)t0 * D + idx];
    for (int idx = threadIdx.x; idx < nt; idx += kEnergyThreads) {
      as[idx] = d.amps[t0 + idx];
      qs[idx] = d.coef[t0 + idx];
    }
    __syncthreads();
    for (int m = 0; m < nt; ++m) {
      float d2 = 0.f;
      for (int j = 0; j < D; ++j) {
        const float df = ys[j * kEnergyThreads + threadIdx.x] - cs[m * D + j];
        d2 = fmaf(df, df, d2);
      }
      const float term = as[m] * expf(-d2 * qs[m]);
      const float yk = term - comp;
      const float tk = sum + yk;
      comp = (tk - sum) - yk;
      sum = tk;
    }
  }
  if (want) {
    d.epart[((size_t)blockIdx.y * 2 + 0) * d.n_envs + e] = sum;
    d.epart[((size_t)blockIdx.y * 2 + 1) * d.n_envs + e] = comp;
  }
}

__device__ float energy_combine(const Dev &d, uint32_t e) {
  float sum = 0.f, comp = 0.f;
  for (int c = 0; c < kEnergyChunks; ++c) {
    const float yk = d.epart[((size_t)c * 2) * d.n_envs + e] - comp;
    const float tk = sum + yk;
    comp = (tk - sum) - yk;
    sum = tk;
  }
  float lo = 0.f;
  for (int c = 0; c < kEnergyChunks; ++c) lo += d.epart[((size_t)c * 2 + 1) * d.n_envs + e];
  return sum - (comp + lo);
}

// x' = x + dx; E' and observed E' = E' + sigma N(0,1) (NOISE, sub 0); reward
// = Eobs(x) - Eobs(x'); done at the episode limit or when E' falls below the
// energy target (App. C: the episode ends in the product basin); reset
// redraws x (RESET).
__global__ void k_landscape_step(Dev d, uint32_t off) {
  const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d.n_envs) return;
  const uint64_t k = step_k(d, off);
  const uint32_t row = ring_row(d, k);
  const size_t o = (size_t)row * d.n_slots + e;
  const int D = (int)d.dim;
  const float *act = (const float *)d.r_act + (size_t)row * D * d.n_slots;
  const float E2 = energy_combine(d, e);
  const uint4 rn = draw(d.seed, (uint32_t)k, d.env_base + e, 0, kTagNoise, 0);
  const float eobs2 = E2 + d.noise_sigma * box_muller(rn.x, rn.y).x;
  d.r_energy[o] = E2;
  d.r_rew[o] = d.eobs[e] - eobs2;
  const int t2 = d.t[e] + 1;
  const bool done = t2 >= (int)d.episode_limit || E2 < d.energy_target;
  d.r_done[o] = (uint8_t)done;
  if (done) {
    landscape_reset_env(d, (uint32_t)k, e);
    d.t[e] = 0;
  } else {
    for (int j = 0; j < D; ++j) {
      float *x = &d.s[(size_t)j * d.n_envs + e];
      *x = *x + act[(size_t)j * d.n_slots + e];
    }
    d.eobs[e] = eobs2;
    d.t[e] = t2;
    d.needs_energy[e] = 0;
  }
}

// After a reset: observed energy of the fresh state (NOISE, sub 1), keyed by
// the step of the reset (or "step -1" for a full reset).
__global__ void k_landscape_reset_finish(Dev d, uint32_t off, int full_reset) {
  const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d.n_envs || !d.needs_energy[e]) return;
  const uint32_t kk = full_reset ? kStepInit : (uint32_t)step_k(d, off);
  const float E = energy_combine(d, e);
  const uint4 rn = draw(d.seed, kk, d.env_base + e, 0, kTagNoise, 1);
  d.eobs[e] = E + d.noise_sigma * box_muller(rn.x, rn.y).x;
  d.needs_energy[e] = 0;
}

size_t energy_smem(const Dev &d) {
  return sizeof(float) * ((size_t)d.dim * kEnergyThreads + (size_t)kEnergyTileM * d.dim + 2 * kEnergyTileM);
}

void landscape_energy(const Dev &d, uint32_t off, int mode, cudaStream_t st) {
  if (d.eimg) {  // BF16 path: hi/lo cross-term on the tensor cores
    launch_energy_tc(d, d.eimg, off, mode, st);
    return;
  }
  dim3 grid((d.n_envs + kEnergyThreads - 1) / kEnergyThreads, kEnergyChunks);
  k_energy_partial<<<grid, kEnergyThreads, energy_smem(d), st>>>(d, off, mode);
}

// ---------------------------------------------------------------- misc
__global__ void k_advance(Dev d, uint32_t n) {
  if (threadIdx.x == 0 && blockIdx.x == 0) d.k[0] += n;
}

// S7: G_t = r_t + gamma (1 - d_t) G_{t+1} over the last n rows, carried as a
// float-float pair (error-free TwoProduct / TwoSum with explicit roundings).
//
// The scan is HBM-bound (9 B per slot-step: reward and done read, return
// written) and each slot's steps are serial, so the bandwidth comes from the
// loads in flight: a thread owns V consecutive slots (V = 4 when the slot count
// keeps every ring row 16-byte aligned: one float4 of rewards and one word of
// four done flags per step) and loads the rewards and done flags of its next
// kRetU steps into registers before it scans the current kRetU.
constexpr int kRetU = 16;

// Branch-free (the done flag selects), so that a thread's V chains interleave.
__device__ __forceinline__ float ret_update(float r, bool dn, float g, float &hi, float &lo) {
  const float p_hi = __fmul_rn(g, hi);
  const float p_lo = __fadd_rn(__fmaf_rn(g, hi, -p_hi), __fmul_rn(g, lo));
  const float s_hi = __fadd_rn(r, p_hi);
  const float bb = __fsub_rn(s_hi, r);
  const float s_lo = __fadd_rn(__fsub_rn(r, __fsub_rn(s_hi, bb)), __fsub_rn(p_hi, bb));
  const float t_lo = __fadd_rn(s_lo, p_lo);
  const float n_hi = __fadd_rn(s_hi, t_lo);
  const float n_lo = __fsub_rn(t_lo, __fsub_rn(n_hi, s_hi));
  hi = dn ? r : n_hi;
  lo = dn ? 0.f : n_lo;
  return hi;
}

template <int V>
struct RetVec;
template <>
struct RetVec<1> {
  float r;
  uint32_t d;
  __device__ __forceinline__ void load(const float *rew, const uint8_t *done, size_t o) {
    r = __ldcs(rew + o);
    d = __ldcs(done + o);
  }
  __device__ __forceinline__ float at(int) const { return r; }
  __device__ __forceinline__ bool dn(int) const { return d != 0; }
  __device__ __forceinline__ static void store(float *ret, size_t o, const float (&g)[1]) {
    __stcs(ret + o, g[0]);
  }
};
template <>
struct RetVec<4> {
  float4 r;
  uint32_t d;  // the four done bytes
  __device__ __forceinline__ void load(const float *rew, const uint8_t *done, size_t o) {
    r = __ldcs((const float4 *)(rew + o));
    d = __ldcs((const unsigned int *)(done + o));
  }
  __device__ __forceinline__ float at(int v) const {
    return v == 0 ? r.x : v == 1 ? r.y : v == 2 ? r.z : r.w;
  }
  __device__ __forceinline__ bool dn(int v) const { return ((d >> (8 * v)) & 0xFFu) != 0; }
  __device__ __forceinline__ static void store(float *ret, size_t o, const float (&g)[4]) {
    __stcs((float4 *)(ret + o), make_float4(g[0], g[1], g[2], g[3]));
  }
};

template <int V>
__device__ __forceinline__ void ret_load(const float *__restrict__ rew,
                                         const uint8_t *__restrict__ done, size_t S, uint32_t R,
                                         size_t s, uint32_t row, uint32_t left,
                                         RetVec<V> (&b)[kRetU]) {
#pragma unroll
  for (int j = 0; j < kRetU; ++j) {
    if ((uint32_t)j < left) b[j].load(rew, done, (size_t)row * S + s);
    row = row == 0 ? R - 1 : row - 1;
  }
}

// Scans the kRetU steps held in b (the first `left` of them), newest first.
template <int V, bool FULL>
__device__ __forceinline__ void ret_scan_n(const RetVec<V> (&b)[kRetU], uint32_t left, float g,
                                           float (&hi)[V], float (&lo)[V],
                                           float *__restrict__ ret, size_t S, uint32_t R,
                                           size_t s, uint32_t &row) {
#pragma unroll
  for (int j = 0; j < kRetU; ++j) {
    if (FULL || (uint32_t)j < left) {
      float G[V];
#pragma unroll
      for (int v = 0; v < V; ++v) G[v] = ret_update(b[j].at(v), b[j].dn(v), g, hi[v], lo[v]);
      RetVec<V>::store(ret, (size_t)row * S + s, G);
    }
    row = row == 0 ? R - 1 : row - 1;
  }
}

template <int V>
__device__ __forceinline__ void ret_scan(const RetVec<V> (&b)[kRetU], uint32_t left, float g,
                                         float (&hi)[V], float (&lo)[V], float *__restrict__ ret,
                                         size_t S, uint32_t R, size_t s, uint32_t &row) {
  if (left >= (uint32_t)kRetU)
    ret_scan_n<V, true>(b, left, g, hi, lo, ret, S, R, s, row);
  else
    ret_scan_n<V, false>(b, left, g, hi, lo, ret, S, R, s, row);
}

// Two register buffers alternate without copies: the loads of one are in
// flight while the other is scanned.
template <int V, int T, int MINB>
__global__ __launch_bounds__(T, MINB) void k_returns(Dev d, uint32_t n) {
  const size_t s = ((size_t)blockIdx.x * T + threadIdx.x) * V;
  if (s >= d.n_slots) return;
  const float *__restrict__ rew = d.r_rew;
  const uint8_t *__restrict__ done = d.r_done;
  float *__restrict__ ret = d.r_ret;
  const size_t S = d.n_slots;
  const uint32_t R = d.ring_steps;
  const float g = d.gamma;
  uint32_t row = (uint32_t)((d.k[0] - 1) % R);  // ring row of step k-1 (scan cursor)
  uint32_t lrow = row;                          // ring row of the next load
  auto back = [&](uint32_t r0) {
#pragma unroll
    for (int j = 0; j < kRetU; ++j) r0 = r0 == 0 ? R - 1 : r0 - 1;
    return r0;
  };
  RetVec<V> bufA[kRetU], bufB[kRetU];
  float hi[V], lo[V];
#pragma unroll
  for (int v = 0; v < V; ++v) hi[v] = lo[v] = 0.f;
  ret_load<V>(rew, done, S, R, s, lrow, n, bufA);
  lrow = back(lrow);
  for (uint32_t i = 0; i < n; i += 2 * kRetU) {
    const uint32_t left = n - i;
    if (left > (uint32_t)kRetU) ret_load<V>(rew, done, S, R, s, lrow, left - kRetU, bufB);
    lrow = back(lrow);
    ret_scan<V>(bufA, left, g, hi, lo, ret, S, R, s, row);
    if (left <= (uint32_t)kRetU) break;
    if (left > (uint32_t)(2 * kRetU)) ret_load<V>(rew, done, S, R, s, lrow, left - 2 * kRetU, bufA);
    lrow = back(lrow);
    ret_scan<V>(bufB, left - kRetU, g, hi, lo, ret, S, R, s, row);
  }
}

// S7 for rings with few slots (the landscape's 8,192, a small control run):
// one serial chain per slot leaves most of the chip idle, so each slot's window
// of n steps is cut into NSEG segments scanned at once.  The recurrence is the
// affine map G_t = B_t + A_t G_{t_end} of a segment's carry-in G_{t_end}, and
// such maps compose; per block, 32 consecutive slots (one per lane) times NSEG
// segments (one per warp):
//   pass 1  each segment scans its steps newest first with carry-in 0: B (the
//           float-float return of the segment alone) and A (the product of
//           gamma (1 - d) over the segment, float-float; 0 after a done)
//   combine lane s of warp 0 walks its slot's segments newest first:
//           carry_{j-1} = B_j + A_j carry_j (float-float), carry_last = 0
//   pass 2  each segment scans its steps again from its carry-in, exactly as
//           the serial kernel does, and writes the returns
// The second read of the rewards and done flags mostly hits L2.
__device__ __forceinline__ void ff_mul(float ah, float al, float bh, float bl, float &ph, float &pl) {
  ph = __fmul_rn(ah, bh);
  pl = __fadd_rn(__fmaf_rn(ah, bh, -ph), __fadd_rn(__fmul_rn(ah, bl), __fmul_rn(al, bh)));
}
__device__ __forceinline__ void ff_add(float ah, float al, float bh, float bl, float &sh, float &sl) {
  const float s = __fadd_rn(ah, bh);
  const float bb = __fsub_rn(s, ah);
  const float e = __fadd_rn(__fsub_rn(ah, __fsub_rn(s, bb)), __fsub_rn(bh, bb));
  const float t = __fadd_rn(e, __fadd_rn(al, bl));
  sh = __fadd_rn(s, t);
  sl = __fsub_rn(t, __fsub_rn(sh, s));
}

template <int NSEG>
__global__ __launch_bounds__(32 * NSEG) void k_returns_seg(Dev d, uint32_t n) {
  __shared__ float2 sA[NSEG][32], sB[NSEG][32], sC[NSEG][32];
  const int lane = threadIdx.x & 31, seg = threadIdx.x >> 5;
  const size_t s = (size_t)blockIdx.x * 32 + (size_t)lane;
  const bool valid = s < d.n_slots;
  const size_t S = d.n_slots;
  const uint32_t R = d.ring_steps;
  const float g = d.gamma;
  const uint32_t L = (n + NSEG - 1) / NSEG;
  const uint32_t t_lo = min(n, (uint32_t)seg * L), t_hi = min(n, (uint32_t)(seg + 1) * L);
  // ring row of window step t (t = 0 is step k - n)
  const uint32_t row0 = (uint32_t)((d.k[0] - n) % R);
  auto row_of = [&](uint32_t t) { const uint32_t r = row0 + t; return r >= R ? r - R : r; };
  // steps are taken in batches of kRetU, all of a batch's loads issued first
  float bh = 0.f, bl = 0.f, ah = 1.f, al = 0.f;
  if (valid) {
    for (uint32_t t = t_hi; t > t_lo;) {
      const uint32_t m = min((uint32_t)kRetU, t - t_lo);
      float rr[kRetU];
      uint8_t dd[kRetU];
#pragma unroll
      for (int j = 0; j < kRetU; ++j)
        if ((uint32_t)j < m) {
          const size_t o = (size_t)row_of(t - 1 - (uint32_t)j) * S + s;
          rr[j] = __ldcg(d.r_rew + o);
          dd[j] = __ldcg(d.r_done + o);
        }
#pragma unroll
      for (int j = 0; j < kRetU; ++j)
        if ((uint32_t)j < m) {
          const bool dn = dd[j] != 0;
          ret_update(rr[j], dn, g, bh, bl);
          float ph, pl;
          ff_mul(g, 0.f, ah, al, ph, pl);
          ah = dn ? 0.f : ph;
          al = dn ? 0.f : pl;
        }
      t -= m;
    }
  }
  sA[seg][lane] = make_float2(ah, al);
  sB[seg][lane] = make_float2(bh, bl);
  __syncthreads();
  if (seg == 0) {
    float ch = 0.f, cl = 0.f;
#pragma unroll 1
    for (int j = NSEG - 1; j >= 0; --j) {
      sC[j][lane] = make_float2(ch, cl);
      const float2 a = sA[j][lane], b = sB[j][lane];
      float ph, pl;
      ff_mul(a.x, a.y, ch, cl, ph, pl);
      ff_add(b.x, b.y, ph, pl, ch, cl);
    }
  }
  __syncthreads();
  if (!valid) return;
  const float2 c = sC[seg][lane];
  float hi = c.x, lo = c.y;
  for (uint32_t t = t_hi; t > t_lo;) {
    const uint32_t m = min((uint32_t)kRetU, t - t_lo);
    float rr[kRetU];
    uint8_t dd[kRetU];
#pragma unroll
    for (int j = 0; j < kRetU; ++j)
      if ((uint32_t)j < m) {
        const size_t o = (size_t)row_of(t - 1 - (uint32_t)j) * S + s;
        rr[j] = __ldcs(d.r_rew + o);
        dd[j] = __ldcs(d.r_done + o);
      }
#pragma unroll
    for (int j = 0; j < kRetU; ++j)
      if ((uint32_t)j < m) {
        const size_t o = (size_t)row_of(t - 1 - (uint32_t)j) * S + s;
        __stcs(d.r_ret + o, ret_update(rr[j], dd[j] != 0, g, hi, lo));
      }
    t -= m;
  }
}

inline unsigned blocks(size_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// ------------------------------------------------------------- launchers
void launch_init_policy(float *params, const PolicyShape &shape, uint64_t seed, uint32_t policy_id,
                        cudaStream_t st) {
  const size_t n = shape.count();
  k_init_policy<<<blocks(n, 256) > 4096 ? 4096 : blocks(n, 256), 256, 0, st>>>(params, shape, seed,
                                                                                policy_id);
}

void launch_init_landscape(const Dev &d, uint64_t param_seed, cudaStream_t st) {
  k_init_landscape<<<blocks(d.n_gauss, 128), 128, 0, st>>>(d.centres, d.widths, d.amps, (int)d.dim,
                                                           (int)d.n_gauss, param_seed);
}

void launch_landscape_derive(const Dev &d, cudaStream_t st) {
  k_landscape_derive<<<blocks(d.n_gauss, 128), 128, 0, st>>>(d);
}

void launch_reset(const Dev &d, cudaStream_t st) {
  const size_t n = d.env == WS_ENV_ECONOMY ? (d.n_agent_slots > d.n_envs ? d.n_agent_slots : d.n_envs)
                                           : d.n_envs;
  k_reset<<<blocks(n, 256), 256, 0, st>>>(d);
  if (d.env == WS_ENV_LANDSCAPE) {
    cudaFuncSetAttribute(k_energy_partial, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)energy_smem(d));
    landscape_energy(d, 0, 1, st);
    k_landscape_reset_finish<<<blocks(d.n_envs, 256), 256, 0, st>>>(d, 0, 1);
  }
}

void launch_plain_step(const Dev &d, uint32_t off, cudaStream_t st, const Branch *br) {
  const int T = d.env_threads > 0 ? d.env_threads : 256;  // per-env kernels' block size
  if (d.env == WS_ENV_CONTROL) {
    k_store_obs<<<blocks(d.n_envs, T), T, 0, st>>>(d, off, d.s, 4, d.n_envs, d.n_envs, 0);
    policy(d, d.s, 1, d.n_envs, d.params, d.pol, 0, d.h0, d.h1, d.out, (int)d.n_envs, st);
    k_sample_cat<<<blocks(d.n_envs, T), T, 0, st>>>(d, off, d.out, 2, 0, d.n_envs, 0);
    k_control_step<<<blocks(d.n_envs, T), T, 0, st>>>(d, off);
  } else if (d.env == WS_ENV_ACROBOT) {
    k_acrobot_observe<<<blocks(d.n_envs, T), T, 0, st>>>(d, off);
    policy(d, d.pobs, 1, d.n_envs, d.params, d.pol, 0, d.h0, d.h1, d.out, (int)d.n_envs, st);
    k_sample_cat<<<blocks(d.n_envs, T), T, 0, st>>>(d, off, d.out, 3, 0, d.n_envs, 0);
    k_acrobot_step<<<blocks(d.n_envs, T), T, 0, st>>>(d, off);
  } else if (d.env == WS_ENV_ECONOMY) {
    k_econ_observe<<<d.n_envs, kEconThreads, 0, st>>>(d, off);
    // the planner's policy and draw are independent of the agents': side branch
    cudaStream_t ps = st;
    if (br) {
      cudaEventRecord(br->fork, st);
      cudaStreamWaitEvent(br->aux, br->fork, 0);
      ps = br->aux;
    }
    policy(d, d.pobs, kEconF, 1, d.params_planner, d.pol_planner, 1, d.ph0, d.ph1, d.pout,
           (int)d.n_envs, ps);
    k_sample_cat<<<blocks(d.n_envs, T), T, 0, ps>>>(d, off, d.pout, (int)d.n_out_planner, 2,
                                                         d.n_envs, d.n_agent_slots);
    policy(d, d.feat, 1, d.n_agent_slots, d.params, d.pol, 0, d.h0, d.h1, d.out,
           (int)d.n_agent_slots, st);
    k_sample_cat<<<blocks(d.n_agent_slots, T), T, 0, st>>>(d, off, d.out, (int)d.n_out, 1,
                                                                d.n_agent_slots, 0);
    if (br) {
      cudaEventRecord(br->join, br->aux);
      cudaStreamWaitEvent(st, br->join, 0);
    }
    k_econ_transfer<<<blocks(d.n_agent_slots, T), T, 0, st>>>(d, off);
    k_econ_finish<<<d.n_envs, kEconThreads, 0, st>>>(d, off);
  } else {
    k_store_obs<<<blocks(d.n_envs, T), T, 0, st>>>(d, off, d.s, (int)d.dim, d.n_envs, d.n_envs, 0);
    policy(d, d.s, 1, d.n_envs, d.params, d.pol, 0, d.h0, d.h1, d.out, (int)d.n_envs, st);
    k_sample_gauss<<<blocks(d.n_envs, T), T, 0, st>>>(d, off);
    landscape_energy(d, off, 0, st);
    k_landscape_step<<<blocks(d.n_envs, T), T, 0, st>>>(d, off);
    landscape_energy(d, off, 1, st);
    k_landscape_reset_finish<<<blocks(d.n_envs, T), T, 0, st>>>(d, off, 0);
  }
}

void launch_advance(const Dev &d, uint32_t n, cudaStream_t st) { k_advance<<<1, 32, 0, st>>>(d, n); }

void launch_returns(const Dev &d, uint32_t n_steps, cudaStream_t st) {
  // few slots: the segmented scan (16 segments per slot keep the chip busy;
  // 32 measured no faster on 8,192 slots x 1,000 steps)
  if (d.n_slots < 32768 && n_steps >= 64) {
    k_returns_seg<16><<<blocks(d.n_slots, 32), 32 * 16, 0, st>>>(d, n_steps);
    return;
  }
  if (d.n_slots % 4 == 0)  // every ring row starts on a 16-byte boundary
    k_returns<4, 32, 8><<<blocks(d.n_slots / 4, 32), 32, 0, st>>>(d, n_steps);
  else
    k_returns<1, 128, 5><<<blocks(d.n_slots, 128), 128, 0, st>>>(d, n_steps);
}

}  // namespace ws

namespace ws {
void launch_dense_fp32(const float *X, long ldr, long ldc, const float *W, const float *b, float *Y,
                       int M, int K, int N, int act, cudaStream_t st) {
  dense(X, ldr, ldc, W, b, Y, M, K, N, act, st);
}
}  // namespace ws
