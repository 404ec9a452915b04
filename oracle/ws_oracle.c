/*
 * ws_oracle.c -- plain, slow, FP64 CPU oracle for the in-place RL roll-out loop.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or call
 * this file: only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline /
 * reference legs use it.  It shares no code, header, table or constant
 * generator with the CUDA library (paper_2408_00930_gb300/csrc); both sides
 * implement Philox4x32-10 independently from its published definition.
 *
 * What the roll-out loop computes (paper Sec. 2 and App. B, "the entire RL
 * workflow ... roll-outs, action inference, reset"): for every environment and
 * every step, observe the state, run the policy network, sample an action, step
 * the environment (state update, reward, done), auto-reset finished
 * environments, and write the transition into the in-place store.  The paper
 * prints no formulas; the environments, policies and random streams below are
 * the synthetic workloads of the build's configuration list (classic-control
 * stand-in, multi-agent economy stand-in, Gaussian-sum reaction landscape
 * stand-in, App. C), with every unstated detail fixed as a documented reading.
 *
 * Everything here is the definition written out step by step, env by env, in
 * double precision, except where the definition itself fixes FP32 (initial
 * uniform draws, which are defined as one FP32 fused multiply-add and are
 * reproduced exactly) or integers (wealth, actions, counters).
 *
 * Pins (tests/test_oracle_*.py): Philox against an independent library
 * implementation; uniformity; hand-computed control steps; exact wealth
 * conservation and hand-computed tiny economies; M=1 closed form and
 * finite-difference gradients of the landscape; sampler closed forms; the
 * closed form of discounted returns.  Policy-training convergence is out of
 * scope ("parity unpinned" does not apply to any function here).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------ */
/* Philox4x32-10: Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11, Sec. 5.  Two 32x32->64 multiplications per round, */
/* the halves XOR-ed with the other two counter words and the round key; the */
/* key is bumped by the Weyl constants (golden ratio, sqrt(3)-1) each round. */
/* ------------------------------------------------------------------------ */
#define OR_PHILOX_M0 0xD2511F53u
#define OR_PHILOX_M1 0xCD9E8D57u
#define OR_PHILOX_W0 0x9E3779B9u
#define OR_PHILOX_W1 0xBB67AE85u

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += OR_PHILOX_W0;
      k1 += OR_PHILOX_W1;
    }
    uint64_t p0 = (uint64_t)OR_PHILOX_M0 * (uint64_t)x0;
    uint64_t p1 = (uint64_t)OR_PHILOX_M1 * (uint64_t)x2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    uint32_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Batch form for tests: n counters [n][4] under one key. */
void or_philox_batch(long n, const uint32_t *ctr, const uint32_t key[2], uint32_t *out) {
  for (long i = 0; i < n; ++i) or_philox4x32_10(ctr + 4 * i, key, out + 4 * i);
}

/* Counter layout of every draw [reading of "(seed, env, agent, step)"]:
 *   key  = (seed low 32, seed high 32)
 *   ctr0 = step counter k (or a draw index for one-off initialisation)
 *   ctr1 = env id,  ctr2 = agent id (planner = 0xFFFFFFFF),
 *   ctr3 = tag << 24 | sub-index                                          */
enum {
  OR_TAG_ACTION = 0,
  OR_TAG_RESET = 1,
  OR_TAG_PARTNER = 2,
  OR_TAG_NOISE = 3,
  OR_TAG_POLICY_INIT = 4,
  OR_TAG_LANDSCAPE_INIT = 5,
  OR_TAG_ECON_INIT = 6
};
#define OR_PLANNER_ID 0xFFFFFFFFu
#define OR_STEP_INIT 0xFFFFFFFFu /* "step -1": the draw made by a full reset */

static void or_draw(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t tag,
                    uint32_t sub, uint32_t out[4]) {
  uint32_t ctr[4] = {c0, c1, c2, (tag << 24) | (sub & 0xFFFFFFu)};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  or_philox4x32_10(ctr, key, out);
}

/* u in [0,1) from the top 24 bits; exact in FP32 and FP64. */
double or_u01(uint32_t w) { return (double)(w >> 8) * 0x1p-24; }

/* U(a,b) is defined as the FP32 value fmaf(b-a, u, a) with b-a an FP32
 * subtraction.  The FP64 product and sum below are exact (24-bit by 24-bit
 * product, operands within 2^26 of each other in magnitude for every range
 * used), so one rounding to float reproduces the fused multiply-add. */
float or_uniform_f32(uint32_t w, float a, float b) {
  float d = b - a;
  double exact = (double)d * or_u01(w) + (double)a;
  return (float)exact;
}

/* Box-Muller on one pair of words: u1 in (0,1], u2 in [0,1). */
void or_box_muller(uint32_t w0, uint32_t w1, double *z_cos, double *z_sin) {
  double u1 = ((double)(w0 >> 8) + 1.0) * 0x1p-24;
  double u2 = (double)(w1 >> 8) * 0x1p-24;
  double rho = sqrt(-2.0 * log(u1));
  *z_cos = rho * cos(2.0 * M_PI * u2);
  *z_sin = rho * sin(2.0 * M_PI * u2);
}

/* floor(w * n / 2^32): Lemire's multiply-shift bounded integer. */
uint32_t or_bounded(uint32_t w, uint32_t n) { return (uint32_t)(((uint64_t)w * n) >> 32); }

/* Round-to-nearest-even to bfloat16, returned as float (finite inputs). */
float or_round_bf16(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  uint32_t lsb = (u >> 16) & 1u;
  u += 0x7FFFu + lsb;
  u &= 0xFFFF0000u;
  float r;
  memcpy(&r, &u, 4);
  return r;
}

/* ------------------------------------------------------------------------ */
/* Policy MLP: widths[0] -> widths[1] -> ... -> widths[n_layers], tanh on   */
/* every hidden layer, linear output (paper App. B: policy models live in   */
/* global memory and every agent thread runs inference on them).            */
/* Parameter layout, per layer l: W_l[n_in][n_out] row-major, then b_l.     */
/* ------------------------------------------------------------------------ */
long or_policy_param_count(int n_layers, const int32_t *widths) {
  long n = 0;
  for (int l = 0; l < n_layers; ++l) n += (long)widths[l] * widths[l + 1] + widths[l + 1];
  return n;
}

/* Random init: every weight and bias of layer l is U(-1/sqrt(n_in), 1/sqrt(n_in))
 * [reading: the usual fan-in bound].  Element i of layer l takes word i&3 of
 * the draw (ctr0=i>>2, ctr1=l, ctr2=policy id, tag POLICY_INIT) under the
 * parameter seed.  The bound is one FP32 square root and one FP32 division. */
void or_policy_init(uint64_t seed, uint32_t policy_id, int n_layers, const int32_t *widths,
                    float *out) {
  long off = 0;
  for (int l = 0; l < n_layers; ++l) {
    int n_in = widths[l], n_out = widths[l + 1];
    float bound = 1.0f / sqrtf((float)n_in);
    long count = (long)n_in * n_out + n_out;
    for (long i = 0; i < count; ++i) {
      uint32_t w[4];
      or_draw(seed, (uint32_t)(i >> 2), (uint32_t)l, policy_id, OR_TAG_POLICY_INIT, 0, w);
      out[off + i] = or_uniform_f32(w[i & 3], -bound, bound);
    }
    off += count;
  }
}

/* Forward pass in FP64.  bf16_layers: bit l set means layer l's GEMM runs on
 * the BF16 tensor path, so its input activations and its weights (not its
 * bias) are first rounded to bfloat16; accumulation stays exact here. */
void or_mlp_forward(int n_layers, const int32_t *widths, const float *params, uint32_t bf16_layers,
                    const double *x, double *y) {
  int maxw = 0;
  for (int l = 0; l <= n_layers; ++l)
    if (widths[l] > maxw) maxw = widths[l];
  double *a = (double *)malloc(sizeof(double) * maxw);
  double *z = (double *)malloc(sizeof(double) * maxw);
  for (int i = 0; i < widths[0]; ++i) a[i] = x[i];
  long off = 0;
  for (int l = 0; l < n_layers; ++l) {
    int n_in = widths[l], n_out = widths[l + 1];
    const float *W = params + off;
    const float *b = W + (long)n_in * n_out;
    int bf = (bf16_layers >> l) & 1u;
    for (int j = 0; j < n_out; ++j) {
      double s = (double)b[j];
      for (int i = 0; i < n_in; ++i) {
        double ai = bf ? (double)or_round_bf16((float)a[i]) : a[i];
        double wij = bf ? (double)or_round_bf16(W[(long)i * n_out + j]) : (double)W[(long)i * n_out + j];
        s += ai * wij;
      }
      z[j] = s;
    }
    int last = (l == n_layers - 1);
    for (int j = 0; j < n_out; ++j) a[j] = last ? z[j] : tanh(z[j]);
    off += (long)n_in * n_out + n_out;
  }
  for (int j = 0; j < widths[n_layers]; ++j) y[j] = a[j];
  free(a);
  free(z);
}

/* ------------------------------------------------------------------------ */
/* Categorical sampling by inverse CDF: a = min{ i : u < CDF_i }, CDF from   */
/* the softmax of the logits; logp = log p_a.  margin = min_i |u - CDF_i|    */
/* over the inner boundaries (the distance of the draw to a decision flip).  */
/* ------------------------------------------------------------------------ */
int or_sample_categorical(int n, const double *logits, double u, double *logp, double *margin) {
  double m = logits[0];
  for (int i = 1; i < n; ++i)
    if (logits[i] > m) m = logits[i];
  double S = 0.0;
  for (int i = 0; i < n; ++i) S += exp(logits[i] - m);
  double cdf = 0.0, mg = INFINITY;
  int a = n - 1, found = 0;
  for (int i = 0; i < n - 1; ++i) {
    cdf += exp(logits[i] - m) / S;
    double d = fabs(u - cdf);
    if (d < mg) mg = d;
    if (!found && u < cdf) {
      a = i;
      found = 1;
    }
  }
  if (logp) *logp = (logits[a] - m) - log(S);
  if (margin) *margin = mg;
  return a;
}

/* Diagonal Gaussian policy head [reading]: out[0:D] = mean, out[D:2D] = log
 * sigma clamped to [-5, 2]; dx_j = clip(mean_j + sigma_j z_j, -clip, clip);
 * logp is the density of the unclipped sample. */
void or_gaussian_action(int D, const double *out, const double *z, double clip, double *dx,
                        double *logp) {
  double lp = 0.0;
  for (int j = 0; j < D; ++j) {
    double ls = out[D + j];
    if (ls < -5.0) ls = -5.0;
    if (ls > 2.0) ls = 2.0;
    double s = out[j] + exp(ls) * z[j];
    if (s > clip) s = clip;
    if (s < -clip) s = -clip;
    dx[j] = s;
    lp += -0.5 * z[j] * z[j] - ls - 0.5 * log(2.0 * M_PI);
  }
  *logp = lp;
}

/* ------------------------------------------------------------------------ */
/* Control environment (cart-pole-like stand-in for gym classic control,    */
/* App. C "Classic Control").  State (x, v, th, w); action 1 pushes u=+10,  */
/* action 0 pushes u=-10 [reading].  x'' = u - 0.5 x - 0.1 v,                */
/* th'' = 9.8 sin th - 0.3 cos th * u, explicit Euler with dt = 0.02, every */
/* update from the old state [reading].  Reward 1 per step.                 */
/* ------------------------------------------------------------------------ */
void or_control_dynamics(const double s[4], int action, double out[4]) {
  double u = action ? 10.0 : -10.0;
  double x = s[0], v = s[1], th = s[2], w = s[3];
  double xacc = u - 0.5 * x - 0.1 * v;
  double thacc = 9.8 * sin(th) - 0.3 * cos(th) * u;
  out[0] = x + 0.02 * v;
  out[1] = v + 0.02 * xacc;
  out[2] = th + 0.02 * w;
  out[3] = w + 0.02 * thacc;
}

/* Done when |x| > 2.4 or |th| > 0.21 (strict) or the episode step count
 * reaches the limit.  margin = relative distance of the deciding quantities
 * to their thresholds (for the float-decides-an-integer rule). */
int or_control_done(const double s[4], int t, int limit, double *margin) {
  double mx = fabs(fabs(s[0]) - 2.4) / 2.4;
  double mt = fabs(fabs(s[2]) - 0.21) / 0.21;
  if (margin) *margin = mx < mt ? mx : mt;
  return (fabs(s[0]) > 2.4) || (fabs(s[2]) > 0.21) || (t >= limit);
}

/* State draw: 4 words of RESET(ctr0=k, env, agent 0) each U(-0.05, 0.05). */
void or_control_reset_draw(uint64_t seed, uint32_t k, uint32_t env, double s[4]) {
  uint32_t w[4];
  or_draw(seed, k, env, 0, OR_TAG_RESET, 0, w);
  for (int d = 0; d < 4; ++d) s[d] = (double)or_uniform_f32(w[d], -0.05f, 0.05f);
}

/* Roll out envs env_ids[0..n_envs) for n_steps from step counter k0.
 * state0/t0 may be NULL: the initial state is then the full-reset draw.
 * Outputs are [n_steps][n_envs] (obs is [n_steps][n_envs][4], logits
 * [n_steps][n_envs][n_out]); any output pointer may be NULL.
 * obs is the pre-step state; the record keeps the terminal transition and
 * the state is redrawn in place (RESET at ctr0 = k) when done. */
void or_control_rollout(const float *params, int hidden0, int hidden1, uint32_t bf16_layers,
                        uint64_t seed, uint32_t k0, const uint32_t *env_ids, int n_envs,
                        const double *state0, const int32_t *t0, int n_steps, int episode_limit,
                        double *obs, int32_t *action, double *logp, double *reward, uint8_t *done,
                        double *logits, double *act_margin, double *done_margin,
                        double *state_out, int32_t *t_out) {
  int32_t widths[4] = {4, hidden0, hidden1, 2};
  for (int e = 0; e < n_envs; ++e) {
    uint32_t env = env_ids[e];
    double s[4];
    int t;
    if (state0) {
      for (int d = 0; d < 4; ++d) s[d] = state0[(long)e * 4 + d];
    } else {
      or_control_reset_draw(seed, OR_STEP_INIT, env, s);
    }
    t = t0 ? t0[e] : 0;
    for (int i = 0; i < n_steps; ++i) {
      uint32_t k = k0 + (uint32_t)i;
      long r = (long)i * n_envs + e;
      double lg[2], lp, mg;
      or_mlp_forward(3, widths, params, bf16_layers, s, lg);
      uint32_t w[4];
      or_draw(seed, k, env, 0, OR_TAG_ACTION, 0, w);
      int a = or_sample_categorical(2, lg, or_u01(w[0]), &lp, &mg);
      double s2[4], dm;
      or_control_dynamics(s, a, s2);
      int dn = or_control_done(s2, t + 1, episode_limit, &dm);
      if (obs)
        for (int d = 0; d < 4; ++d) obs[r * 4 + d] = s[d];
      if (action) action[r] = a;
      if (logp) logp[r] = lp;
      if (reward) reward[r] = 1.0;
      if (done) done[r] = (uint8_t)dn;
      if (logits) {
        logits[r * 2 + 0] = lg[0];
        logits[r * 2 + 1] = lg[1];
      }
      if (act_margin) act_margin[r] = mg;
      if (done_margin) done_margin[r] = dm;
      if (dn) {
        or_control_reset_draw(seed, k, env, s);
        t = 0;
      } else {
        for (int d = 0; d < 4; ++d) s[d] = s2[d];
        t = t + 1;
      }
    }
    if (state_out)
      for (int d = 0; d < 4; ++d) state_out[(long)e * 4 + d] = s[d];
    if (t_out) t_out[e] = t;
  }
}

/* ------------------------------------------------------------------------ */
/* Acrobot (App. C "Classic Control": the gym Acrobot-v1 benchmark).  Two    */
/* links hang from a pivot; only the joint between them is actuated.  The     */
/* physics is the two-link acrobot of Sutton & Barto (1998, Sec. 11.3) in     */
/* its book form: m1 = m2 = 1, l1 = 1, lc1 = lc2 = 0.5 (centres of mass),     */
/* I1 = I2 = 1, g = 9.8, angles from hanging straight down.  With            */
/*   d1 = m1 lc1^2 + m2 (l1^2 + lc2^2 + 2 l1 lc2 cos th2) + I1 + I2          */
/*   d2 = m2 (lc2^2 + l1 lc2 cos th2) + I2                                   */
/*   phi2 = m2 lc2 g sin(th1 + th2)                                          */
/*   phi1 = -m2 l1 lc2 w2^2 sin th2 - 2 m2 l1 lc2 w2 w1 sin th2              */
/*          + (m1 lc1 + m2 l1) g sin th1 + phi2                              */
/* the accelerations are                                                     */
/*   th2'' = (tau + d2/d1 phi1 - m2 l1 lc2 w1^2 sin th2 - phi2)              */
/*           / (m2 lc2^2 + I2 - d2^2 / d1)                                   */
/*   th1'' = -(d2 th2'' + phi1) / d1.                                        */
/* Readings: action a in {0, 1, 2} applies torque tau = a - 1; one classic  */
/* Runge-Kutta (RK4) step of dt = 0.2 with tau held; then both angles are    */
/* wrapped into [-pi, pi] and the velocities clipped to |w1| <= 4 pi,        */
/* |w2| <= 9 pi.  Terminal when the tip is more than one link above the     */
/* pivot, -cos th1 - cos(th1 + th2) > 1.  Reward -1 per step, 0 on the      */
/* terminal step.  Observation (cos th1, sin th1, cos th2, sin th2, w1, w2); */
/* a reset draws the state (th1, th2, w1, w2) from U(-0.1, 0.1)^4.          */
/* ------------------------------------------------------------------------ */
void or_acrobot_deriv(const double s[4], double tau, double ds[4]) {
  const double m1 = 1.0, m2 = 1.0, l1 = 1.0, lc1 = 0.5, lc2 = 0.5, I1 = 1.0, I2 = 1.0, g = 9.8;
  double th1 = s[0], th2 = s[1], w1 = s[2], w2 = s[3];
  double d1 = m1 * lc1 * lc1 + m2 * (l1 * l1 + lc2 * lc2 + 2.0 * l1 * lc2 * cos(th2)) + I1 + I2;
  double d2 = m2 * (lc2 * lc2 + l1 * lc2 * cos(th2)) + I2;
  double phi2 = m2 * lc2 * g * sin(th1 + th2);
  double phi1 = -m2 * l1 * lc2 * w2 * w2 * sin(th2) - 2.0 * m2 * l1 * lc2 * w2 * w1 * sin(th2) +
                (m1 * lc1 + m2 * l1) * g * sin(th1) + phi2;
  double acc2 = (tau + d2 / d1 * phi1 - m2 * l1 * lc2 * w1 * w1 * sin(th2) - phi2) /
                (m2 * lc2 * lc2 + I2 - d2 * d2 / d1);
  double acc1 = -(d2 * acc2 + phi1) / d1;
  ds[0] = w1;
  ds[1] = w2;
  ds[2] = acc1;
  ds[3] = acc2;
}

static double or_wrap_pi(double x) {
  while (x > M_PI) x -= 2.0 * M_PI;
  while (x < -M_PI) x += 2.0 * M_PI;
  return x;
}

/* One step: RK4 over dt, then wrap and clip.  raw (may be NULL) receives the
 * RK4 result before wrapping and clipping. */
void or_acrobot_step(const double s[4], int action, double dt, double out[4], double raw[4]) {
  double tau = (double)action - 1.0;
  double k1[4], k2[4], k3[4], k4[4], y[4];
  or_acrobot_deriv(s, tau, k1);
  for (int i = 0; i < 4; ++i) y[i] = s[i] + 0.5 * dt * k1[i];
  or_acrobot_deriv(y, tau, k2);
  for (int i = 0; i < 4; ++i) y[i] = s[i] + 0.5 * dt * k2[i];
  or_acrobot_deriv(y, tau, k3);
  for (int i = 0; i < 4; ++i) y[i] = s[i] + dt * k3[i];
  or_acrobot_deriv(y, tau, k4);
  for (int i = 0; i < 4; ++i) y[i] = s[i] + dt / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
  if (raw)
    for (int i = 0; i < 4; ++i) raw[i] = y[i];
  const double v1 = 4.0 * M_PI, v2 = 9.0 * M_PI;
  out[0] = or_wrap_pi(y[0]);
  out[1] = or_wrap_pi(y[1]);
  out[2] = y[2] < -v1 ? -v1 : (y[2] > v1 ? v1 : y[2]);
  out[3] = y[3] < -v2 ? -v2 : (y[3] > v2 ? v2 : y[3]);
}

void or_acrobot_obs(const double s[4], double o[6]) {
  o[0] = cos(s[0]);
  o[1] = sin(s[0]);
  o[2] = cos(s[1]);
  o[3] = sin(s[1]);
  o[4] = s[2];
  o[5] = s[3];
}

/* Tip height above the pivot in link lengths: -cos th1 - cos(th1 + th2);
 * terminal when it exceeds 1.  margin = |height - 1|. */
int or_acrobot_terminal(const double s[4], double *margin) {
  double h = -cos(s[0]) - cos(s[0] + s[1]);
  if (margin) *margin = fabs(h - 1.0);
  return h > 1.0;
}

void or_acrobot_reset_draw(uint64_t seed, uint32_t k, uint32_t env, double s[4]) {
  uint32_t w[4];
  or_draw(seed, k, env, 0, OR_TAG_RESET, 0, w);
  for (int d = 0; d < 4; ++d) s[d] = (double)or_uniform_f32(w[d], -0.1f, 0.1f);
}

/* Roll out envs env_ids[] for n_steps from step counter k0 (as the control
 * roll-out): policy 6 -> hidden0 -> hidden1 -> 3 on the observation, action
 * drawn from ACTION(k, env) word 0, done on the terminal height or at the
 * episode limit, reset in place.  obs [n_steps][n_envs][6] is the pre-step
 * observation, state_rec [n_steps][n_envs][4] the pre-step state; margins
 * are the sampler's distance to its tie band and the height's distance to 1. */
void or_acrobot_rollout(const float *params, int hidden0, int hidden1, uint32_t bf16_layers,
                        uint64_t seed, uint32_t k0, const uint32_t *env_ids, int n_envs,
                        const double *state0, const int32_t *t0, int n_steps, int episode_limit,
                        double *obs, double *state_rec, int32_t *action, double *logp,
                        double *reward, uint8_t *done, double *logits, double *act_margin,
                        double *done_margin, double *state_out, int32_t *t_out) {
  int32_t widths[4] = {6, hidden0, hidden1, 3};
  for (int e = 0; e < n_envs; ++e) {
    uint32_t env = env_ids[e];
    double s[4];
    int t = t0 ? t0[e] : 0;
    if (state0)
      for (int d = 0; d < 4; ++d) s[d] = state0[(long)e * 4 + d];
    else
      or_acrobot_reset_draw(seed, OR_STEP_INIT, env, s);
    for (int i = 0; i < n_steps; ++i) {
      uint32_t k = k0 + (uint32_t)i;
      long r = (long)i * n_envs + e;
      double o[6], lg[3], lp, mg;
      or_acrobot_obs(s, o);
      or_mlp_forward(3, widths, params, bf16_layers, o, lg);
      uint32_t w[4];
      or_draw(seed, k, env, 0, OR_TAG_ACTION, 0, w);
      int a = or_sample_categorical(3, lg, or_u01(w[0]), &lp, &mg);
      double s2[4], dm;
      or_acrobot_step(s, a, 0.2, s2, NULL);
      int term = or_acrobot_terminal(s2, &dm);
      int dn = term || (t + 1 >= episode_limit);
      if (obs)
        for (int d = 0; d < 6; ++d) obs[r * 6 + d] = o[d];
      if (state_rec)
        for (int d = 0; d < 4; ++d) state_rec[r * 4 + d] = s[d];
      if (action) action[r] = a;
      if (logp) logp[r] = lp;
      if (reward) reward[r] = term ? 0.0 : -1.0;
      if (done) done[r] = (uint8_t)dn;
      if (logits)
        for (int c = 0; c < 3; ++c) logits[r * 3 + c] = lg[c];
      if (act_margin) act_margin[r] = mg;
      if (done_margin) done_margin[r] = dm;
      if (dn) {
        or_acrobot_reset_draw(seed, k, env, s);
        t = 0;
      } else {
        for (int d = 0; d < 4; ++d) s[d] = s2[d];
        t = t + 1;
      }
    }
    if (state_out)
      for (int d = 0; d < 4; ++d) state_out[(long)e * 4 + d] = s[d];
    if (t_out) t_out[e] = t;
  }
}

/* ------------------------------------------------------------------------ */
/* Multi-agent economy (stand-in for the two-level economic simulation of   */
/* App. C "Multi-Agent Economics": many agents plus one planner per env,    */
/* agent interactions across threads).  Whole definition is a reading:     */
/*  - agents choose activity a in {0..19}, the planner a tax level in {0..9}*/
/*  - transfer t_i = floor(w_i a_i / 400) to partner                        */
/*    p_i = (i + 1 + floor(r (n-1) / 2^32)) mod n, from pre-step wealth     */
/*  - tax_i = floor(income_i tau / 20); pool T shared as floor(T/n) each,   */
/*    the first (T mod n) agents one more: total wealth is conserved exactly*/
/*  - features f_k <- 0.95 f_k + 0.05 (-1)^k (a-9.5)/9.5 (k<15),            */
/*    f_15 = ln(w)/ln(1e6)                                                  */
/*  - reward r_i = (w_i' - w_i)/1e4 - 1e-3 a_i^2; planner: mean of r_i      */
/*  - done at the episode limit; reset redraws wealth U[1e4, 1e6] (64-bit   */
/*    word mod 990001) and features N(0,1); agent counts stay fixed.        */
/* ------------------------------------------------------------------------ */
#define OR_ECON_F 16

uint32_t or_econ_agent_count(uint64_t param_seed, uint32_t env) {
  uint32_t w[4];
  or_draw(param_seed, 0, env, 0, OR_TAG_ECON_INIT, 0, w);
  return 8u + or_bounded(w[0], 249u);
}

void or_econ_reset_agent(uint64_t seed, uint32_t k, uint32_t env, uint32_t agent, int64_t *wealth,
                         double *f) {
  uint32_t w[4];
  or_draw(seed, k, env, agent, OR_TAG_RESET, 0, w);
  uint64_t big = ((uint64_t)w[1] << 32) | (uint64_t)w[0];
  *wealth = 10000 + (int64_t)(big % 990001ull);
  for (int j = 0; j < 4; ++j) {
    or_draw(seed, k, env, agent, OR_TAG_RESET, 1 + j, w);
    or_box_muller(w[0], w[1], &f[4 * j + 0], &f[4 * j + 1]);
    or_box_muller(w[2], w[3], &f[4 * j + 2], &f[4 * j + 3]);
  }
}

/* One step of one env with n agents.  Inputs: wealth[n], feat[n][16], step t,
 * step counter k; actions are sampled here from the two policies.  Outputs
 * the records (obs = pre-step) for the n agents and the planner and updates
 * wealth/feat/t in place (including the auto-reset). */
void or_econ_env_step(const float *agent_params, const float *planner_params, uint32_t bf16_layers,
                      uint64_t seed, uint32_t k, uint32_t env, int n, int episode_limit,
                      int64_t *wealth, double *feat, int32_t *t_io,
                      /* per-agent records [n] and planner record [1] */
                      double *rec_obs, int32_t *rec_action, double *rec_logp, double *rec_reward,
                      uint8_t *rec_done, int64_t *rec_wealth, double *rec_margin,
                      double *pl_obs, int32_t *pl_action, double *pl_logp, double *pl_reward,
                      uint8_t *pl_done, int64_t *pl_wealth, double *pl_margin) {
  const int32_t aw[4] = {OR_ECON_F, 128, 128, 20};
  const int32_t pw[4] = {OR_ECON_F, 128, 128, 10};
  int32_t *a = (int32_t *)malloc(sizeof(int32_t) * n);
  int64_t *w0 = (int64_t *)malloc(sizeof(int64_t) * n);
  int64_t *income = (int64_t *)calloc(n, sizeof(int64_t));
  double lg[20], lp, mg;
  uint32_t wd[4];
  /* agents: observe, infer, sample */
  for (int i = 0; i < n; ++i) {
    w0[i] = wealth[i];
    or_mlp_forward(3, aw, agent_params, bf16_layers, feat + (long)i * OR_ECON_F, lg);
    or_draw(seed, k, env, (uint32_t)i, OR_TAG_ACTION, 0, wd);
    a[i] = or_sample_categorical(20, lg, or_u01(wd[0]), &lp, &mg);
    if (rec_obs)
      for (int j = 0; j < OR_ECON_F; ++j) rec_obs[(long)i * OR_ECON_F + j] = feat[(long)i * OR_ECON_F + j];
    rec_action[i] = a[i];
    rec_logp[i] = lp;
    if (rec_margin) rec_margin[i] = mg;
    rec_wealth[i] = w0[i];
  }
  /* planner: observes the mean agent features */
  double mean[OR_ECON_F];
  for (int j = 0; j < OR_ECON_F; ++j) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += feat[(long)i * OR_ECON_F + j];
    mean[j] = s / n;
  }
  double plg[10];
  or_mlp_forward(3, pw, planner_params, bf16_layers, mean, plg);
  or_draw(seed, k, env, OR_PLANNER_ID, OR_TAG_ACTION, 0, wd);
  double plp, pmg;
  int tau = or_sample_categorical(10, plg, or_u01(wd[0]), &plp, &pmg);
  /* transfers, all amounts from pre-step wealth */
  int64_t total0 = 0;
  for (int i = 0; i < n; ++i) total0 += w0[i];
  for (int i = 0; i < n; ++i) {
    or_draw(seed, k, env, (uint32_t)i, OR_TAG_PARTNER, 0, wd);
    int p = (int)(((uint32_t)i + 1u + or_bounded(wd[0], (uint32_t)(n - 1))) % (uint32_t)n);
    int64_t amt = (w0[i] * (int64_t)a[i]) / 400;
    wealth[i] -= amt;
    wealth[p] += amt;
    income[p] += amt;
  }
  /* tax on income, redistributed evenly (remainder to the lowest indices) */
  int64_t T = 0;
  for (int i = 0; i < n; ++i) {
    int64_t tax = (income[i] * (int64_t)tau) / 20;
    wealth[i] -= tax;
    T += tax;
  }
  int64_t share = T / n, rem = T % n; /* floor division, any sign of the pool */
  if (rem < 0) {
    rem += n;
    share -= 1;
  }
  for (int i = 0; i < n; ++i) wealth[i] += share + (i < rem ? 1 : 0);
  /* features and rewards */
  double rsum = 0.0;
  for (int i = 0; i < n; ++i) {
    double *f = feat + (long)i * OR_ECON_F;
    double drive = ((double)a[i] - 9.5) / 9.5;
    for (int j = 0; j < OR_ECON_F - 1; ++j) f[j] = 0.95 * f[j] + 0.05 * ((j & 1) ? -drive : drive);
    f[OR_ECON_F - 1] = log((double)wealth[i]) / log(1e6);
    double r = (double)(wealth[i] - w0[i]) / 1e4 - 1e-3 * (double)a[i] * (double)a[i];
    rec_reward[i] = r;
    rsum += r;
  }
  int t = *t_io + 1;
  int dn = t >= episode_limit;
  for (int i = 0; i < n; ++i) rec_done[i] = (uint8_t)dn;
  if (pl_obs)
    for (int j = 0; j < OR_ECON_F; ++j) pl_obs[j] = mean[j];
  *pl_action = tau;
  *pl_logp = plp;
  *pl_reward = rsum / n;
  *pl_done = (uint8_t)dn;
  *pl_wealth = total0;
  if (pl_margin) *pl_margin = pmg;
  if (dn) {
    for (int i = 0; i < n; ++i)
      or_econ_reset_agent(seed, k, env, (uint32_t)i, &wealth[i], feat + (long)i * OR_ECON_F);
    t = 0;
  }
  *t_io = t;
  free(a);
  free(w0);
  free(income);
}

/* Roll out envs env_ids[0..n_envs) with agent counts n_agents[] for n_steps.
 * Slot layout of the outputs: the agents of env_ids[0], then of env_ids[1],
 * ..., then one planner slot per env in the same order.  Initial state is the
 * full-reset draw unless wealth0/feat0/t0 are given (in slot layout). */
void or_econ_rollout(const float *agent_params, const float *planner_params, uint32_t bf16_layers,
                     uint64_t seed, uint32_t k0, const uint32_t *env_ids, const int32_t *n_agents,
                     int n_envs, const int64_t *wealth0, const double *feat0, const int32_t *t0,
                     int n_steps, int episode_limit,
                     /* [n_steps][n_slots] (obs [n_steps][n_slots][16]) */
                     double *obs, int32_t *action, double *logp, double *reward, uint8_t *done,
                     int64_t *wealth_rec, double *act_margin,
                     /* final state in slot layout (agents only) */
                     int64_t *wealth_out, double *feat_out, int32_t *t_out) {
  long n_agent_slots = 0;
  for (int e = 0; e < n_envs; ++e) n_agent_slots += n_agents[e];
  long n_slots = n_agent_slots + n_envs;
  long off = 0;
  for (int e = 0; e < n_envs; ++e) {
    int n = n_agents[e];
    uint32_t env = env_ids[e];
    int64_t *w = (int64_t *)malloc(sizeof(int64_t) * n);
    double *f = (double *)malloc(sizeof(double) * n * OR_ECON_F);
    int t = t0 ? t0[e] : 0;
    for (int i = 0; i < n; ++i) {
      if (wealth0) {
        w[i] = wealth0[off + i];
        for (int j = 0; j < OR_ECON_F; ++j) f[(long)i * OR_ECON_F + j] = feat0[(off + i) * OR_ECON_F + j];
      } else {
        or_econ_reset_agent(seed, OR_STEP_INIT, env, (uint32_t)i, &w[i], f + (long)i * OR_ECON_F);
      }
    }
    for (int s = 0; s < n_steps; ++s) {
      long base = (long)s * n_slots;
      long ps = base + n_agent_slots + e;
      or_econ_env_step(agent_params, planner_params, bf16_layers, seed, k0 + (uint32_t)s, env, n,
                       episode_limit, w, f, &t, obs ? obs + (base + off) * OR_ECON_F : NULL,
                       action + base + off, logp + base + off, reward + base + off, done + base + off,
                       wealth_rec + base + off, act_margin ? act_margin + base + off : NULL,
                       obs ? obs + ps * OR_ECON_F : NULL, action + ps, logp + ps, reward + ps,
                       done + ps, wealth_rec + ps, act_margin ? act_margin + ps : NULL);
    }
    for (int i = 0; i < n; ++i) {
      if (wealth_out) wealth_out[off + i] = w[i];
      if (feat_out)
        for (int j = 0; j < OR_ECON_F; ++j) feat_out[(off + i) * OR_ECON_F + j] = f[(long)i * OR_ECON_F + j];
    }
    if (t_out) t_out[e] = t;
    free(w);
    free(f);
    off += n;
  }
}

/* ------------------------------------------------------------------------ */
/* Reaction-path landscape (stand-in for the first-principles potential     */
/* energy landscape of App. C "Catalytic Reactions": the environment is a   */
/* function of the coordinates alone).                                      */
/*   E(x) = sum_m a_m exp(-|x - c_m|^2 / (2 w_m^2))                         */
/* centres U[-3,3]^D, widths lognormal(0, 0.3), amplitudes N(0,1); the      */
/* observed energy adds sigma * N(0,1) noise; reward = E_obs(x) - E_obs(x').*/
/* ------------------------------------------------------------------------ */
/* Gaussian m (ctr0 = m): subs 0..ceil(D/4)-1 give the centre coordinates, 4
 * per draw; sub 64 gives the width exp(0.3 z) from the cos branch of the
 * first word pair and the amplitude z from the cos branch of the second. */
void or_landscape_init(uint64_t param_seed, int D, int M, double *centres, double *widths,
                       double *amps) {
  for (int m = 0; m < M; ++m) {
    uint32_t w[4];
    for (int j = 0; j < D; ++j) {
      if ((j & 3) == 0) or_draw(param_seed, (uint32_t)m, 0, 0, OR_TAG_LANDSCAPE_INIT, (uint32_t)(j >> 2), w);
      centres[(long)m * D + j] = (double)or_uniform_f32(w[j & 3], -3.0f, 3.0f);
    }
    or_draw(param_seed, (uint32_t)m, 0, 0, OR_TAG_LANDSCAPE_INIT, 64, w);
    double z0, z1, z2, z3;
    or_box_muller(w[0], w[1], &z0, &z1);
    or_box_muller(w[2], w[3], &z2, &z3);
    widths[m] = exp(0.3 * z0);
    amps[m] = z2;
  }
}

/* Direct (unexpanded) definition. */
double or_landscape_energy(int D, int M, const double *c, const double *w, const double *a,
                           const double *x) {
  double E = 0.0;
  for (int m = 0; m < M; ++m) {
    double d2 = 0.0;
    for (int j = 0; j < D; ++j) {
      double d = x[j] - c[(long)m * D + j];
      d2 += d * d;
    }
    E += a[m] * exp(-d2 / (2.0 * w[m] * w[m]));
  }
  return E;
}

/* sum_m |a_m| exp(...): the scale against which energy errors are measured. */
double or_landscape_energy_scale(int D, int M, const double *c, const double *w, const double *a,
                                 const double *x) {
  double E = 0.0;
  for (int m = 0; m < M; ++m) {
    double d2 = 0.0;
    for (int j = 0; j < D; ++j) {
      double d = x[j] - c[(long)m * D + j];
      d2 += d * d;
    }
    E += fabs(a[m]) * exp(-d2 / (2.0 * w[m] * w[m]));
  }
  return E;
}

/* Analytic gradient dE/dx_j = -sum_m a_m e_m (x_j - c_mj) / w_m^2. */
void or_landscape_grad(int D, int M, const double *c, const double *w, const double *a,
                       const double *x, double *g) {
  for (int j = 0; j < D; ++j) g[j] = 0.0;
  for (int m = 0; m < M; ++m) {
    double d2 = 0.0;
    for (int j = 0; j < D; ++j) {
      double d = x[j] - c[(long)m * D + j];
      d2 += d * d;
    }
    double e = a[m] * exp(-d2 / (2.0 * w[m] * w[m]));
    for (int j = 0; j < D; ++j) g[j] -= e * (x[j] - c[(long)m * D + j]) / (w[m] * w[m]);
  }
}

/* Normals for the action (ACTION tag, subs 0..ceil(D/4)-1, 4 per draw as two
 * Box-Muller pairs: cos of (w0,w1), sin of (w0,w1), cos of (w2,w3), sin). */
void or_landscape_action_normals(uint64_t seed, uint32_t k, uint32_t env, int D, double *z) {
  uint32_t w[4];
  for (int j = 0; j < D; j += 4) {
    or_draw(seed, k, env, 0, OR_TAG_ACTION, (uint32_t)(j >> 2), w);
    double q[4];
    or_box_muller(w[0], w[1], &q[0], &q[1]);
    or_box_muller(w[2], w[3], &q[2], &q[3]);
    for (int i = 0; i < 4 && j + i < D; ++i) z[j + i] = q[i];
  }
}

/* Observation noise N(0,1): NOISE tag, sub 0 for the post-step state, sub 1
 * for a freshly reset state; cos branch of (w0, w1). */
double or_landscape_noise(uint64_t seed, uint32_t k, uint32_t env, uint32_t sub) {
  uint32_t w[4];
  or_draw(seed, k, env, 0, OR_TAG_NOISE, sub, w);
  double zc, zs;
  or_box_muller(w[0], w[1], &zc, &zs);
  return zc;
}

void or_landscape_reset_draw(uint64_t seed, uint32_t k, uint32_t env, int D, double *x) {
  uint32_t w[4];
  for (int j = 0; j < D; ++j) {
    if ((j & 3) == 0) or_draw(seed, k, env, 0, OR_TAG_RESET, (uint32_t)(j >> 2), w);
    x[j] = (double)or_uniform_f32(w[j & 3], -3.0f, 3.0f);
  }
}

/* Roll out envs env_ids[] for n_steps.  Policy D -> h0 -> h1 -> 2D.  Outputs
 * [n_steps][n_envs] (obs and act [n_steps][n_envs][D]); energy is the pure
 * E of the post-step (pre-reset) state and energy_scale its error scale.
 * An episode ends at the step limit or, when the pure energy of the post-step
 * state falls below energy_target, on reaching the low-energy (product) basin
 * (App. C: an episode runs from the initial to the terminal state of the
 * reaction; -INFINITY turns the energy condition off). */
void or_landscape_rollout(int D, int M, const double *c, const double *wd, const double *am,
                          const float *params, int hidden0, int hidden1, uint32_t bf16_layers,
                          double noise_sigma, double step_clip, uint64_t seed, uint32_t k0,
                          const uint32_t *env_ids, int n_envs, const double *x0,
                          const double *eobs0, const int32_t *t0, int n_steps, int episode_limit,
                          double energy_target, double *obs, double *act, double *logp, double *reward, uint8_t *done,
                          double *energy, double *energy_scale, double *x_out, double *eobs_out,
                          int32_t *t_out) {
  int32_t widths[4] = {D, hidden0, hidden1, 2 * D};
  double *x = (double *)malloc(sizeof(double) * D);
  double *x2 = (double *)malloc(sizeof(double) * D);
  double *out = (double *)malloc(sizeof(double) * 2 * D);
  double *z = (double *)malloc(sizeof(double) * D);
  double *dx = (double *)malloc(sizeof(double) * D);
  for (int e = 0; e < n_envs; ++e) {
    uint32_t env = env_ids[e];
    double eobs;
    int t = t0 ? t0[e] : 0;
    if (x0) {
      for (int j = 0; j < D; ++j) x[j] = x0[(long)e * D + j];
      eobs = eobs0[e];
    } else {
      or_landscape_reset_draw(seed, OR_STEP_INIT, env, D, x);
      eobs = or_landscape_energy(D, M, c, wd, am, x) +
             noise_sigma * or_landscape_noise(seed, OR_STEP_INIT, env, 1);
    }
    for (int s = 0; s < n_steps; ++s) {
      uint32_t k = k0 + (uint32_t)s;
      long r = (long)s * n_envs + e;
      or_mlp_forward(3, widths, params, bf16_layers, x, out);
      or_landscape_action_normals(seed, k, env, D, z);
      double lp;
      or_gaussian_action(D, out, z, step_clip, dx, &lp);
      for (int j = 0; j < D; ++j) x2[j] = x[j] + dx[j];
      double E2 = or_landscape_energy(D, M, c, wd, am, x2);
      double eobs2 = E2 + noise_sigma * or_landscape_noise(seed, k, env, 0);
      if (obs)
        for (int j = 0; j < D; ++j) obs[r * D + j] = x[j];
      if (act)
        for (int j = 0; j < D; ++j) act[r * D + j] = dx[j];
      if (logp) logp[r] = lp;
      if (reward) reward[r] = eobs - eobs2;
      if (energy) energy[r] = E2;
      if (energy_scale) energy_scale[r] = or_landscape_energy_scale(D, M, c, wd, am, x2);
      t = t + 1;
      int dn = t >= episode_limit || E2 < energy_target;
      if (done) done[r] = (uint8_t)dn;
      if (dn) {
        or_landscape_reset_draw(seed, k, env, D, x);
        eobs = or_landscape_energy(D, M, c, wd, am, x) + noise_sigma * or_landscape_noise(seed, k, env, 1);
        t = 0;
      } else {
        for (int j = 0; j < D; ++j) x[j] = x2[j];
        eobs = eobs2;
      }
    }
    if (x_out)
      for (int j = 0; j < D; ++j) x_out[(long)e * D + j] = x[j];
    if (eobs_out) eobs_out[e] = eobs;
    if (t_out) t_out[e] = t;
  }
  free(x);
  free(x2);
  free(out);
  free(z);
  free(dx);
}

/* ------------------------------------------------------------------------ */
/* Actor-critic update on recorded transitions (paper Sec. 2 and App. B: the */
/* roll-out store feeds training on the GPU).  Advantage actor-critic with   */
/* Monte-Carlo returns [reading]: the actor is the roll-out policy          */
/* (categorical head), the critic an MLP of the same widths with one output. */
/* Over the R recorded rows (obs s_i, action a_i, return G_i):               */
/*   A_i = G_i - V(s_i)              (a constant in the actor's loss)        */
/*   L   = (1/R) sum_i [ -A_i log pi(a_i | s_i) - c_e H(pi(. | s_i))         */
/*                       + c_v (G_i - V(s_i))^2 ]                            */
/* Gradients by the chain rule through the tanh layers, in FP64.            */
/* ------------------------------------------------------------------------ */
typedef struct {
  double *a[4];  /* activations per layer (a[0] = input) */
  double *z[4];  /* pre-activations */
} or_trace;

static void or_trace_alloc(or_trace *t, const int32_t *w) {
  for (int l = 0; l < 4; ++l) {
    t->a[l] = (double *)malloc(sizeof(double) * w[l]);
    t->z[l] = (double *)malloc(sizeof(double) * w[l]);
  }
}
static void or_trace_free(or_trace *t) {
  for (int l = 0; l < 4; ++l) {
    free(t->a[l]);
    free(t->z[l]);
  }
}

/* Forward with every activation kept (three layers, tanh hidden, linear out). */
static void or_mlp_trace(const int32_t *w, const float *params, const double *x, or_trace *t) {
  for (int i = 0; i < w[0]; ++i) t->a[0][i] = x[i];
  long off = 0;
  for (int l = 0; l < 3; ++l) {
    const float *W = params + off, *b = W + (long)w[l] * w[l + 1];
    for (int j = 0; j < w[l + 1]; ++j) {
      double s = (double)b[j];
      for (int i = 0; i < w[l]; ++i) s += t->a[l][i] * (double)W[(long)i * w[l + 1] + j];
      t->z[l + 1][j] = s;
      t->a[l + 1][j] = l == 2 ? s : tanh(s);
    }
    off += (long)w[l] * w[l + 1] + w[l + 1];
  }
}

/* Accumulate into grad the gradient of (dy . output) through the traced pass. */
static void or_mlp_backward(const int32_t *w, const float *params, const or_trace *t,
                            const double *dy, double *grad) {
  int maxw = 0;
  for (int l = 0; l < 4; ++l)
    if (w[l] > maxw) maxw = w[l];
  double *d = (double *)malloc(sizeof(double) * maxw);
  double *dn = (double *)malloc(sizeof(double) * maxw);
  long offs[3], off = 0;
  for (int l = 0; l < 3; ++l) {
    offs[l] = off;
    off += (long)w[l] * w[l + 1] + w[l + 1];
  }
  for (int j = 0; j < w[3]; ++j) d[j] = dy[j];  /* d of layer 3's pre-activation */
  for (int l = 2; l >= 0; --l) {
    const float *W = params + offs[l];
    double *gW = grad + offs[l], *gb = gW + (long)w[l] * w[l + 1];
    for (int j = 0; j < w[l + 1]; ++j) {
      gb[j] += d[j];
      for (int i = 0; i < w[l]; ++i) gW[(long)i * w[l + 1] + j] += t->a[l][i] * d[j];
    }
    if (l > 0) {
      for (int i = 0; i < w[l]; ++i) {
        double s = 0.0;
        for (int j = 0; j < w[l + 1]; ++j) s += (double)W[(long)i * w[l + 1] + j] * d[j];
        dn[i] = s * (1.0 - t->a[l][i] * t->a[l][i]);  /* tanh' = 1 - tanh^2 */
      }
      for (int i = 0; i < w[l]; ++i) d[i] = dn[i];
    }
  }
  free(d);
  free(dn);
}

/* Loss terms and (optionally) gradients.  obs [R][obs_dim], act [R], ret [R];
 * adv [R] may be NULL (then A = G - V from the critic).  grad_actor /
 * grad_critic may be NULL; else they receive dL/dparams (zeroed first).
 * stats: {mean -A log pi, mean (G - V)^2, mean entropy}. */
void or_a2c(int R, int obs_dim, int n_act, int h0, int h1, const float *actor, const float *critic,
            const double *obs, const int32_t *act, const double *ret, const double *adv,
            double c_v, double c_e, double *grad_actor, double *grad_critic, double stats[3]) {
  int32_t wa[4] = {obs_dim, h0, h1, n_act}, wc[4] = {obs_dim, h0, h1, 1};
  long na = 0, nc = 0;
  for (int l = 0; l < 3; ++l) {
    na += (long)wa[l] * wa[l + 1] + wa[l + 1];
    nc += (long)wc[l] * wc[l + 1] + wc[l + 1];
  }
  if (grad_actor) memset(grad_actor, 0, sizeof(double) * na);
  if (grad_critic) memset(grad_critic, 0, sizeof(double) * nc);
  or_trace ta, tc;
  or_trace_alloc(&ta, wa);
  or_trace_alloc(&tc, wc);
  double *p = (double *)malloc(sizeof(double) * n_act);
  double *dl = (double *)malloc(sizeof(double) * n_act);
  double s_pg = 0.0, s_v = 0.0, s_h = 0.0;
  for (int i = 0; i < R; ++i) {
    const double *x = obs + (long)i * obs_dim;
    or_mlp_trace(wa, actor, x, &ta);
    or_mlp_trace(wc, critic, x, &tc);
    const double *lg = ta.a[3];
    double m = lg[0];
    for (int k = 1; k < n_act; ++k)
      if (lg[k] > m) m = lg[k];
    double S = 0.0;
    for (int k = 0; k < n_act; ++k) S += exp(lg[k] - m);
    double H = 0.0;
    for (int k = 0; k < n_act; ++k) {
      p[k] = exp(lg[k] - m) / S;
      H -= p[k] * ((lg[k] - m) - log(S));
    }
    const double V = tc.a[3][0];
    const double A = adv ? adv[i] : ret[i] - V;
    const double logp = (lg[act[i]] - m) - log(S);
    s_pg += -A * logp;
    s_v += (ret[i] - V) * (ret[i] - V);
    s_h += H;
    if (grad_actor) {
      /* d(-A log p_a)/dl_k = A (p_k - [k = a]);
       * d(-c_e H)/dl_k = c_e p_k (log p_k + H) */
      for (int k = 0; k < n_act; ++k) {
        const double lpk = (lg[k] - m) - log(S);
        dl[k] = (A * (p[k] - (k == act[i] ? 1.0 : 0.0)) + c_e * p[k] * (lpk + H)) / R;
      }
      or_mlp_backward(wa, actor, &ta, dl, grad_actor);
    }
    if (grad_critic) {
      double dv = 2.0 * c_v * (V - ret[i]) / R;
      or_mlp_backward(wc, critic, &tc, &dv, grad_critic);
    }
  }
  if (stats) {
    stats[0] = s_pg / R;
    stats[1] = s_v / R;
    stats[2] = s_h / R;
  }
  free(p);
  free(dl);
  or_trace_free(&ta);
  or_trace_free(&tc);
}

/* The same update for the diagonal Gaussian head (landscape): out = (mean,
 * raw log sigma), log sigma = clamp(raw, -5, 2).  On policy, the recorded
 * sample is x = mean + sigma z with the row's normals z [R][D], so at the
 * current parameters log pi(x) = sum_j (-z_j^2 / 2 - log sigma_j - log(2 pi)/2),
 * d log pi / d mean_j = z_j / sigma_j, d log pi / d raw_j = z_j^2 - 1 and
 * H = sum_j (log sigma_j + (1 + log 2 pi) / 2), d H / d raw_j = 1 (both 0 where
 * the clamp holds raw outside (-5, 2)). */
void or_a2c_gauss(int R, int D, int h0, int h1, const float *actor, const float *critic,
                  const double *obs, const double *z, const double *ret, const double *adv,
                  double c_v, double c_e, double *grad_actor, double *grad_critic,
                  double stats[3]) {
  int32_t wa[4] = {D, h0, h1, 2 * D}, wc[4] = {D, h0, h1, 1};
  long na = 0, nc = 0;
  for (int l = 0; l < 3; ++l) {
    na += (long)wa[l] * wa[l + 1] + wa[l + 1];
    nc += (long)wc[l] * wc[l + 1] + wc[l + 1];
  }
  if (grad_actor) memset(grad_actor, 0, sizeof(double) * na);
  if (grad_critic) memset(grad_critic, 0, sizeof(double) * nc);
  or_trace ta, tc;
  or_trace_alloc(&ta, wa);
  or_trace_alloc(&tc, wc);
  double *dl = (double *)malloc(sizeof(double) * 2 * D);
  const double half_log_2pi = 0.5 * log(2.0 * M_PI);
  double s_pg = 0.0, s_v = 0.0, s_h = 0.0;
  for (int i = 0; i < R; ++i) {
    or_mlp_trace(wa, actor, obs + (long)i * D, &ta);
    or_mlp_trace(wc, critic, obs + (long)i * D, &tc);
    const double *out = ta.a[3], *zi = z + (long)i * D;
    const double V = tc.a[3][0];
    const double A = adv ? adv[i] : ret[i] - V;
    double logp = 0.0, H = 0.0;
    for (int j = 0; j < D; ++j) {
      const double raw = out[D + j];
      const double ls = raw < -5.0 ? -5.0 : (raw > 2.0 ? 2.0 : raw);
      const double sig = exp(ls);
      const int free_ls = raw > -5.0 && raw < 2.0;
      logp += -0.5 * zi[j] * zi[j] - ls - half_log_2pi;
      H += ls + 0.5 + half_log_2pi;
      dl[j] = -A * zi[j] / sig / R;
      dl[D + j] = free_ls ? (-A * (zi[j] * zi[j] - 1.0) - c_e) / R : 0.0;
    }
    s_pg += -A * logp;
    s_v += (ret[i] - V) * (ret[i] - V);
    s_h += H;
    if (grad_actor) or_mlp_backward(wa, actor, &ta, dl, grad_actor);
    if (grad_critic) {
      double dv = 2.0 * c_v * (V - ret[i]) / R;
      or_mlp_backward(wc, critic, &tc, &dv, grad_critic);
    }
  }
  if (stats) {
    stats[0] = s_pg / R;
    stats[1] = s_v / R;
    stats[2] = s_h / R;
  }
  free(dl);
  or_trace_free(&ta);
  or_trace_free(&tc);
}

/* ------------------------------------------------------------------------ */
/* Proximal policy optimisation, clipped surrogate [reading]: the same      */
/* actor and critic as or_a2c; the advantage A_i is held from before the    */
/* update (G_i - V(s_i) under the critic as it was), and the roll-out's     */
/* recorded log-probability logp_old_i of its action is the behaviour       */
/* policy.  With rho_i = exp(log pi(a_i | s_i) - logp_old_i):               */
/*   L = (1/R) sum_i [ -min(rho_i A_i, clip(rho_i, 1 - eps, 1 + eps) A_i)   */
/*                     - c_e H(pi(. | s_i)) + c_v (G_i - V(s_i))^2 ]         */
/* The min takes the clipped (constant) term, and rho gets no gradient,     */
/* exactly where A > 0 and rho > 1 + eps or A < 0 and rho < 1 - eps; inside */
/* [1 - eps, 1 + eps] both terms agree and the gradient is d(rho A).        */
/* stats: {mean -min(..), mean (G - V)^2, mean entropy, fraction of rows    */
/*         with |rho - 1| > eps}.                                           */
/* ------------------------------------------------------------------------ */
void or_ppo(int R, int obs_dim, int n_act, int h0, int h1, const float *actor, const float *critic,
            const double *obs, const int32_t *act, const double *ret, const double *adv,
            const double *logp_old, double eps, double c_v, double c_e, double *grad_actor,
            double *grad_critic, double stats[4]) {
  int32_t wa[4] = {obs_dim, h0, h1, n_act}, wc[4] = {obs_dim, h0, h1, 1};
  long na = 0, nc = 0;
  for (int l = 0; l < 3; ++l) {
    na += (long)wa[l] * wa[l + 1] + wa[l + 1];
    nc += (long)wc[l] * wc[l + 1] + wc[l + 1];
  }
  if (grad_actor) memset(grad_actor, 0, sizeof(double) * na);
  if (grad_critic) memset(grad_critic, 0, sizeof(double) * nc);
  or_trace ta, tc;
  or_trace_alloc(&ta, wa);
  or_trace_alloc(&tc, wc);
  double *lp = (double *)malloc(sizeof(double) * n_act);
  double *dl = (double *)malloc(sizeof(double) * n_act);
  double s_pg = 0.0, s_v = 0.0, s_h = 0.0, s_clip = 0.0;
  for (int i = 0; i < R; ++i) {
    const double *x = obs + (long)i * obs_dim;
    or_mlp_trace(wa, actor, x, &ta);
    or_mlp_trace(wc, critic, x, &tc);
    const double *lg = ta.a[3];
    double m = lg[0];
    for (int k = 1; k < n_act; ++k)
      if (lg[k] > m) m = lg[k];
    double S = 0.0;
    for (int k = 0; k < n_act; ++k) S += exp(lg[k] - m);
    double H = 0.0;
    for (int k = 0; k < n_act; ++k) {
      lp[k] = (lg[k] - m) - log(S);
      H -= exp(lp[k]) * lp[k];
    }
    const double A = adv[i], V = tc.a[3][0];
    const double rho = exp(lp[act[i]] - logp_old[i]);
    const double rc = rho < 1.0 - eps ? 1.0 - eps : (rho > 1.0 + eps ? 1.0 + eps : rho);
    const double surr = rho * A < rc * A ? rho * A : rc * A;
    const int held = (A > 0.0 && rho > 1.0 + eps) || (A < 0.0 && rho < 1.0 - eps);
    s_pg += -surr;
    s_v += (ret[i] - V) * (ret[i] - V);
    s_h += H;
    s_clip += fabs(rho - 1.0) > eps ? 1.0 : 0.0;
    if (grad_actor) {
      /* d(-rho A)/dl_k = A rho (p_k - [k = a]);  d(-c_e H)/dl_k = c_e p_k (log p_k + H) */
      for (int k = 0; k < n_act; ++k) {
        const double pk = exp(lp[k]);
        const double g_pg = held ? 0.0 : A * rho * (pk - (k == act[i] ? 1.0 : 0.0));
        dl[k] = (g_pg + c_e * pk * (lp[k] + H)) / R;
      }
      or_mlp_backward(wa, actor, &ta, dl, grad_actor);
    }
    if (grad_critic) {
      double dv = 2.0 * c_v * (V - ret[i]) / R;
      or_mlp_backward(wc, critic, &tc, &dv, grad_critic);
    }
  }
  if (stats) {
    stats[0] = s_pg / R;
    stats[1] = s_v / R;
    stats[2] = s_h / R;
    stats[3] = s_clip / R;
  }
  free(lp);
  free(dl);
  or_trace_free(&ta);
  or_trace_free(&tc);
}

/* PPO for the diagonal Gaussian head (landscape) [reading]: the behaviour */
/* sample u [R][D] is the unclipped mean + sigma z of the policy held at   */
/* the advantage pass, logp_old its recorded log-density; at the current   */
/* parameters y_j = (u_j - mean_j) / sigma_j and                            */
/*   log pi(u) = sum_j (-y_j^2 / 2 - log sigma_j - log(2 pi) / 2),          */
/*   d log pi / d mean_j = y_j / sigma_j, d log pi / d raw_j = y_j^2 - 1,   */
/* with H and the clamp of log sigma as in or_a2c_gauss; the surrogate, the */
/* held side of the clip and the stats as in or_ppo.                        */
void or_ppo_gauss(int R, int D, int h0, int h1, const float *actor, const float *critic,
                  const double *obs, const double *u, const double *ret, const double *adv,
                  const double *logp_old, double eps, double c_v, double c_e, double *grad_actor,
                  double *grad_critic, double stats[4]) {
  int32_t wa[4] = {D, h0, h1, 2 * D}, wc[4] = {D, h0, h1, 1};
  long na = 0, nc = 0;
  for (int l = 0; l < 3; ++l) {
    na += (long)wa[l] * wa[l + 1] + wa[l + 1];
    nc += (long)wc[l] * wc[l + 1] + wc[l + 1];
  }
  if (grad_actor) memset(grad_actor, 0, sizeof(double) * na);
  if (grad_critic) memset(grad_critic, 0, sizeof(double) * nc);
  or_trace ta, tc;
  or_trace_alloc(&ta, wa);
  or_trace_alloc(&tc, wc);
  double *y = (double *)malloc(sizeof(double) * D);
  double *sg = (double *)malloc(sizeof(double) * D);
  double *dl = (double *)malloc(sizeof(double) * 2 * D);
  const double half_log_2pi = 0.5 * log(2.0 * M_PI);
  double s_pg = 0.0, s_v = 0.0, s_h = 0.0, s_clip = 0.0;
  for (int i = 0; i < R; ++i) {
    or_mlp_trace(wa, actor, obs + (long)i * D, &ta);
    or_mlp_trace(wc, critic, obs + (long)i * D, &tc);
    const double *out = ta.a[3], *ui = u + (long)i * D;
    double logp = 0.0, H = 0.0;
    for (int j = 0; j < D; ++j) {
      const double raw = out[D + j];
      const double ls = raw < -5.0 ? -5.0 : (raw > 2.0 ? 2.0 : raw);
      sg[j] = exp(ls);
      y[j] = (ui[j] - out[j]) / sg[j];
      logp += -0.5 * y[j] * y[j] - ls - half_log_2pi;
      H += ls + 0.5 + half_log_2pi;
    }
    const double A = adv[i], V = tc.a[3][0];
    const double rho = exp(logp - logp_old[i]);
    const double rc = rho < 1.0 - eps ? 1.0 - eps : (rho > 1.0 + eps ? 1.0 + eps : rho);
    const double surr = rho * A < rc * A ? rho * A : rc * A;
    const int held = (A > 0.0 && rho > 1.0 + eps) || (A < 0.0 && rho < 1.0 - eps);
    const double gA = held ? 0.0 : A * rho;  /* d(-surrogate)/d log pi = -gA */
    s_pg += -surr;
    s_v += (ret[i] - V) * (ret[i] - V);
    s_h += H;
    s_clip += fabs(rho - 1.0) > eps ? 1.0 : 0.0;
    if (grad_actor) {
      for (int j = 0; j < D; ++j) {
        const double raw = out[D + j];
        const int free_ls = raw > -5.0 && raw < 2.0;
        dl[j] = -gA * y[j] / sg[j] / R;
        dl[D + j] = free_ls ? (-gA * (y[j] * y[j] - 1.0) - c_e) / R : 0.0;
      }
      or_mlp_backward(wa, actor, &ta, dl, grad_actor);
    }
    if (grad_critic) {
      double dv = 2.0 * c_v * (V - ret[i]) / R;
      or_mlp_backward(wc, critic, &tc, &dv, grad_critic);
    }
  }
  if (stats) {
    stats[0] = s_pg / R;
    stats[1] = s_v / R;
    stats[2] = s_h / R;
    stats[3] = s_clip / R;
  }
  free(y);
  free(sg);
  free(dl);
  or_trace_free(&ta);
  or_trace_free(&tc);
}

/* ------------------------------------------------------------------------ */
/* Discounted returns over a window of n_steps records ([n_steps][n_slots]):*/
/*   G_t = r_t + gamma (1 - d_t) G_{t+1},  G_{n_steps} = 0.                 */
/* ------------------------------------------------------------------------ */
void or_returns(int n_steps, long n_slots, const double *reward, const uint8_t *done, double gamma,
                double *G) {
  for (long s = 0; s < n_slots; ++s) {
    double g = 0.0;
    for (int t = n_steps - 1; t >= 0; --t) {
      long r = (long)t * n_slots + s;
      g = reward[r] + gamma * (done[r] ? 0.0 : 1.0) * g;
      G[r] = g;
    }
  }
}
