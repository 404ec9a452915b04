// ws_train.cu -- actor-critic update consuming the trajectory ring in place
// (ws_a2c_update, ws_advantages, ws_ppo_update).
//
// Paper grounding: Sec. 2 and App. B keep roll-out and training on the GPU,
// the roll-out store feeding the trainer with no host round trip.  The update
// is advantage actor-critic with Monte-Carlo returns: the actor is the roll-out
// policy (categorical head, or the landscape's diagonal Gaussian head), the
// critic an MLP of the same hidden widths with one output, held in the context;
// the economy's agents and planners are two such pairs, each on its own slots.  Over the R = n_steps x n_slots recorded
// rows (observation s, action a, return G from the returns scan):
//   A = G - V(s) (a constant of the actor's loss),
//   L = (1/R) sum [ -A log pi(a|s) - c_e H(pi(.|s)) + c_v (G - V(s))^2 ],
// then one SGD step on both networks.  PPO (clipped surrogate): the advantage
// A = G - V(s) is computed once (ws_advantages, into the ring's ADVANTAGE
// field) and held; each epoch replaces -A log pi with -min(rho A,
// clip(rho, 1 - eps, 1 + eps) A), rho = pi(a|s) / exp(recorded logp), whose
// gradient is A rho d log pi except where the min holds the clipped constant;
// the Gaussian head's action is the unclipped sample mean + sigma z rebuilt by
// ws_advantages (the SAMPLE field), scored under the current mean and sigma.
//
// FP32 SIMT throughout, in chunks of kTrainChunk rows: gather the chunk's rows from
// the ring, forward both MLPs keeping the activations, the loss head
// (softmax, advantage, dL/dlogits, dL/dV), then the backward pass per layer:
// weight gradients as row-sliced partial products summed in a fixed order
// (deterministic), data gradients through W^T and tanh' = 1 - tanh^2.
#include "ws_kernels.cuh"

namespace ws {

namespace {

constexpr int kSliceRows = 1024;   // rows per weight-gradient partial (128 x 128 GEMM)
constexpr int kThinSlice = 128;    // rows per partial of the thin kernels (more blocks)

// Ring offset (row of step, slot) of row i of the chunk starting at global
// row q0 of a group: step index t and slot slot0 + s with q = t * ns + s over
// the last n steps.
__device__ __forceinline__ size_t ring_pos(const Dev &d, uint32_t n, size_t q0, uint32_t i,
                                           uint32_t slot0, uint32_t ns, size_t *rowR) {
  const size_t q = q0 + i;
  const uint64_t k = d.k[0] - n + q / ns;
  *rowR = (size_t)(k % d.ring_steps);
  return slot0 + q % ns;
}

// The chunk's rows from the ring: obs, return, action (categorical), and for
// PPO the held advantage and the recorded log-probability.
__global__ void k_a2c_gather(Dev d, uint32_t n, size_t q0, uint32_t rows, uint32_t slot0,
                             uint32_t ns, int od, int ppo, TrainBufs tb) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows) return;
  const size_t S = d.n_slots;
  size_t rowR;
  const size_t s = ring_pos(d, n, q0, i, slot0, ns, &rowR);
  for (int j = 0; j < od; ++j) tb.x[(size_t)i * od + j] = d.r_obs[(rowR * od + j) * S + s];
  tb.ret[i] = d.r_ret[rowR * S + s];
  if (d.env != WS_ENV_LANDSCAPE) tb.act[i] = ((const int32_t *)d.r_act)[rowR * S + s];
  if (ppo) {
    tb.adv[i] = d.r_adv[rowR * S + s];
    tb.lpo[i] = d.r_logp[rowR * S + s];
  }
}

// A = G - V(s) of the chunk's rows into the ADVANTAGE field.
__global__ void k_adv_store(Dev d, uint32_t n, size_t q0, uint32_t rows, uint32_t slot0,
                            uint32_t ns, TrainBufs tb) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows) return;
  size_t rowR;
  const size_t s = ring_pos(d, n, q0, i, slot0, ns, &rowR);
  d.r_adv[rowR * d.n_slots + s] = tb.ret[i] - tb.vout[i];
}

// The Philox normals z[j..j+3] of the Gaussian head's sample of (step k,
// env e), as the sampler drew them: one draw per four coordinates.
__device__ __forceinline__ void action_normals4(const Dev &d, uint32_t k, uint32_t e, int j,
                                                float (&z)[4]) {
  const uint4 r = draw(d.seed, k, d.env_base + e, 0, kTagAction, (uint32_t)(j >> 2));
  const float2 p = box_muller(r.x, r.y), p2 = box_muller(r.z, r.w);
  z[0] = p.x;
  z[1] = p.y;
  z[2] = p2.x;
  z[3] = p2.y;
}

// Landscape: the chunk's behaviour samples u = mean + sigma z (unclipped)
// from the actor's outputs into the SAMPLE field.
__global__ void k_sample_store(Dev d, uint32_t n, size_t q0, uint32_t rows, uint32_t ns,
                               TrainBufs tb) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows) return;
  const int D = (int)d.dim;
  size_t rowR;
  const size_t s = ring_pos(d, n, q0, i, 0, ns, &rowR);
  const size_t q = q0 + i;
  const uint32_t k = (uint32_t)(d.k[0] - n + q / ns), e = (uint32_t)(q % ns);
  const float *o = tb.out + (size_t)i * 2 * D;
  for (int j = 0; j < D; j += 4) {
    float z[4];
    action_normals4(d, k, e, j, z);
    for (int u = 0; u < 4 && j + u < D; ++u) {
      const float ls = fminf(fmaxf(o[D + j + u], -5.0f), 2.0f);
      d.r_sample[(rowR * D + j + u) * d.n_slots + s] = o[j + u] + expf(ls) * z[u];
    }
  }
}

// The loss sums: reduced over the warp first, one atomic per warp (every
// thread of the warp calls it, rows past the end with zeros).
__device__ __forceinline__ void add_stats(const TrainBufs &tb, double a, double b, double c,
                                          double e) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
    e += __shfl_xor_sync(0xffffffffu, e, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(tb.stats + 0, a);
    atomicAdd(tb.stats + 1, b);
    atomicAdd(tb.stats + 2, c);
    atomicAdd(tb.stats + 3, e);
  }
}

// Per row: the advantage, dL/d(policy outputs) and dL/dV (the 1/R of the mean
// folded in), and the three loss terms (double atomics; they are statistics
// only).  Categorical head: softmax of the logits.  Diagonal Gaussian head
// (landscape): outputs (mean, raw log sigma), log sigma = clamp(raw, -5, 2);
// on policy the recorded sample is mean + sigma z with the row's Philox
// normals z (redrawn here as the sampler drew them), so d log pi / d mean =
// z / sigma and d log pi / d raw = z^2 - 1, and dH / d raw = 1, where the
// clamp does not hold raw.
__global__ void k_a2c_head(Dev d, uint32_t n, size_t q0, uint32_t rows, uint32_t ns, int na,
                           double inv_r, float c_v, float c_e, TrainBufs tb) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  double s_pg = 0.0, s_v = 0.0, s_h = 0.0;  // rows past the end add zeros
  if (i < rows && d.env == WS_ENV_LANDSCAPE) {  // one group: every slot
    const int D = (int)d.dim;
    const size_t q = q0 + i;
    const uint32_t k = (uint32_t)(d.k[0] - n + q / ns), e = (uint32_t)(q % ns);
    float *o = tb.out + (size_t)i * 2 * D;
    const float V = tb.vout[i], G = tb.ret[i], A = G - V;
    const float half_log_2pi = 0.91893853320467274f;
    float logp = 0.f, H = 0.f;
    for (int j = 0; j < D; j += 4) {
      float z4[4];
      action_normals4(d, k, e, j, z4);
      for (int u = 0; u < 4 && j + u < D; ++u) {
        const float z = z4[u], raw = o[D + j + u];
        const float ls = fminf(fmaxf(raw, -5.0f), 2.0f);
        const bool free_ls = raw > -5.0f && raw < 2.0f;
        logp += -0.5f * z * z - ls - half_log_2pi;
        H += ls + 0.5f + half_log_2pi;
        o[j + u] = (float)(-A * z / expf(ls) * inv_r);
        o[D + j + u] = free_ls ? (float)((-A * (z * z - 1.f) - c_e) * inv_r) : 0.f;
      }
    }
    tb.vout[i] = (float)(2.0 * c_v * (V - G) * inv_r);
    s_pg = -(double)A * logp;
    s_v = (double)(G - V) * (G - V);
    s_h = H;
  } else if (i < rows) {
    float *lg = tb.out + (size_t)i * na;
    float m = lg[0];
    for (int c = 1; c < na; ++c) m = fmaxf(m, lg[c]);
    float S = 0.f;
    for (int c = 0; c < na; ++c) S += expf(lg[c] - m);
    const float lS = logf(S);
    float H = 0.f;
    for (int c = 0; c < na; ++c) {
      const float lp = (lg[c] - m) - lS;
      H -= expf(lp) * lp;
    }
    const float V = tb.vout[i], G = tb.ret[i], A = G - V;
    const int a = tb.act[i];
    const float lpa = (lg[a] - m) - lS;
    for (int c = 0; c < na; ++c) {
      const float lp = (lg[c] - m) - lS, p = expf(lp);
      lg[c] = (float)((A * (p - (c == a ? 1.f : 0.f)) + c_e * p * (lp + H)) * inv_r);
    }
    tb.vout[i] = (float)(2.0 * c_v * (V - G) * inv_r);
    s_pg = -(double)A * lpa;
    s_v = (double)(G - V) * (G - V);
    s_h = H;
  }
  add_stats(tb, s_pg, s_v, s_h, 0.0);
}

// PPO heads.  Per row rho = exp(log pi(a|s) - logp_old), the surrogate
// min(rho A, clip(rho) A), and dL/d(outputs) = -g d log pi / d(outputs) with
// g = A rho, or 0 where A > 0 and rho > 1 + eps or A < 0 and rho < 1 - eps
// (the min then holds the clipped constant), plus the entropy term; dL/dV as
// the A2C head; the sums of -surrogate, (G - V)^2, H and the rows with
// |rho - 1| > eps.  Categorical: d log pi / d logits = onehot(a) - p.
// Diagonal Gaussian (landscape): the action is the SAMPLE field's u, y =
// (u - mean) / sigma, d log pi / d mean = y / sigma, d log pi / d raw = y^2 - 1
// and dH / d raw = 1 where the clamp of log sigma to [-5, 2] does not hold.
__device__ __forceinline__ void ppo_ratio(float lp, float lpo, float A, float eps, float &rho,
                                          float &g, double &s_pg, double &s_c) {
  rho = expf(lp - lpo);
  const float rc = fminf(fmaxf(rho, 1.f - eps), 1.f + eps);
  const bool held = (A > 0.f && rho > 1.f + eps) || (A < 0.f && rho < 1.f - eps);
  g = held ? 0.f : A * rho;
  s_pg = -(double)fminf(rho * A, rc * A);
  s_c = fabsf(rho - 1.f) > eps ? 1.0 : 0.0;
}

__global__ void k_ppo_head(Dev d, uint32_t n, size_t q0, uint32_t rows, uint32_t ns, int na,
                           double inv_r, float eps, float c_v, float c_e, TrainBufs tb) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  double s_pg = 0.0, s_v = 0.0, s_h = 0.0, s_c = 0.0;
  if (i < rows && d.env == WS_ENV_LANDSCAPE) {  // one group: every slot
    const int D = (int)d.dim;
    size_t rowR;
    const size_t s = ring_pos(d, n, q0, i, 0, ns, &rowR);
    float *o = tb.out + (size_t)i * 2 * D;
    const float half_log_2pi = 0.91893853320467274f;
    float lp = 0.f, H = 0.f;
    for (int j = 0; j < D; ++j) {
      const float ls = fminf(fmaxf(o[D + j], -5.0f), 2.0f);
      const float y = (d.r_sample[(rowR * D + j) * d.n_slots + s] - o[j]) / expf(ls);
      lp += -0.5f * y * y - ls - half_log_2pi;
      H += ls + 0.5f + half_log_2pi;
    }
    const float V = tb.vout[i], G = tb.ret[i], A = tb.adv[i];
    float rho, g;
    ppo_ratio(lp, tb.lpo[i], A, eps, rho, g, s_pg, s_c);
    for (int j = 0; j < D; ++j) {
      const float raw = o[D + j];
      const float ls = fminf(fmaxf(raw, -5.0f), 2.0f), sig = expf(ls);
      const float y = (d.r_sample[(rowR * D + j) * d.n_slots + s] - o[j]) / sig;
      const bool free_ls = raw > -5.0f && raw < 2.0f;
      o[j] = (float)(-g * y / sig * inv_r);
      o[D + j] = free_ls ? (float)((-g * (y * y - 1.f) - c_e) * inv_r) : 0.f;
    }
    tb.vout[i] = (float)(2.0 * c_v * (V - G) * inv_r);
    s_v = (double)(G - V) * (G - V);
    s_h = H;
  } else if (i < rows) {
    float *lg = tb.out + (size_t)i * na;
    float m = lg[0];
    for (int c = 1; c < na; ++c) m = fmaxf(m, lg[c]);
    float S = 0.f;
    for (int c = 0; c < na; ++c) S += expf(lg[c] - m);
    const float lS = logf(S);
    float H = 0.f;
    for (int c = 0; c < na; ++c) {
      const float lp = (lg[c] - m) - lS;
      H -= expf(lp) * lp;
    }
    const float V = tb.vout[i], G = tb.ret[i], A = tb.adv[i];
    const int a = tb.act[i];
    float rho, g;
    ppo_ratio((lg[a] - m) - lS, tb.lpo[i], A, eps, rho, g, s_pg, s_c);
    for (int c = 0; c < na; ++c) {
      const float lp = (lg[c] - m) - lS, p = expf(lp);
      lg[c] = (float)((g * (p - (c == a ? 1.f : 0.f)) + c_e * p * (lp + H)) * inv_r);
    }
    tb.vout[i] = (float)(2.0 * c_v * (V - G) * inv_r);
    s_v = (double)(G - V) * (G - V);
    s_h = H;
  }
  add_stats(tb, s_pg, s_v, s_h, s_c);
}

// FP32 GEMM C[M][N] = sum_k A(m, k) B(k, n) over k in [k_lo, k_hi), with
// A(m, k) = TA ? A[k lda + m] : A[m lda + k] and B(k, n) = TB ? B[n ldb + k] :
// B[k ldb + n].  128 x 128 tiles, 8 x 8 outputs per thread (rows ty*4 + {0..3}
// and 64 + ty*4 + {0..3}, columns likewise), K staged 8 at a time through two
// shared-memory buffers.  The FMAs are packed (fma.rn.f32x2: two columns of a
// row per instruction, each lane rounded as a scalar fmaf, in the same k
// order): the A tile is staged as duplicated pairs {a, a}, so one 16-byte
// shared load gives the broadcast operands of two rows.  Epilogues: the forward layer (+ bias, tanh or not),
// the data gradient of a tanh layer (* (1 - H^2)), or none (a partial product
// of row slice z, written at C + z slice_stride).
enum { kEpiBiasTanh = 0, kEpiBias = 1, kEpiDTanh = 2, kEpiNone = 3 };
constexpr int kGM = 128, kGN = 128, kGK = 8, kGT = 256;

// Loads one 4-element vector of an operand tile: along the contiguous dimension
// from (row r, column c) of a matrix with leading dimension ld, valid up to
// r < rmax and c + i < cmax; VEC: one 16-byte load when all four are in range.
template <bool VEC>
__device__ __forceinline__ void ld4(const float *__restrict__ X, long ld, int r, int c, int rmax,
                                    int cmax, float (&v)[4]) {
  const float *p = X + (long)r * ld + c;
  if (VEC && r < rmax && c + 3 < cmax) {
    const float4 q = __ldg((const float4 *)p);
    v[0] = q.x;
    v[1] = q.y;
    v[2] = q.z;
    v[3] = q.w;
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = (r < rmax && c + i < cmax) ? p[i] : 0.f;
  }
}

__device__ __forceinline__ uint64_t fma_f32x2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ float2 unpack_f32x2(uint64_t v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}

template <bool TA, bool TB, int EPI, bool VEC>
__global__ __launch_bounds__(kGT, 2) void k_sgemm(const float *__restrict__ A, int lda,
                                                const float *__restrict__ B, int ldb,
                                                float *__restrict__ C, int M, int N, int k_lo,
                                                int k_hi, int k_slice, size_t slice_stride,
                                                const float *__restrict__ aux) {
  // As holds A(m, k) twice at [k][2m] and [k][2m + 1]; rows padded by 8 (4)
  // floats: the transposing stores of k-contiguous operands (8 k of 4 rows
  // per warp) then fall in distinct banks
  __shared__ __align__(16) float As[2][kGK][2 * kGM + 8];
  __shared__ __align__(16) float Bs[2][kGK][kGN + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.x * kGM, n0 = blockIdx.y * kGN;
  int kb = k_lo, ke = k_hi;
  if (k_slice > 0) {  // weight gradients: block z takes rows [k_lo + z k_slice, +k_slice)
    kb = k_lo + (int)blockIdx.z * k_slice;
    ke = min(k_hi, kb + k_slice);
  }
  // staging: 1,024 elements of each operand per K step, 4 consecutive ones (in
  // memory order) per thread: a k-contiguous operand tile is 128 rows of two
  // 4-vectors, an m- (n-) contiguous one 8 rows of 32 4-vectors
  float ra[4], rb[4];
  auto load = [&](int k0) {
    if (TA)  // A(m, k) = A[k lda + m]
      ld4<VEC>(A, lda, k0 + (tid >> 5), m0 + (tid & 31) * 4, ke, M, ra);
    else     // A(m, k) = A[m lda + k]
      ld4<VEC>(A, lda, m0 + (tid >> 1), k0 + (tid & 1) * 4, M, ke, ra);
    if (TB)  // B(k, n) = B[n ldb + k]
      ld4<VEC>(B, ldb, n0 + (tid >> 1), k0 + (tid & 1) * 4, N, ke, rb);
    else     // B(k, n) = B[k ldb + n]
      ld4<VEC>(B, ldb, k0 + (tid >> 5), n0 + (tid & 31) * 4, ke, N, rb);
  };
  auto store = [&](int buf) {
    if (TA) {
      float *d = &As[buf][tid >> 5][(tid & 31) * 8];
      *(float4 *)d = make_float4(ra[0], ra[0], ra[1], ra[1]);
      *(float4 *)(d + 4) = make_float4(ra[2], ra[2], ra[3], ra[3]);
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i)
        *(float2 *)&As[buf][(tid & 1) * 4 + i][(tid >> 1) * 2] = make_float2(ra[i], ra[i]);
    }
    if (TB) {
#pragma unroll
      for (int i = 0; i < 4; ++i) Bs[buf][(tid & 1) * 4 + i][tid >> 1] = rb[i];
    } else {
      *(float4 *)&Bs[buf][tid >> 5][(tid & 31) * 4] = make_float4(rb[0], rb[1], rb[2], rb[3]);
    }
  };
  // acc[i][p]: row i, columns 2p and 2p + 1 of the thread's eight
  uint64_t acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int p = 0; p < 4; ++p) acc[i][p] = 0ull;
  int buf = 0;
  if (kb < ke) {
    load(kb);
    store(0);
  }
  __syncthreads();
  for (int k0 = kb; k0 < ke; k0 += kGK) {
    const bool more = k0 + kGK < ke;
    if (more) load(k0 + kGK);  // next tile's loads in flight during this tile's FMAs
#pragma unroll
    for (int kk = 0; kk < kGK; ++kk) {
      const ulonglong2 b0 = *(const ulonglong2 *)&Bs[buf][kk][tx * 4];
      const ulonglong2 b1 = *(const ulonglong2 *)&Bs[buf][kk][64 + tx * 4];
      const uint64_t bv[4] = {b0.x, b0.y, b1.x, b1.y};
#pragma unroll
      for (int h = 0; h < 4; ++h) {  // rows 2h, 2h + 1 of the eight: one shared load
        const int r = (h < 2 ? ty * 4 : 64 + ty * 4) + (h & 1) * 2;
        const ulonglong2 a = *(const ulonglong2 *)&As[buf][kk][2 * r];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          acc[2 * h][p] = fma_f32x2(a.x, bv[p], acc[2 * h][p]);
          acc[2 * h + 1][p] = fma_f32x2(a.y, bv[p], acc[2 * h + 1][p]);
        }
      }
    }
    if (more) {
      store(buf ^ 1);
      __syncthreads();
      buf ^= 1;
    }
  }
  float *Cz = C + (k_slice > 0 ? (size_t)blockIdx.z * slice_stride : 0);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int m = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int n = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + j - 4);
      if (n >= N) continue;
      const float2 pr = unpack_f32x2(acc[i][j >> 1]);
      float v = (j & 1) ? pr.y : pr.x;
      if (EPI == kEpiBiasTanh) v = tanhf(v + aux[n]);
      if (EPI == kEpiBias) v = v + aux[n];
      if (EPI == kEpiDTanh) {
        const float h = aux[(size_t)m * N + n];
        v = v * (1.f - h * h);
      }
      Cz[(size_t)m * N + n] = v;
    }
  }
}

// Bias-gradient row of slice z: P[z][M][n] = sum over the slice's rows of
// D[r][n].  A block per (32 columns, slice): the lanes over the columns (each
// row's 32 columns are one coalesced load), warp w over rows rb + w, rb + w +
// 8, ... in order; the eight warp sums are added in warp order.
__global__ __launch_bounds__(256) void k_colsum_slices(const float *__restrict__ D,
                                                       float *__restrict__ P, int rows, int M,
                                                       int N) {
  __shared__ float part[8][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int n = blockIdx.x * 32 + lane, z = blockIdx.y;
  const int rb = z * kSliceRows, re = min(rows, rb + kSliceRows);
  float s = 0.f;
  if (n < N) {
#pragma unroll 8
    for (int r = rb + w; r < re; r += 8) s += D[(size_t)r * N + n];
  }
  part[w][lane] = s;
  __syncthreads();
  if (w == 0 && n < N) {
    float t = part[0][lane];
#pragma unroll
    for (int q = 1; q < 8; ++q) t += part[q][lane];
    P[((size_t)z * (M + 1) + M) * N + n] = t;
  }
}

// Thin layers (32 or fewer outputs, or 32 or fewer inputs) would leave most of
// a 128 x 128 tile idle; they get their own kernels.
constexpr int kThin = 32;

// The thin kernels are instantiated for the narrow width rounded up to a power
// of two (NT or MT >= the true width), so that their per-row work is that of
// the layer, not of the widest thin layer.
inline int thin_width(int v) { return v <= 1 ? 1 : v <= 2 ? 2 : v <= 4 ? 4 : v <= 8 ? 8 : v <= 16 ? 16 : 32; }

// Forward of a layer with N <= NT outputs: a warp per row, the lanes over the
// inputs, a fixed-order warp reduction per output.
template <bool TANH, int NT>
__global__ void k_fwd_thin(const float *__restrict__ X, const float *__restrict__ W,
                           const float *__restrict__ b, float *__restrict__ Y, int rows, int K,
                           int N) {
  const int r = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (r >= rows) return;  // whole warps leave together
  float acc[NT];
#pragma unroll
  for (int n = 0; n < NT; ++n) acc[n] = 0.f;
  int k = lane;
  for (; k + 96 < K; k += 128) {  // four of the lane's inputs in flight, the sums in k order
    float x[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) x[u] = X[(size_t)r * K + k + 32 * u];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int n = 0; n < NT; ++n)
        if (n < N) acc[n] = fmaf(x[u], W[(size_t)(k + 32 * u) * N + n], acc[n]);
  }
  for (; k < K; k += 32) {
    const float x = X[(size_t)r * K + k];
#pragma unroll
    for (int n = 0; n < NT; ++n)
      if (n < N) acc[n] = fmaf(x, W[(size_t)k * N + n], acc[n]);
  }
#pragma unroll
  for (int n = 0; n < NT; ++n) {
    if (n >= N) break;
    float v = acc[n];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) Y[(size_t)r * N + n] = TANH ? tanhf(v + b[n]) : v + b[n];
  }
}

// Forward of a layer with K <= KT inputs and a wide output: a thread per
// output column n (its K weights and bias in registers), kFwdRows rows per
// block with their inputs staged in shared memory; the sum runs over k in
// order from 0 and then adds the bias, as the GEMM's epilogue does.
constexpr int kFwdRows = 32;
template <bool TANH, int KT>
__global__ __launch_bounds__(256) void k_fwd_thin_k(const float *__restrict__ X,
                                                    const float *__restrict__ W,
                                                    const float *__restrict__ b,
                                                    float *__restrict__ Y, int rows, int K, int N) {
  __shared__ float Xs[kFwdRows][KT];
  const int n = blockIdx.x * blockDim.x + threadIdx.x, r0 = blockIdx.y * kFwdRows;
  for (int idx = threadIdx.x; idx < kFwdRows * KT; idx += blockDim.x) {
    const int rr = idx / KT, k = idx % KT;
    Xs[rr][k] = (r0 + rr < rows && k < K) ? X[(size_t)(r0 + rr) * K + k] : 0.f;
  }
  __syncthreads();
  if (n >= N) return;
  float w[KT];
#pragma unroll
  for (int k = 0; k < KT; ++k) w[k] = k < K ? W[(size_t)k * N + n] : 0.f;
  const float bn = b[n];
  const int nr = min(kFwdRows, rows - r0);
  int rr = 0;
  for (; rr + 4 <= nr; rr += 4) {  // four independent rows in flight
    float acc[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      acc[u] = 0.f;
#pragma unroll
      for (int k = 0; k < KT; ++k)
        if (k < K) acc[u] = fmaf(Xs[rr + u][k], w[k], acc[u]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) Y[(size_t)(r0 + rr + u) * N + n] = TANH ? tanhf(acc[u] + bn) : acc[u] + bn;
  }
  for (; rr < nr; ++rr) {
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k < KT; ++k)
      if (k < K) acc = fmaf(Xs[rr][k], w[k], acc);
    Y[(size_t)(r0 + rr) * N + n] = TANH ? tanhf(acc + bn) : acc + bn;
  }
}

// Data gradient through a layer with K <= KT outputs into its M inputs:
// out[r][m] = (sum_k D[r][k] W[m][k]) (1 - H[r][m]^2), a thread per input m
// (its K weights in registers), kFwdRows rows per block with their D rows
// staged in shared memory; the sum over k in order from 0, as the GEMM's.
template <int KT>
__global__ __launch_bounds__(256) void k_dgrad_thin_k(const float *__restrict__ D,
                                                      const float *__restrict__ W,
                                                      const float *__restrict__ H,
                                                      float *__restrict__ out, int rows, int K,
                                                      int M) {
  __shared__ float Ds[kFwdRows][KT];
  const int m = blockIdx.x * blockDim.x + threadIdx.x, r0 = blockIdx.y * kFwdRows;
  for (int idx = threadIdx.x; idx < kFwdRows * KT; idx += blockDim.x) {
    const int rr = idx / KT, k = idx % KT;
    Ds[rr][k] = (r0 + rr < rows && k < K) ? D[(size_t)(r0 + rr) * K + k] : 0.f;
  }
  __syncthreads();
  if (m >= M) return;
  float w[KT];
#pragma unroll
  for (int k = 0; k < KT; ++k) w[k] = k < K ? W[(size_t)m * K + k] : 0.f;
  const int nr = min(kFwdRows, rows - r0);
  for (int rr = 0; rr < nr; ++rr) {
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k < KT; ++k)
      if (k < K) acc = fmaf(Ds[rr][k], w[k], acc);
    const size_t o = (size_t)(r0 + rr) * M + m;
    const float h = H[o];
    out[o] = acc * (1.f - h * h);
  }
}

// Weight gradient of a layer with N <= NT outputs, slice z: P[z][m][n] for
// every input m (and the bias row m = M): a thread per m, the slice's D rows
// staged through shared memory 64 at a time.
template <int NT>
__global__ __launch_bounds__(256) void k_wgrad_thin_n(const float *__restrict__ Ain,
                                                      const float *__restrict__ D,
                                                      float *__restrict__ P, int rows, int M,
                                                      int N) {
  __shared__ float Ds[64][NT];
  const int m = blockIdx.x * blockDim.x + threadIdx.x, z = blockIdx.y;
  const int rb = z * kThinSlice, re = min(rows, rb + kThinSlice);
  float acc[NT];
#pragma unroll
  for (int n = 0; n < NT; ++n) acc[n] = 0.f;
  for (int r0 = rb; r0 < re; r0 += 64) {
    const int nr = min(64, re - r0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < 64 * NT; idx += blockDim.x) {
      const int rr = idx / NT, n = idx % NT;
      Ds[rr][n] = (rr < nr && n < N) ? D[(size_t)(r0 + rr) * N + n] : 0.f;
    }
    __syncthreads();
    if (m <= M) {
      int rr = 0;
      for (; rr + 8 <= nr; rr += 8) {  // eight rows' loads in flight, the sums in row order
        float a[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) a[u] = m == M ? 1.f : Ain[(size_t)(r0 + rr + u) * M + m];
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
          for (int n = 0; n < NT; ++n) acc[n] = fmaf(a[u], Ds[rr + u][n], acc[n]);
      }
      for (; rr < nr; ++rr) {
        const float a = m == M ? 1.f : Ain[(size_t)(r0 + rr) * M + m];
#pragma unroll
        for (int n = 0; n < NT; ++n) acc[n] = fmaf(a, Ds[rr][n], acc[n]);
      }
    }
  }
  if (m > M) return;
  float *out = P + (size_t)z * (M + 1) * N + (size_t)m * N;
#pragma unroll
  for (int n = 0; n < NT; ++n)
    if (n < N) out[n] = acc[n];
}

// Weight gradient of a layer with M <= MT inputs, slice z: P[z][m][n] for every
// output n, all m (and the bias row): a thread per n, the slice's input rows
// staged through shared memory 64 at a time.
template <int MT>
__global__ __launch_bounds__(256) void k_wgrad_thin_m(const float *__restrict__ Ain,
                                                      const float *__restrict__ D,
                                                      float *__restrict__ P, int rows, int M,
                                                      int N) {
  __shared__ float As[64][MT + 1];
  const int n = blockIdx.x * blockDim.x + threadIdx.x, z = blockIdx.y;
  const int rb = z * kThinSlice, re = min(rows, rb + kThinSlice);
  float acc[MT + 1];
#pragma unroll
  for (int m = 0; m <= MT; ++m) acc[m] = 0.f;
  for (int r0 = rb; r0 < re; r0 += 64) {
    const int nr = min(64, re - r0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < 64 * (MT + 1); idx += blockDim.x) {
      const int rr = idx / (MT + 1), m = idx % (MT + 1);
      As[rr][m] = (rr < nr && m < M) ? Ain[(size_t)(r0 + rr) * M + m] : (rr < nr && m == M ? 1.f : 0.f);
    }
    __syncthreads();
    if (n < N) {
      int rr = 0;
      for (; rr + 8 <= nr; rr += 8) {  // eight rows' loads in flight, the sums in row order
        float dv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) dv[u] = D[(size_t)(r0 + rr + u) * N + n];
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
          for (int m = 0; m <= MT; ++m) acc[m] = fmaf(As[rr + u][m], dv[u], acc[m]);
      }
      for (; rr < nr; ++rr) {
        const float dv = D[(size_t)(r0 + rr) * N + n];
#pragma unroll
        for (int m = 0; m <= MT; ++m) acc[m] = fmaf(As[rr][m], dv, acc[m]);
      }
    }
  }
  if (n >= N) return;
  float *out = P + (size_t)z * (M + 1) * N + n;
#pragma unroll
  for (int m = 0; m <= MT; ++m)
    if (m <= M) out[(size_t)m * N] = acc[m];
}

// Launch a thin kernel instantiated for thin_width(w).
#define WS_THIN_DISPATCH(w, LAUNCH) \
  switch (thin_width(w)) {          \
    case 1: LAUNCH(1); break;       \
    case 2: LAUNCH(2); break;       \
    case 4: LAUNCH(4); break;       \
    case 8: LAUNCH(8); break;       \
    case 16: LAUNCH(16); break;     \
    default: LAUNCH(32); break;     \
  }

// grad[i] += sum_z P[z][i] in a fixed order: a block per 32 consecutive i (the
// lanes), warp w summing slices z = w, w + 8, ... in order, then the eight
// warp sums added to grad[i] in warp order.
__global__ __launch_bounds__(256) void k_reduce_slices(const float *__restrict__ P, int nz,
                                                       size_t len, float *grad) {
  __shared__ float part[8][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const size_t i = (size_t)blockIdx.x * 32 + lane;
  float s = 0.f;
  if (i < len) {
#pragma unroll 8
    for (int z = w; z < nz; z += 8) s += P[(size_t)z * len + i];
  }
  part[w][lane] = s;
  __syncthreads();
  if (w == 0 && i < len) {
    float t = grad[i];
#pragma unroll
    for (int q = 0; q < 8; ++q) t += part[q][lane];
    grad[i] = t;
  }
}

__global__ void k_sgd(float *p, const float *g, size_t n, float lr) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = fmaf(-lr, g[i], p[i]);
}

inline unsigned nblk(size_t n, int t) { return (unsigned)((n + t - 1) / t); }

// A layer's weight gradient goes to the thin kernels when it has 32 or fewer
// outputs or inputs; their row slices are shorter.
inline bool thin_layer(int M, int N) { return N <= kThin || M <= kThin; }
inline int slice_rows(int M, int N) { return thin_layer(M, N) ? kThinSlice : kSliceRows; }

// 16-byte loads when both operands' rows start on 16-byte boundaries.
inline bool vec_ok(const void *A, int lda, const void *B, int ldb) {
  return lda % 4 == 0 && ldb % 4 == 0 && ((uintptr_t)A & 15) == 0 && ((uintptr_t)B & 15) == 0;
}

// Launch k_sgemm with the 16-byte-load variant when the operands allow it.
template <bool TA, bool TB, int EPI>
void sgemm(dim3 g, cudaStream_t st, const float *A, int lda, const float *B, int ldb, float *C,
           int M, int N, int k_lo, int k_hi, int k_slice, size_t slice_stride, const float *aux) {
  if (vec_ok(A, lda, B, ldb))
    k_sgemm<TA, TB, EPI, true><<<g, kGT, 0, st>>>(A, lda, B, ldb, C, M, N, k_lo, k_hi, k_slice,
                                                  slice_stride, aux);
  else
    k_sgemm<TA, TB, EPI, false><<<g, kGT, 0, st>>>(A, lda, B, ldb, C, M, N, k_lo, k_hi, k_slice,
                                                   slice_stride, aux);
}

inline dim3 ggrid(int M, int N, int z = 1) {
  return dim3((unsigned)((M + kGM - 1) / kGM), (unsigned)((N + kGN - 1) / kGN), (unsigned)z);
}

// A hidden-layer GEMM of the update: on tcgen05 with FP32 operands split into
// BF16 hi + lo (ws_gemm_tc.cu), or on the FP32 CUDA cores when the launch asks
// for them (ws_launch.update_gemm).  The epilogue codes are shared.
static_assert((int)kEpiBiasTanh == (int)kGemmBiasTanh && (int)kEpiBias == (int)kGemmBias &&
                  (int)kEpiDTanh == (int)kGemmDTanh && (int)kEpiNone == (int)kGemmNone,
              "epilogue codes");
template <bool TA, bool TB, int EPI>
void hgemm(const Dev &d, dim3 g, cudaStream_t st, const float *A, int lda, const float *B, int ldb,
           float *C, int M, int N, int k_lo, int k_hi, int k_slice, size_t slice_stride,
           const float *aux) {
  // a tensor-core launch that is refused (a shape it does not take) falls back
  // to the CUDA-core GEMM
  if (!d.update_simt && launch_gemm_tc(TA, TB, EPI, A, lda, B, ldb, C, M, N, k_lo, k_hi, k_slice,
                                       slice_stride, aux, d.err, st) == cudaSuccess)
    return;
  sgemm<TA, TB, EPI>(g, st, A, lda, B, ldb, C, M, N, k_lo, k_hi, k_slice, slice_stride, aux);
}

// Forward of one three-layer MLP for a chunk (rows x w0 row-major input),
// keeping the tanh activations h1, h2.
void mlp_forward(const Dev &d, const PolicyShape &sh, const float *params, const float *X, float *h1,
                 float *h2, float *out, int rows, cudaStream_t st) {
  const float *in[3] = {X, h1, h2};
  float *o[3] = {h1, h2, out};
  for (int l = 0; l < 3; ++l) {
    const int K = sh.w[l], N = sh.w[l + 1];
    const float *W = params + sh.layer_offset(l), *b = W + (size_t)K * N;
    if (N <= kThin) {
      const unsigned g = nblk((size_t)rows * 32, 256);
#define WS_FWD_TANH(NT) k_fwd_thin<true, NT><<<g, 256, 0, st>>>(in[l], W, b, o[l], rows, K, N)
#define WS_FWD_LIN(NT) k_fwd_thin<false, NT><<<g, 256, 0, st>>>(in[l], W, b, o[l], rows, K, N)
      if (l < 2) {
        WS_THIN_DISPATCH(N, WS_FWD_TANH)
      } else {
        WS_THIN_DISPATCH(N, WS_FWD_LIN)
      }
#undef WS_FWD_TANH
#undef WS_FWD_LIN
    } else if (K <= kThin) {
      const dim3 g(nblk(N, 256), nblk(rows, kFwdRows));
#define WS_FWDK_TANH(KT) k_fwd_thin_k<true, KT><<<g, 256, 0, st>>>(in[l], W, b, o[l], rows, K, N)
#define WS_FWDK_LIN(KT) k_fwd_thin_k<false, KT><<<g, 256, 0, st>>>(in[l], W, b, o[l], rows, K, N)
      if (l < 2) {
        WS_THIN_DISPATCH(K, WS_FWDK_TANH)
      } else {
        WS_THIN_DISPATCH(K, WS_FWDK_LIN)
      }
#undef WS_FWDK_TANH
#undef WS_FWDK_LIN
    } else if (l < 2) {
      hgemm<false, false, kEpiBiasTanh>(d, ggrid(rows, N), st, in[l], K, W, N, o[l], rows, N, 0, K,
                                        0, 0, b);
    } else {
      hgemm<false, false, kEpiBias>(d, ggrid(rows, N), st, in[l], K, W, N, o[l], rows, N, 0, K, 0, 0,
                                    b);
    }
  }
}

// Backward through one three-layer MLP for a chunk: X [rows][w0], h1, h2 the
// tanh activations, dout [rows][w3] the gradient at the output.  Per layer the
// weight gradient as row-slice partials (and the bias row), summed into
// grad in slice order, then the data gradient into the layer below.
void mlp_backward(const Dev &d, const PolicyShape &sh, const float *params, const float *X,
                  const float *h1, const float *h2, const float *dout, float *grad, float *d1, float *d2,
                  float *part, int rows, cudaStream_t st) {
  const float *ain[3] = {X, h1, h2};
  float *dl[3] = {nullptr, d1, d2};
  for (int l = 2; l >= 0; --l) {
    const int M = sh.w[l], N = sh.w[l + 1];
    const int sr = slice_rows(M, N), nz = (rows + sr - 1) / sr;
    const float *D = l == 2 ? dout : dl[l + 1];
    // P[z][m][n] = sum over slice z of Ain[r][m] D[r][n]; the partials of one
    // slice are (M + 1) x N apart so that the bias row fits after them
    const size_t len = (size_t)(M + 1) * N;
    if (N <= kThin) {
      const dim3 g(nblk(M + 1, 256), (unsigned)nz);
#define WS_WG_N(NT) k_wgrad_thin_n<NT><<<g, 256, 0, st>>>(ain[l], D, part, rows, M, N)
      WS_THIN_DISPATCH(N, WS_WG_N)
#undef WS_WG_N
    } else if (M <= kThin) {
      const dim3 g(nblk(N, 256), (unsigned)nz);
#define WS_WG_M(MT) k_wgrad_thin_m<MT><<<g, 256, 0, st>>>(ain[l], D, part, rows, M, N)
      WS_THIN_DISPATCH(M, WS_WG_M)
#undef WS_WG_M
    } else {
      hgemm<true, false, kEpiNone>(d, ggrid(M, N, nz), st, ain[l], M, D, N, part, M, N, 0, rows,
                                   kSliceRows, len, nullptr);
      k_colsum_slices<<<dim3(nblk(N, 32), (unsigned)nz), 256, 0, st>>>(D, part, rows, M, N);
    }
    k_reduce_slices<<<nblk(len, 32), 256, 0, st>>>(part, nz, len, grad + sh.layer_offset(l));
    if (l > 0 && N <= kThin) {
      // gradient at layer l's input pre-activation: (D W_l^T) * (1 - a_l^2)
      const dim3 g(nblk(M, 256), nblk(rows, kFwdRows));
#define WS_DG(KT) k_dgrad_thin_k<KT><<<g, 256, 0, st>>>(D, params + sh.layer_offset(l), ain[l], \
                                                        dl[l], rows, N, M)
      WS_THIN_DISPATCH(N, WS_DG)
#undef WS_DG
    } else if (l > 0) {
      hgemm<false, true, kEpiDTanh>(d, ggrid(rows, M), st, D, N, params + sh.layer_offset(l), N,
                                    dl[l], rows, M, 0, N, 0, 0, ain[l]);
    }
  }
}

// The scratch of one update chunk, carved from base (or, with base null, only
// measured): returns its size in bytes.
size_t train_layout(uint8_t *base, const PolicyShape &pol, TrainBufs *t) {
  const PolicyShape crit{{pol.w[0], pol.w[1], pol.w[2], 1}};
  const size_t CH = kTrainChunk, w0 = pol.w[0], H0 = pol.w[1], H1 = pol.w[2], NA = pol.w[3];
  const size_t hmax = H0 > H1 ? H0 : H1;
  size_t part_len = 0;  // the largest slice-partial set over the layers of both networks
  for (int l = 0; l < kMaxLayers; ++l) {
    const size_t len = (size_t)(pol.w[l] + 1) * pol.w[l + 1];
    const size_t sr = (size_t)slice_rows(pol.w[l], pol.w[l + 1]);
    const size_t v = (CH + sr - 1) / sr * len;
    if (v > part_len) part_len = v;
    const size_t lenc = (size_t)(crit.w[l] + 1) * crit.w[l + 1];
    const size_t src = (size_t)slice_rows(crit.w[l], crit.w[l + 1]);
    const size_t vc = (CH + src - 1) / src * lenc;
    if (vc > part_len) part_len = vc;
  }
  size_t o = 0;
  auto take = [&](size_t n) {
    uint8_t *p = base ? base + o : nullptr;
    o += (n + 63) / 64 * 64;
    return p;
  };
  TrainBufs b{};
  b.x = (float *)take(CH * w0 * 4);
  b.ret = (float *)take(CH * 4);
  b.act = (int32_t *)take(CH * 4);
  b.adv = (float *)take(CH * 4);
  b.lpo = (float *)take(CH * 4);
  b.h1 = (float *)take(CH * H0 * 4);    // actor activations
  b.h2 = (float *)take(CH * H1 * 4);
  b.out = (float *)take(CH * NA * 4);   // logits, then dL/dlogits
  b.c1 = (float *)take(CH * H0 * 4);    // critic activations
  b.c2 = (float *)take(CH * H1 * 4);
  b.vout = (float *)take(CH * 4);       // V, then dL/dV
  b.d1 = (float *)take(CH * hmax * 4);  // data gradients
  b.d2 = (float *)take(CH * hmax * 4);
  b.part = (float *)take(part_len * 4); // weight-gradient partials
  b.stats = (double *)take(4 * 8);
  b.grad = (float *)take((pol.count() + crit.count()) * 4);
  if (t) *t = b;
  return o;
}

}  // namespace

size_t train_scratch_bytes(const PolicyShape &pol) { return train_layout(nullptr, pol, nullptr); }

TrainBufs train_bufs(uint8_t *base, const PolicyShape &pol) {
  TrainBufs t;
  train_layout(base, pol, &t);
  return t;
}

namespace {

// Per group (the economy: agents, then planners; else one group of all
// slots): gradients over the group's rows in chunks, then the SGD step.  ppo
// selects the clipped-surrogate head (eps) over the A2C head.
void run_update(const Dev &d, const TrainBufs &tb, const TrainGroup *groups, int n_groups,
                uint32_t n, float lr, float c_v, float c_e, bool ppo, float eps, cudaStream_t st) {
  cudaMemsetAsync(tb.stats, 0, 4 * 8, st);
  for (int gi = 0; gi < n_groups; ++gi) {
    const TrainGroup &G = groups[gi];
    const size_t R = (size_t)n * G.n_slots;
    const size_t na = G.pol.count(), nc = G.crit.count();
    float *ga = tb.grad, *gc = tb.grad + na;
    cudaMemsetAsync(tb.grad, 0, (na + nc) * 4, st);
    const double inv_r = 1.0 / (double)R;
    for (size_t q0 = 0; q0 < R; q0 += kTrainChunk) {
      const int rows = (int)((R - q0) < (size_t)kTrainChunk ? (R - q0) : (size_t)kTrainChunk);
      k_a2c_gather<<<nblk(rows, 256), 256, 0, st>>>(d, n, q0, (uint32_t)rows, G.slot0, G.n_slots,
                                                    G.pol.w[0], ppo ? 1 : 0, tb);
      mlp_forward(d, G.pol, G.params, tb.x, tb.h1, tb.h2, tb.out, rows, st);
      mlp_forward(d, G.crit, G.critic, tb.x, tb.c1, tb.c2, tb.vout, rows, st);
      if (ppo)
        k_ppo_head<<<nblk(rows, 256), 256, 0, st>>>(d, n, q0, (uint32_t)rows, G.n_slots,
                                                    G.pol.w[3], inv_r, eps, c_v, c_e, tb);
      else
        k_a2c_head<<<nblk(rows, 256), 256, 0, st>>>(d, n, q0, (uint32_t)rows, G.n_slots,
                                                    G.pol.w[3], inv_r, c_v, c_e, tb);
      mlp_backward(d, G.pol, G.params, tb.x, tb.h1, tb.h2, tb.out, ga, tb.d1, tb.d2, tb.part, rows,
                   st);
      mlp_backward(d, G.crit, G.critic, tb.x, tb.c1, tb.c2, tb.vout, gc, tb.d1, tb.d2, tb.part, rows,
                   st);
    }
    k_sgd<<<nblk(na, 256), 256, 0, st>>>(G.params, ga, na, lr);
    k_sgd<<<nblk(nc, 256), 256, 0, st>>>(G.critic, gc, nc, lr);
  }
}

}  // namespace

void launch_a2c_update(const Dev &d, const TrainBufs &tb, const TrainGroup *groups, int n_groups,
                       uint32_t n, float lr, float c_v, float c_e, cudaStream_t st) {
  run_update(d, tb, groups, n_groups, n, lr, c_v, c_e, false, 0.f, st);
}

void launch_ppo_update(const Dev &d, const TrainBufs &tb, const TrainGroup *groups, int n_groups,
                       uint32_t n, float lr, float eps, float c_v, float c_e, cudaStream_t st) {
  run_update(d, tb, groups, n_groups, n, lr, c_v, c_e, true, eps, st);
}

// Per group and chunk: gather, the critic's forward, A = G - V into the ring;
// landscape: the actor's forward and the behaviour samples.
void launch_advantages(const Dev &d, const TrainBufs &tb, const TrainGroup *groups, int n_groups,
                       uint32_t n, cudaStream_t st) {
  for (int gi = 0; gi < n_groups; ++gi) {
    const TrainGroup &G = groups[gi];
    const size_t R = (size_t)n * G.n_slots;
    for (size_t q0 = 0; q0 < R; q0 += kTrainChunk) {
      const int rows = (int)((R - q0) < (size_t)kTrainChunk ? (R - q0) : (size_t)kTrainChunk);
      k_a2c_gather<<<nblk(rows, 256), 256, 0, st>>>(d, n, q0, (uint32_t)rows, G.slot0, G.n_slots,
                                                    G.pol.w[0], 0, tb);
      mlp_forward(d, G.crit, G.critic, tb.x, tb.c1, tb.c2, tb.vout, rows, st);
      k_adv_store<<<nblk(rows, 256), 256, 0, st>>>(d, n, q0, (uint32_t)rows, G.slot0, G.n_slots,
                                                   tb);
      if (d.env == WS_ENV_LANDSCAPE) {  // one group: every slot
        mlp_forward(d, G.pol, G.params, tb.x, tb.h1, tb.h2, tb.out, rows, st);
        k_sample_store<<<nblk(rows, 256), 256, 0, st>>>(d, n, q0, (uint32_t)rows, G.n_slots, tb);
      }
    }
  }
}

}  // namespace ws
