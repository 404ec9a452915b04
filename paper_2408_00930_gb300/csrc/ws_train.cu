// ws_train.cu -- actor-critic update consuming the trajectory ring in place
// (ws_a2c_update).
//
// Paper grounding: Sec. 2 and App. B keep roll-out and training on the GPU,
// the roll-out store feeding the trainer with no host round trip.  The update
// is advantage actor-critic with Monte-Carlo returns: the actor is the roll-out
// policy (categorical head), the critic an MLP of the same hidden widths with
// one output, held in the context.  Over the R = n_steps x n_slots recorded
// rows (observation s, action a, return G from the returns scan):
//   A = G - V(s) (a constant of the actor's loss),
//   L = (1/R) sum [ -A log pi(a|s) - c_e H(pi(.|s)) + c_v (G - V(s))^2 ],
// then one SGD step on both networks.
//
// FP32 SIMT throughout, in chunks of kTrainChunk rows: gather the chunk's rows from
// the ring, forward both MLPs (the per-step path's dense kernel), the loss head
// (softmax, advantage, dL/dlogits, dL/dV), then the backward pass per layer:
// weight gradients as row-sliced partial products summed in a fixed order
// (deterministic), data gradients through W^T and tanh' = 1 - tanh^2.
#include "ws_kernels.cuh"

namespace ws {

namespace {

constexpr int kTB = 64, kTK = 16;  // GEMM tiles: 64 x 64 outputs, K staged 16 at a time
constexpr int kTT = 256;           // threads per GEMM block (4 x 4 outputs each)
constexpr int kSliceRows = 512;    // rows per weight-gradient partial

// Row i of the chunk starting at global row q0: (step index t, slot s) with
// q = t * S + s over the last n steps.
__global__ void k_a2c_gather(Dev d, uint32_t n, size_t q0, uint32_t rows, TrainBufs tb) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows) return;
  const size_t q = q0 + i, S = d.n_slots;
  const uint64_t k = d.k[0] - n + q / S;
  const size_t rowR = (size_t)(k % d.ring_steps), s = q % S;
  const int od = d.pol.w[0];
  for (int j = 0; j < od; ++j) tb.x[(size_t)i * od + j] = d.r_obs[(rowR * od + j) * S + s];
  tb.ret[i] = d.r_ret[rowR * S + s];
  tb.act[i] = ((const int32_t *)d.r_act)[rowR * S + s];
}

// Per row: softmax of the logits, the advantage, dL/dlogits and dL/dV (the
// 1/R of the mean folded in), and the three loss terms (double atomics; they
// are statistics only).
__global__ void k_a2c_head(Dev d, uint32_t rows, double inv_r, float c_v, float c_e, TrainBufs tb) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows) return;
  const int na = d.pol.w[3];
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
  atomicAdd(tb.stats + 0, -(double)A * lpa);
  atomicAdd(tb.stats + 1, (double)(G - V) * (G - V));
  atomicAdd(tb.stats + 2, (double)H);
}

// Y[r][n] = (sum_k Dout[r][k] W[n][k]) * (1 - H[r][n]^2): the gradient at the
// pre-activation of a tanh layer, W stored [n_in = N][n_out = K] row-major.
__global__ __launch_bounds__(kTT) void k_bwd_data(const float *__restrict__ Dout,
                                                   const float *__restrict__ W,
                                                   const float *__restrict__ Hact,
                                                   float *__restrict__ Y, int rows, int K, int N) {
  __shared__ float As[kTK][kTB + 4];
  __shared__ float Bs[kTK][kTB + 4];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const long r0 = (long)blockIdx.x * kTB;
  const int n0 = blockIdx.y * kTB;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += kTK) {
    for (int idx = tid; idx < kTB * kTK; idx += kTT) {
      const int kk = idx % kTK, m = idx / kTK;
      const long r = r0 + m;
      As[kk][m] = (r < rows && k0 + kk < K) ? Dout[r * K + k0 + kk] : 0.f;
      const int nn = n0 + m;
      Bs[kk][m] = (nn < N && k0 + kk < K) ? W[(long)nn * K + k0 + kk] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kTK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const long r = r0 + ty * 4 + i;
    if (r >= rows) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = n0 + tx * 4 + j;
      if (c >= N) continue;
      const float h = Hact[r * N + c];
      Y[r * N + c] = acc[i][j] * (1.f - h * h);
    }
  }
}

// Partial weight gradient of slice z: P[z][m][n] = sum over the slice's rows r
// of Ain[r][m] * Dout[r][n], with row m = M standing for the bias (Ain = 1).
// The layer's parameters are laid out exactly so: W [M][N] then b [N].
__global__ __launch_bounds__(kTT) void k_wgrad(const float *__restrict__ Ain,
                                                const float *__restrict__ Dout,
                                                float *__restrict__ P, int rows, int M, int N) {
  __shared__ float As[kTK][kTB + 4];
  __shared__ float Bs[kTK][kTB + 4];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int m0 = blockIdx.x * kTB, n0 = blockIdx.y * kTB;
  const int rb = blockIdx.z * kSliceRows, re = min(rows, rb + kSliceRows);
  float acc[4][4] = {};
  for (int k0 = rb; k0 < re; k0 += kTK) {
    for (int idx = tid; idx < kTB * kTK; idx += kTT) {
      const int mm = idx % kTB, kk = idx / kTB;
      const int r = k0 + kk, m = m0 + mm, nn = n0 + mm;
      As[kk][mm] = (r < re && m <= M) ? (m == M ? 1.f : Ain[(long)r * M + m]) : 0.f;
      Bs[kk][mm] = (r < re && nn < N) ? Dout[(long)r * N + nn] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kTK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  float *out = P + (size_t)blockIdx.z * (M + 1) * N;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty * 4 + i;
    if (m > M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = n0 + tx * 4 + j;
      if (c < N) out[(size_t)m * N + c] = acc[i][j];
    }
  }
}

// grad[i] += sum_z P[z][i], the slices in order.
__global__ void k_reduce_slices(const float *__restrict__ P, int nz, size_t len, float *grad) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= len) return;
  float s = grad[i];
  for (int z = 0; z < nz; ++z) s += P[(size_t)z * len + i];
  grad[i] = s;
}

__global__ void k_sgd(float *p, const float *g, size_t n, float lr) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = fmaf(-lr, g[i], p[i]);
}

inline unsigned nblk(size_t n, int t) { return (unsigned)((n + t - 1) / t); }

// Backward through one three-layer MLP for a chunk: X [rows][w0], h1, h2 the
// tanh activations, dout [rows][w3] the gradient at the output.
void mlp_backward(const PolicyShape &sh, const float *params, const float *X, const float *h1,
                  const float *h2, const float *dout, float *grad, float *d1, float *d2,
                  float *part, int rows, cudaStream_t st) {
  const int nz = (rows + kSliceRows - 1) / kSliceRows;
  const float *ain[3] = {X, h1, h2};
  const float *dl[3] = {nullptr, d1, d2};
  // layer 3, then the data gradient into layer 2, and so on
  for (int l = 2; l >= 0; --l) {
    const int M = sh.w[l], N = sh.w[l + 1];
    const float *D = l == 2 ? dout : dl[l + 1];
    dim3 g((unsigned)((M + 1 + kTB - 1) / kTB), (unsigned)((N + kTB - 1) / kTB), (unsigned)nz);
    k_wgrad<<<g, kTT, 0, st>>>(ain[l], D, part, rows, M, N);
    const size_t len = (size_t)(M + 1) * N;
    k_reduce_slices<<<nblk(len, 256), 256, 0, st>>>(part, nz, len, grad + sh.layer_offset(l));
    if (l > 0) {
      // gradient at layer l's input pre-activation: (D W_l^T) * (1 - a_l^2)
      dim3 gb((unsigned)((rows + kTB - 1) / kTB), (unsigned)((M + kTB - 1) / kTB));
      k_bwd_data<<<gb, kTT, 0, st>>>(D, params + sh.layer_offset(l), ain[l], (float *)dl[l], rows, N,
                                     M);
    }
  }
}

}  // namespace

size_t train_scratch_bytes(const PolicyShape &pol, const PolicyShape &crit) {
  const size_t CH = kTrainChunk, w0 = pol.w[0], H0 = pol.w[1], H1 = pol.w[2], NA = pol.w[3];
  const size_t hmax = H0 > H1 ? H0 : H1;
  const size_t nz = (CH + kSliceRows - 1) / kSliceRows;
  size_t maxlen = 0;
  for (int l = 0; l < kMaxLayers; ++l) {
    const size_t len = (size_t)(pol.w[l] + 1) * pol.w[l + 1];
    if (len > maxlen) maxlen = len;
  }
  size_t b = 0;
  auto add = [&](size_t n) { b += (n + 63) / 64 * 64; };
  add(CH * w0 * 4);              // x
  add(CH * 4);                   // ret
  add(CH * 4);                   // act
  add(CH * H0 * 4);              // actor h1
  add(CH * H1 * 4);              // actor h2
  add(CH * NA * 4);              // logits / dlogits
  add(CH * H0 * 4);              // critic h1
  add(CH * H1 * 4);              // critic h2
  add(CH * 4);                   // v / dv
  add(CH * hmax * 4);            // d1
  add(CH * hmax * 4);            // d2
  add(nz * maxlen * 4);          // weight-gradient partials
  add(3 * 8);                    // stats
  add((pol.count() + crit.count()) * 4);  // gradients
  return b;
}

TrainBufs train_bufs(uint8_t *base, const PolicyShape &pol, const PolicyShape &crit) {
  const size_t CH = kTrainChunk, w0 = pol.w[0], H0 = pol.w[1], H1 = pol.w[2], NA = pol.w[3];
  const size_t hmax = H0 > H1 ? H0 : H1;
  const size_t nz = (CH + kSliceRows - 1) / kSliceRows;
  size_t maxlen = 0;
  for (int l = 0; l < kMaxLayers; ++l) {
    const size_t len = (size_t)(pol.w[l] + 1) * pol.w[l + 1];
    if (len > maxlen) maxlen = len;
  }
  TrainBufs t{};
  size_t o = 0;
  auto take = [&](size_t n) {
    uint8_t *p = base + o;
    o += (n + 63) / 64 * 64;
    return p;
  };
  t.x = (float *)take(CH * w0 * 4);
  t.ret = (float *)take(CH * 4);
  t.act = (int32_t *)take(CH * 4);
  t.h1 = (float *)take(CH * H0 * 4);
  t.h2 = (float *)take(CH * H1 * 4);
  t.out = (float *)take(CH * NA * 4);
  t.c1 = (float *)take(CH * H0 * 4);
  t.c2 = (float *)take(CH * H1 * 4);
  t.vout = (float *)take(CH * 4);
  t.d1 = (float *)take(CH * hmax * 4);
  t.d2 = (float *)take(CH * hmax * 4);
  t.part = (float *)take(nz * maxlen * 4);
  t.stats = (double *)take(3 * 8);
  t.grad = (float *)take((pol.count() + crit.count()) * 4);
  return t;
}

void launch_a2c_update(const Dev &d, const TrainBufs &tb, float *critic, const PolicyShape &crit,
                       uint32_t n, float lr, float c_v, float c_e, cudaStream_t st) {
  const PolicyShape &pol = d.pol;
  const size_t R = (size_t)n * d.n_slots;
  const size_t na = pol.count(), nc = crit.count();
  float *ga = tb.grad, *gc = tb.grad + na;
  cudaMemsetAsync(tb.grad, 0, (na + nc) * 4, st);
  cudaMemsetAsync(tb.stats, 0, 3 * 8, st);
  const double inv_r = 1.0 / (double)R;
  for (size_t q0 = 0; q0 < R; q0 += kTrainChunk) {
    const int rows = (int)((R - q0) < (size_t)kTrainChunk ? (R - q0) : (size_t)kTrainChunk);
    k_a2c_gather<<<nblk(rows, 256), 256, 0, st>>>(d, n, q0, (uint32_t)rows, tb);
    // forward: actor and critic
    launch_mlp3_f32(tb.x, pol.w[0], 1, d.params, pol, tb.h1, tb.h2, tb.out, rows, st);
    launch_mlp3_f32(tb.x, pol.w[0], 1, critic, crit, tb.c1, tb.c2, tb.vout, rows, st);
    k_a2c_head<<<nblk(rows, 256), 256, 0, st>>>(d, (uint32_t)rows, inv_r, c_v, c_e, tb);
    mlp_backward(pol, d.params, tb.x, tb.h1, tb.h2, tb.out, ga, tb.d1, tb.d2, tb.part, rows, st);
    mlp_backward(crit, critic, tb.x, tb.c1, tb.c2, tb.vout, gc, tb.d1, tb.d2, tb.part, rows, st);
  }
  k_sgd<<<nblk(na, 256), 256, 0, st>>>((float *)d.params, ga, na, lr);
  k_sgd<<<nblk(nc, 256), 256, 0, st>>>(critic, gc, nc, lr);
}

}  // namespace ws
