// ws_econ_tc.cu -- fused persistent BF16 tensor-core roll-out kernel of the
// multi-agent economy: one launch runs a whole chunk of steps for every env,
// pulling work items (runs of whole envs) from a device work queue.
//
// Paper grounding: App. B (Fig. 1) gives every env its own block of the GPU
// and every agent its own thread, with agents interacting inside the env and
// the policy models referenced from GPU memory; Sec. 2 keeps roll-out,
// inference and reset on the GPU with an in-place store.  Here that mapping is
// re-cut for tensor cores and uneven agent counts: a work item is a run of
// consecutive envs whose agents fill up to AT tiles of 128 rows (one agent per
// thread and TMEM lane), and the CTA keeps the item's whole state (features and
// int64 wealth in registers, transfers and tax pools in shared memory) on chip
// for all the steps of the chunk.  Per step and item:
//   observe   records of the pre-step observation and wealth; the agents'
//             layer-1 operand (BF16 features) into shared memory; per-env
//             wealth totals (segmented warp sums, then shared-memory atomics)
//   agents    16-128-128-20 MLP per tile on tcgen05 (FP32 accumulators in
//             TMEM, bias + tanh epilogues writing the next layer's 128B-swizzled
//             operand; layers 2 and 3 pipelined over 64-column halves), then
//             the categorical draw (Philox, inverse CDF in FP32)
//   planner   its own warpgroup: mean agent features per env (fixed-order warp
//             sums), then the 16-128-128-10 MLP with the operands swapped
//             (D[hidden][env] = W^T obs^T: the envs of the item become the N
//             columns, so a handful of planner rows costs N = 16..64, not a
//             128-row tile), the last layer in normal orientation, the draw
//   transfer  t_i = floor(w_i a_i / 400) to a Philox partner, credited with
//             shared-memory int64 atomics (exact, order-free)
//   tax       floor(income tau / 20) into the env pool (segmented sums + int64
//             atomics); even redistribution with the remainder to low indices
//   finish    features, rewards (the planner's reward is a fixed-order mean),
//             done at the episode limit and the Philox auto-reset in registers
// The agents' warps and the planner's warpgroup meet at three CTA barriers per
// step (observation ready; transfers done and tax level known; pool complete).
// Every mbarrier wait is bounded; a wait that runs out is voted on at the next
// CTA barrier and the whole CTA leaves, drains its MMAs and sets the error flag.
#include "ws_kernels.cuh"
#include "ws_tc.cuh"

namespace ws {

namespace {

constexpr int kTile = 128;
constexpr int kH = 128;                 // hidden width of both policies
constexpr int kNA = 20, kNAp = 32;      // agent classes, padded layer-3 N
constexpr int kNP = 10, kNPp = 16;      // planner classes, padded layer-3 N
constexpr int kMaxEnvs = 64;            // envs per work item (planner MMA N <= 64)

// Packed global image (the kernel copies it verbatim into shared memory):
//   W2A  agent W2^T, B operand, SW128 K-major [128 n][128 k]
//   W2P  planner W2^T, A operand of the swapped product, SW128 [128 m][128 k]
//   W3A  agent W3^T, B operand, SW128 [32 n][128 k] (rows >= 20 zero)
//   W3P  planner W3^T, B operand, SW128 [16 n][128 k] (rows >= 10 zero)
//   W1A  agent W1^T, B operand, K = 16 without swizzle [128 n][16 k]
//   W1P  planner W1^T, A operand of the swapped product, [128 m][16 k]
//   BIAS b1a 128 | b2a 128 | b3a 32 | b1p 128 | b2p 128 | b3p 16 (FP32)
constexpr int PK_W2A = 0;
constexpr int PK_W2P = 32768;
constexpr int PK_W3A = 65536;
constexpr int PK_W3P = PK_W3A + 8192;
constexpr int PK_W1A = PK_W3P + 4096;
constexpr int PK_W1P = PK_W1A + 4096;
constexpr int PK_BIAS = PK_W1P + 4096;
constexpr int BIAS_N = 560;
constexpr int PACKED = PK_BIAS + BIAS_N * 4;
constexpr int BO_B1A = 0, BO_B2A = 128, BO_B3A = 256, BO_B1P = 288, BO_B2P = 416, BO_B3P = 544;

template <int AT>
struct EconTc {
  static constexpr int ROWS = AT * kTile;          // agent rows (threads) per item
  static constexpr int THREADS = ROWS + kTile;     // + the planner warpgroup
  static constexpr uint32_t PCOL = AT * kTile;     // planner's TMEM columns
  static constexpr uint32_t TMEM_COLS = AT == 1 ? 256u : 512u;
  static constexpr int OFF_W2A = 0;
  static constexpr int OFF_W2P = 32768;
  static constexpr int OFF_HS = 65536;             // [tile] 32 KB: h1 / h2, layer-1 A at its start
  static constexpr int OFF_HP = OFF_HS + AT * 32768;  // planner activations [128 env rows][128 k]
  static constexpr int OFF_SFEAT = OFF_HP;            // aliases HP: float4 [4][ROWS]
  static constexpr int OFF_SREW = OFF_HP + 16 * ROWS * 4;  // aliases HP: f32 [ROWS]
  static constexpr int OFF_W3A = OFF_HP + 32768;   // W3A | W3P | W1A | W1P | BIAS as packed
  static constexpr int OFF_W3P = OFF_W3A + 8192;
  static constexpr int OFF_W1A = OFF_W3P + 4096;
  static constexpr int OFF_W1P = OFF_W1A + 4096;
  static constexpr int OFF_BIAS = OFF_W1P + 4096;
  static constexpr int OFF_POBS = (OFF_BIAS + BIAS_N * 4 + 127) / 128 * 128;  // [64][16] K=16
  static constexpr int OFF_INC = OFF_POBS + kMaxEnvs * 32;  // i64 [ROWS] income (credits)
  static constexpr int OFF_ENVT = OFF_INC + ROWS * 8;       // i64 [64] tax pool
  static constexpr int OFF_WSUM = OFF_ENVT + kMaxEnvs * 8;  // i64 [64] pre-step wealth total
  static constexpr int OFF_ENVI = OFF_WSUM + kMaxEnvs * 8;  // int4 [64] {a0 in item, n, env, tau}
  // MMA barriers: [AT + 1] one per tile and the planner, the drain, [AT] a
  // second one per tile
  static constexpr int OFF_BAR = OFF_ENVI + kMaxEnvs * 16;
  static constexpr int OFF_TM = OFF_BAR + 8 * (2 * AT + 2);
  static constexpr int OFF_ITEM = OFF_TM + 16;
  static constexpr int SMEM = OFF_ITEM + 16 + 1024;
  static_assert(SMEM <= 232448, "shared memory over the 227 KB per-CTA limit");
  static_assert(16 * ROWS * 4 + ROWS * 4 <= 32768, "feature / reward staging must fit the HP slot");
  static_assert(OFF_HP % 1024 == 0 && OFF_W3A % 1024 == 0 && OFF_W3P % 1024 == 0,
                "SW128 operands need 1024-byte alignment");
  static_assert(PCOL + 64 <= TMEM_COLS, "planner columns");
};

__device__ __forceinline__ uint16_t bf16_bits(float f) {
  return (uint16_t)(tc::pack_bf16x2(f, 0.f) & 0xFFFFu);
}
// Element (row n, k) of a 128B-swizzled K-major operand with `rows` rows per
// K-block of 64 elements.
__device__ __forceinline__ int sw128_off(int n, int k, int rows) {
  const int kb = k >> 6, kk = k & 63;
  return kb * (rows * 128) + n * 128 + (((kk >> 3) ^ (n & 7)) << 4) + (kk & 7) * 2;
}
// Element (row n, q) of a K = 16 operand without swizzle (8-row core matrices
// of 16-byte rows; the two K-halves 128 B apart, 8-row groups 256 B apart).
__device__ __forceinline__ int k16_off(int n, int q) {
  return (n >> 3) * 256 + (q >> 3) * 128 + (n & 7) * 16 + (q & 7) * 2;
}

__global__ void k_econ_tc_pack(const float *__restrict__ pa, const float *__restrict__ pp,
                               uint8_t *__restrict__ out) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  // agent: W1 [16][128] b1 W2 [128][128] b2 W3 [128][20] b3; planner likewise with 10
  const float *W1a = pa, *b1a = W1a + 16 * kH, *W2a = b1a + kH, *b2a = W2a + kH * kH;
  const float *W3a = b2a + kH, *b3a = W3a + kH * kNA;
  const float *W1p = pp, *b1p = W1p + 16 * kH, *W2p = b1p + kH, *b2p = W2p + kH * kH;
  const float *W3p = b2p + kH, *b3p = W3p + kH * kNP;
  for (int i = tid; i < kH * kH; i += stride) {
    const int n = i / kH, k = i % kH;
    *(uint16_t *)(out + PK_W2A + sw128_off(n, k, kH)) = bf16_bits(W2a[k * kH + n]);
    *(uint16_t *)(out + PK_W2P + sw128_off(n, k, kH)) = bf16_bits(W2p[k * kH + n]);
  }
  for (int i = tid; i < kNAp * kH; i += stride) {
    const int n = i / kH, k = i % kH;
    *(uint16_t *)(out + PK_W3A + sw128_off(n, k, kNAp)) = bf16_bits(n < kNA ? W3a[k * kNA + n] : 0.f);
  }
  for (int i = tid; i < kNPp * kH; i += stride) {
    const int n = i / kH, k = i % kH;
    *(uint16_t *)(out + PK_W3P + sw128_off(n, k, kNPp)) = bf16_bits(n < kNP ? W3p[k * kNP + n] : 0.f);
  }
  for (int i = tid; i < kH * 16; i += stride) {
    const int n = i / 16, q = i % 16;
    *(uint16_t *)(out + PK_W1A + k16_off(n, q)) = bf16_bits(W1a[q * kH + n]);
    *(uint16_t *)(out + PK_W1P + k16_off(n, q)) = bf16_bits(W1p[q * kH + n]);
  }
  float *bias = (float *)(out + PK_BIAS);
  for (int i = tid; i < BIAS_N; i += stride) {
    float v = 0.f;
    if (i < BO_B2A) v = b1a[i];
    else if (i < BO_B3A) v = b2a[i - BO_B2A];
    else if (i < BO_B1P) v = (i - BO_B3A) < kNA ? b3a[i - BO_B3A] : 0.f;
    else if (i < BO_B2P) v = b1p[i - BO_B1P];
    else if (i < BO_B3P) v = b2p[i - BO_B2P];
    else v = (i - BO_B3P) < kNP ? b3p[i - BO_B3P] : 0.f;
    bias[i] = v;
  }
}

// ---- small helpers ------------------------------------------------------------
__device__ __forceinline__ void bar_sync_n(uint32_t id, uint32_t n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void bar_arrive_n(uint32_t id, uint32_t n) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}
// AND of a predicate over the n threads of barrier `id`.
__device__ __forceinline__ bool bar_all_n(uint32_t id, uint32_t n, bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.and.pred q, %2, %3, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(id), "r"(n)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ float4 lds128f(uint32_t addr) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(addr));
  return v;
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&z)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(z[0]), "=r"(z[1]), "=r"(z[2]), "=r"(z[3]), "=r"(z[4]), "=r"(z[5]), "=r"(z[6]),
        "=r"(z[7]), "=r"(z[8]), "=r"(z[9]), "=r"(z[10]), "=r"(z[11]), "=r"(z[12]), "=r"(z[13]),
        "=r"(z[14]), "=r"(z[15])
      : "r"(taddr));
}
__device__ __forceinline__ void atom_add_i64(uint32_t addr, long long v) {
  asm volatile("red.shared.add.u64 [%0], %1;" ::"r"(addr), "l"(v) : "memory");
}

// Segmented inclusive warp sum over lanes whose keys are equal and contiguous
// (each warp holds consecutive rows, and an env's rows are consecutive).  On
// return `tail` marks the last lane of each segment, whose v is the segment sum.
__device__ __forceinline__ long long seg_sum(long long v, int key, bool &tail) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const long long o = __shfl_up_sync(0xffffffffu, v, off);
    const int ko = __shfl_up_sync(0xffffffffu, key, off);
    if (lane >= off && ko == key) v += o;
  }
  const int kn = __shfl_down_sync(0xffffffffu, key, 1);
  tail = lane == 31 || kn != key;
  return v;
}

// Sums of 16 per-lane values over a warp by recursive halving: at each level a
// lane keeps half of its values and adds the partner's copy of that half (8, 4,
// 2, 1 shuffles), then one exchange completes the sum.  Returns the total of
// value (lane >> 1) & 15; 16 shuffles in place of 80 for 16 butterflies.
__device__ __forceinline__ float warp_sum16(float (&v)[kEconF], int lane) {
#pragma unroll
  for (int w = 8, o = 16; w >= 1; w >>= 1, o >>= 1) {
    const bool up = (lane & o) != 0;  // keep the upper half of the w-pairs
#pragma unroll
    for (int i = 0; i < w; ++i) {
      const float keep = up ? v[w + i] : v[i];
      const float send = up ? v[i] : v[w + i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// Categorical draw by inverse CDF in FP32 (the arithmetic of the plain path's
// sampler): a = min{i : u S < C_i}, C_i the running sum of exp(l - max), S the
// total; logp = (l_a - max) - log S.
template <int N>
__device__ __forceinline__ int sample_cat(const float (&l)[N], float u, float &logp) {
  float m = l[0];
#pragma unroll
  for (int c = 1; c < N; ++c) m = fmaxf(m, l[c]);
  float e[N];
  float S = 0.f;
#pragma unroll
  for (int c = 0; c < N; ++c) {
    e[c] = expf(l[c] - m);
    S += e[c];
  }
  const float thr = u * S;
  float C = 0.f;
  int a = N - 1;
  bool found = false;
#pragma unroll
  for (int c = 0; c < N; ++c) {
    C += e[c];
    if (!found && thr < C) {
      a = c;
      found = true;
    }
  }
  float la = l[0];
#pragma unroll
  for (int c = 1; c < N; ++c)
    if (c == a) la = l[c];
  logp = (la - m) - logf(S);
  return a;
}

// tanh(acc + bias) of 64 accumulator columns as 32 packed bf16x2.
__device__ __forceinline__ void act64(uint32_t taddr, uint32_t bias, uint32_t (&hp)[32]) {
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    uint32_t z[32];
    tc::tmem_ld32(taddr + (uint32_t)(half * 32), z);
    tc::tmem_wait_ld();
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float4 b = lds128f(bias + (uint32_t)((half * 32 + 4 * i) * 4));
      hp[half * 16 + 2 * i] = tc::tanh_bf16x2(
          tc::pack_bf16x2(__uint_as_float(z[4 * i]) + b.x, __uint_as_float(z[4 * i + 1]) + b.y));
      hp[half * 16 + 2 * i + 1] = tc::tanh_bf16x2(tc::pack_bf16x2(
          __uint_as_float(z[4 * i + 2]) + b.z, __uint_as_float(z[4 * i + 3]) + b.w));
    }
  }
}

__device__ __forceinline__ void store_row_sw128(uint32_t row_addr, uint32_t swz,
                                                const uint32_t (&p)[32]) {
#pragma unroll
  for (int ch = 0; ch < 8; ++ch)
    tc::sts128(row_addr + (((uint32_t)ch ^ swz) << 4), p[ch * 4 + 0], p[ch * 4 + 1], p[ch * 4 + 2],
               p[ch * 4 + 3]);
}

// Economy auto-reset of one agent (draws RESET sub 0..4 at step k).
__device__ __forceinline__ void reset_agent(uint64_t seed, uint32_t k, uint32_t env,
                                            uint32_t agent, long long &w, float (&f)[kEconF]) {
  uint4 r = draw(seed, k, env, agent, kTagReset, 0);
  const uint64_t big = ((uint64_t)r.y << 32) | (uint64_t)r.x;
  w = 10000 + (long long)(big % 990001ull);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    r = draw(seed, k, env, agent, kTagReset, 1 + j);
    const float2 a = box_muller(r.x, r.y), b = box_muller(r.z, r.w);
    f[4 * j + 0] = a.x;
    f[4 * j + 1] = a.y;
    f[4 * j + 2] = b.x;
    f[4 * j + 3] = b.y;
  }
}

// Barrier ids: 0 __syncthreads; 1 observation ready (agents arrive, planner
// waits); 2 transfers done + tax level known (vote); 3 pool complete; 4.. one
// per agent tile; 4 + AT the planner warpgroup.
constexpr uint32_t kBarObs = 1, kBarTax = 2, kBarPool = 3, kBarTile0 = 4;

template <int AT>
__global__ void __launch_bounds__((AT + 1) * 128, 1)
    k_econ_tc(Dev d, const uint8_t *__restrict__ packed, uint32_t n_steps) {
  using C = EconTc<AT>;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = tc::smem_u32(smem_raw);
  uint8_t *sm = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
  const uint32_t sb = tc::smem_u32(sm);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool planner = tid >= C::ROWS;
  uint64_t *bars = (uint64_t *)(sm + C::OFF_BAR);
  uint32_t *tm_holder = (uint32_t *)(sm + C::OFF_TM);
  volatile uint32_t *s_item = (volatile uint32_t *)(sm + C::OFF_ITEM);
  int4 *envi = (int4 *)(sm + C::OFF_ENVI);
  long long *envT = (long long *)(sm + C::OFF_ENVT);
  long long *wsum = (long long *)(sm + C::OFF_WSUM);
  long long *income = (long long *)(sm + C::OFF_INC);
  float4 *sfeat = (float4 *)(sm + C::OFF_SFEAT);
  float *srew = (float *)(sm + C::OFF_SREW);

  {
    const uint4 *src = (const uint4 *)packed;
    uint4 *dst = (uint4 *)sm;
    for (int i = tid; i < PK_W3A / 16; i += C::THREADS) dst[i] = __ldg(src + i);
    src = (const uint4 *)(packed + PK_W3A);
    dst = (uint4 *)(sm + C::OFF_W3A);
    for (int i = tid; i < (PACKED - PK_W3A) / 16; i += C::THREADS) dst[i] = __ldg(src + i);
  }
  if (tid == 0) {
    for (int i = 0; i <= AT; ++i) tc::mbar_init(bars + i, 1);
    tc::mbar_init(bars + AT + 1, AT + 1);
    for (int i = 0; i < AT; ++i) tc::mbar_init(bars + AT + 2 + i, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tc::tmem_alloc(tm_holder, C::TMEM_COLS);
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();

  const uint32_t tbase = *tm_holder;
  const uint32_t lane_sel = (uint32_t)((warp & 3) * 32) << 16;
  const int tile = planner ? AT : (tid >> 7);
  const int r = tid & 127;
  const bool issuer = r == 0;
  uint64_t *bar = bars + tile;
  uint64_t *bar2 = bars + AT + 2 + tile;  // an agent tile's second MMA barrier
  const uint32_t my_bar_id = kBarTile0 + (uint32_t)tile;  // tile or planner warpgroup barrier
  const uint32_t tcol = tbase + (uint32_t)tile * 128u;    // this warpgroup's TMEM columns (lane 0)
  const uint32_t hs = sb + C::OFF_HS + (uint32_t)(planner ? 0 : tile) * 32768u;
  const uint32_t bias = sb + C::OFF_BIAS;
  const uint64_t seed = d.seed;
  const uint64_t k0 = d.k[0];
  const uint32_t R = d.ring_steps;
  const size_t S = d.n_slots, Sa = d.n_agent_slots;
  const int4 *items = (const int4 *)d.items;
  const float inv_ln_1e6 = 0.0723824136505f;

  uint32_t ph = 0u, ph2 = 0u;
  bool ok = true, wfail = false;
  uint32_t fsite = 0;

  for (;;) {
    if (tid == 0) s_item[0] = atomicAdd(d.queue, 1u);
    __syncthreads();
    const uint32_t it = s_item[0];
    if (it >= d.n_items) break;
    const int4 I = items[it];
    const uint32_t slot0 = (uint32_t)I.x;
    const int n_rows = I.y, n_env = I.w;
    const uint32_t env0 = (uint32_t)I.z;

    if (!planner) {
      // =========================== agent rows ===========================
      const int row = tid;
      const bool valid = row < n_rows;
      const bool tile_on = tile * kTile < n_rows;
      const bool warp_on = (row & ~31) < n_rows;
      const uint32_t slot = slot0 + (uint32_t)row;
      uint32_t env = 0, agent = 0;
      int e_loc = -1, n = 1, t = 0;
      long long w = 0;
      float f[kEconF];
#pragma unroll
      for (int j = 0; j < kEconF; ++j) f[j] = 0.f;
      if (valid) {
        env = (uint32_t)d.slot_env[slot];
        const int a0 = d.agent_off[env];
        n = d.agent_off[env + 1] - a0;
        agent = slot - (uint32_t)a0;
        e_loc = (int)(env - env0);
        w = d.wealth[slot];
#pragma unroll
        for (int j = 0; j < kEconF; ++j) f[j] = d.feat[(size_t)j * Sa + slot];
        t = d.t[env];
      }
      income[row] = 0;
      const uint32_t a1_row = hs + (uint32_t)(r >> 3) * 256u + (uint32_t)(r & 7) * 16u;
      const uint32_t tm = tcol + lane_sel;
      const uint64_t da1 = tc::smem_desc(hs, 128, 256, tc::kSwizzleNone);
      const uint64_t db1 = tc::smem_desc(sb + C::OFF_W1A, 128, 256, tc::kSwizzleNone);
      constexpr uint32_t id12 = tc::idesc_bf16_f32(128, kH);
      constexpr uint32_t id2h = tc::idesc_bf16_f32(128, kH / 2);
      constexpr uint32_t id3 = tc::idesc_bf16_f32(128, kNAp);
      __syncthreads();

      for (uint32_t s = 0; s < n_steps; ++s) {
        const uint32_t k = (uint32_t)(k0 + s);
        const size_t rowR = (size_t)((k0 + s) % R);
        // ---- observe
        if (valid) {
          float *ob = d.r_obs + rowR * kEconF * S + slot;
#pragma unroll
          for (int j = 0; j < kEconF; ++j) ob[(size_t)j * S] = f[j];
#pragma unroll
          for (int q = 0; q < 4; ++q)
            sfeat[q * C::ROWS + row] = make_float4(f[4 * q], f[4 * q + 1], f[4 * q + 2], f[4 * q + 3]);
          d.r_wealth[rowR * S + slot] = w;
        }
        tc::sts128(a1_row, tc::pack_bf16x2(f[0], f[1]), tc::pack_bf16x2(f[2], f[3]),
                   tc::pack_bf16x2(f[4], f[5]), tc::pack_bf16x2(f[6], f[7]));
        tc::sts128(a1_row + 128, tc::pack_bf16x2(f[8], f[9]), tc::pack_bf16x2(f[10], f[11]),
                   tc::pack_bf16x2(f[12], f[13]), tc::pack_bf16x2(f[14], f[15]));
        {
          bool tail;
          const long long ws = seg_sum(valid ? w : 0, e_loc, tail);
          if (tail && e_loc >= 0) atom_add_i64(sb + C::OFF_WSUM + 8u * (uint32_t)e_loc, ws);
        }
        // (the named barrier orders these shared-memory writes before the
        // planner's reads; the async-proxy fence covers the MMA's operand)
        tc::fence_async_smem();
        bar_arrive_n(kBarObs, C::THREADS);
        // ---- agent policy on the tensor core
        float lg[kNA];
#pragma unroll
        for (int c = 0; c < kNA; ++c) lg[c] = 0.f;
        if (tile_on) {
          tc::fence_before_sync();  // last step's TMEM reads precede this step's MMAs
          bar_sync_n(my_bar_id, 128);
          if (issuer) {
            tc::fence_after_sync();
            tc::mma_bf16(tcol, da1, db1, id12, false);
            tc::mma_commit(bar);
          }
          if (!tc::mbar_wait(bar, ph, d.wait_ns) && !wfail) { wfail = true; fsite = 1; }
          ph ^= 1u;
          tc::fence_after_sync();
          // Layers 2 and 3 are pipelined over 64-column halves, so that the
          // tensor core works while the tile's warps run their tanh: act 1 of
          // columns 0-63 is h1's K block 0, whose layer-2 product into output
          // columns 0-63 runs while act 1 reads columns 64-127; the rest of
          // layer 2 is committed in two parts (output columns 0-63, then
          // 64-127), and act 2 of each half (h2's K block) starts layer 3's
          // product over that K block.  An MMA writes only columns that the
          // warps have read out, and h1 / h2 share the tile's operand buffer
          // by K block: a block is overwritten only after every MMA that reads
          // it has completed (the commits waited on before).
          //   commit   MMAs (output columns, K block)       waited before
          //   bar      L2 (0-63, 0) (64-127, 0) (0-63, 1)   act 2 of 0-63
          //   bar2     L2 (64-127, 1)                       act 2 of 64-127
          //   bar      L3 (0-31, 0) (0-31, 1)               the logits
          auto l2_mma = [&](int nh, int kb) {
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const uint32_t ka = (uint32_t)(kb * 16384 + kk * 32);
              const uint64_t da = tc::smem_desc(hs + ka, 16, 1024, tc::kSwizzle128B);
              const uint64_t db = tc::smem_desc(sb + C::OFF_W2A + ka + (uint32_t)nh * 8192u, 16, 1024,
                                                tc::kSwizzle128B);
              tc::mma_bf16(tcol + (uint32_t)nh * 64u, da, db, id2h, (kb | kk) != 0);
            }
          };
          auto l3_mma = [&](int kb) {
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const uint32_t ka = (uint32_t)(kb * 16384 + kk * 32);
              const uint64_t da = tc::smem_desc(hs + ka, 16, 1024, tc::kSwizzle128B);
              const uint64_t db = tc::smem_desc(
                  sb + C::OFF_W3A + (uint32_t)(kb * kNAp * 128 + kk * 32), 16, 1024, tc::kSwizzle128B);
              tc::mma_bf16(tcol, da, db, id3, (kb | kk) != 0);
            }
          };
          auto act_half = [&](int l, int kb) {
            if (warp_on) {
              uint32_t hp[32];
              act64(tm + (uint32_t)(kb * 64), bias + (uint32_t)(((l == 0 ? BO_B1A : BO_B2A) + kb * 64) * 4),
                    hp);
              store_row_sw128(hs + (uint32_t)kb * 16384u + (uint32_t)r * 128u, (uint32_t)(r & 7), hp);
            }
            tc::fence_async_smem();
            tc::fence_before_sync();
            bar_sync_n(my_bar_id, 128);
          };
          act_half(0, 0);
          if (issuer) {
            tc::fence_after_sync();
            l2_mma(0, 0);
          }
          act_half(0, 1);
          if (issuer) {
            tc::fence_after_sync();
            l2_mma(1, 0);
            l2_mma(0, 1);
            tc::mma_commit(bar);
            l2_mma(1, 1);
            tc::mma_commit(bar2);
          }
          if (!tc::mbar_wait(bar, ph, d.wait_ns) && !wfail) { wfail = true; fsite = 2; }
          ph ^= 1u;
          tc::fence_after_sync();
          act_half(1, 0);
          if (issuer) {
            tc::fence_after_sync();
            l3_mma(0);
          }
          if (!tc::mbar_wait(bar2, ph2, d.wait_ns) && !wfail) { wfail = true; fsite = 2; }
          ph2 ^= 1u;
          tc::fence_after_sync();
          act_half(1, 1);
          if (issuer) {
            tc::fence_after_sync();
            l3_mma(1);
            tc::mma_commit(bar);
          }
          if (!tc::mbar_wait(bar, ph, d.wait_ns) && !wfail) { wfail = true; fsite = 3; }
          ph ^= 1u;
          tc::fence_after_sync();
          if (warp_on) {
            uint32_t z0[16], z1[16];
            tmem_ld16(tm, z0);
            tmem_ld16(tm + 16, z1);
            tc::tmem_wait_ld();
#pragma unroll
            for (int q = 0; q < kNA / 4; ++q) {
              const float4 b = lds128f(bias + (uint32_t)((BO_B3A + 4 * q) * 4));
              const uint32_t *z = q < 4 ? z0 + 4 * q : z1 + 4 * (q - 4);
              lg[4 * q] = __uint_as_float(z[0]) + b.x;
              lg[4 * q + 1] = __uint_as_float(z[1]) + b.y;
              lg[4 * q + 2] = __uint_as_float(z[2]) + b.z;
              lg[4 * q + 3] = __uint_as_float(z[3]) + b.w;
            }
          }
        }
        // ---- sample, transfer
        int a = 0;
        long long w_after = w;
        if (valid) {
          const float u = u01(draw(seed, k, d.env_base + env, agent, kTagAction, 0).x);
          float lp;
          a = sample_cat<kNA>(lg, u, lp);
          const size_t o = rowR * S + slot;
          ((int32_t *)d.r_act)[o] = a;
          d.r_logp[o] = lp;
          if (d.dbg_logits) {
#pragma unroll
            for (int c = 0; c < kNA; ++c) d.out[(size_t)slot * kNA + c] = lg[c];
#pragma unroll
            for (int c = 0; c < kNA; ++c) d.r_pout[(rowR * kNA + c) * S + slot] = lg[c];
          }
          const uint32_t rp = draw(seed, k, d.env_base + env, agent, kTagPartner, 0).x;
          const uint32_t p = (agent + 1u + bounded(rp, (uint32_t)(n - 1))) % (uint32_t)n;
          const long long amt = (w * (long long)a) / 400;
          w_after = w - amt;
          atom_add_i64(sb + C::OFF_INC + 8u * (uint32_t)(row - (int)agent + (int)p), amt);
        }
        ok = bar_all_n(kBarTax, C::THREADS, !wfail);
        if (!ok) break;
        // ---- tax on income into the env pool
        long long w_mid = w_after, tax = 0;
        if (valid) {
          const long long inc = income[row];
          income[row] = 0;
          tax = (inc * (long long)envi[e_loc].w) / 20;
          w_mid = w_after + inc - tax;
        }
        {
          bool tail;
          const long long ts = seg_sum(tax, e_loc, tail);
          if (tail && e_loc >= 0) atom_add_i64(sb + C::OFF_ENVT + 8u * (uint32_t)e_loc, ts);
        }
        bar_sync_n(kBarPool, C::THREADS);
        // ---- redistribution, features, reward, done, auto-reset
        if (valid) {
          const long long T = envT[e_loc];
          long long share, rem;
          if (T >= 0 && T <= 0x7fffffffLL) {  // the usual case, in 32-bit arithmetic
            const uint32_t q = (uint32_t)T / (uint32_t)n;
            share = q;
            rem = (long long)((uint32_t)T - q * (uint32_t)n);
          } else {  // floor division for a pool of either sign
            share = T / n;
            rem = T % n;
            if (rem < 0) {
              rem += n;
              share -= 1;
            }
          }
          const long long w2 = w_mid + share + ((long long)agent < rem ? 1 : 0);
          const float drive = ((float)a - 9.5f) / 9.5f;
#pragma unroll
          for (int j = 0; j < kEconF - 1; ++j) f[j] = 0.95f * f[j] + 0.05f * ((j & 1) ? -drive : drive);
          f[kEconF - 1] = logf((float)w2) * inv_ln_1e6;
          const float rew = (float)(w2 - w) / 1e4f - 1e-3f * (float)(a * a);
          const int t2 = t + 1;
          const bool done = t2 >= (int)d.episode_limit;
          const size_t o = rowR * S + slot;
          d.r_rew[o] = rew;
          d.r_done[o] = (uint8_t)done;
          srew[row] = rew;
          if (done) {
            reset_agent(seed, k, d.env_base + env, agent, w, f);
            t = 0;
          } else {
            w = w2;
            t = t2;
          }
        }
      }
      if (ok) bar_arrive_n(kBarObs, C::THREADS);  // the planner's reward of the last step
      if (ok && valid) {
        d.wealth[slot] = w;
#pragma unroll
        for (int j = 0; j < kEconF; ++j) d.feat[(size_t)j * Sa + slot] = f[j];
      }
    } else {
      // =========================== planner ===========================
      const int pt = tid - C::ROWS, pw = pt >> 5;
      const int npad = n_env <= 16 ? 16 : (n_env + 15) / 16 * 16;
      int t = 0, pdone = 0;
      uint32_t penv = env0 + (uint32_t)pt;
      if (pt < n_env) {
        const int a0 = d.agent_off[penv];
        envi[pt] = make_int4(a0 - (int)slot0, d.agent_off[penv + 1] - a0, (int)penv, 0);
        envT[pt] = 0;
        wsum[pt] = 0;
        t = d.t[penv];
      }
      const uint32_t tm = tcol + lane_sel;
      const uint32_t hp_base = sb + C::OFF_HP;
      const uint64_t dw1 = tc::smem_desc(sb + C::OFF_W1P, 128, 256, tc::kSwizzleNone);
      const uint64_t dpo = tc::smem_desc(sb + C::OFF_POBS, 128, 256, tc::kSwizzleNone);
      const uint32_t idn = tc::idesc_bf16_f32(128, (uint32_t)npad);
      constexpr uint32_t id3 = tc::idesc_bf16_f32(128, kNPp);
      const size_t ps = Sa + penv;
      __syncthreads();

      for (uint32_t s = 0; s <= n_steps; ++s) {
        bar_sync_n(kBarObs, C::THREADS);
        if (s > 0) {
          // reward (fixed-order mean of the agents' rewards) and done of step s - 1
          const size_t rowP = (size_t)((k0 + s - 1) % R);
          for (int e = pw; e < n_env; e += 4) {
            const int4 ei = envi[e];
            float acc = 0.f;
            for (int i = lane; i < ei.y; i += 32) acc += srew[ei.x + i];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) d.r_rew[rowP * S + Sa + (uint32_t)ei.z] = acc / (float)ei.y;
          }
          if (pt < n_env) d.r_done[rowP * S + ps] = (uint8_t)pdone;
        }
        if (s == n_steps) break;
        const uint32_t k = (uint32_t)(k0 + s);
        const size_t rowR = (size_t)((k0 + s) % R);
        if (pt < n_env) {
          d.r_wealth[rowR * S + ps] = wsum[pt];
          wsum[pt] = 0;
          envT[pt] = 0;
        }
        // ---- observation: mean agent features per env (fixed-order sums)
        for (int e = pw; e < n_env; e += 4) {
          const int4 ei = envi[e];
          float acc[kEconF];
#pragma unroll
          for (int j = 0; j < kEconF; ++j) acc[j] = 0.f;
          for (int i = lane; i < ei.y; i += 32) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const float4 v = sfeat[q * C::ROWS + ei.x + i];
              acc[4 * q] += v.x;
              acc[4 * q + 1] += v.y;
              acc[4 * q + 2] += v.z;
              acc[4 * q + 3] += v.w;
            }
          }
          // reduce-scatter over the warp (fixed order): after it, lanes 2j and
          // 2j + 1 hold the total of feature j
          const float tot = warp_sum16(acc, lane);
          if ((lane & 1) == 0) {
            const int j = lane >> 1;
            const float mean = tot / (float)ei.y;
            d.r_obs[(rowR * kEconF + (size_t)j) * S + Sa + (uint32_t)ei.z] = mean;
            *(uint16_t *)(sm + C::OFF_POBS + k16_off(e, j)) = bf16_bits(mean);
          }
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        bar_sync_n(my_bar_id, 128);
        if (issuer) {
          tc::fence_after_sync();
          tc::mma_bf16(tcol, dw1, dpo, idn, false);
          tc::mma_commit(bar);
        }
        if (!tc::mbar_wait(bar, ph, d.wait_ns) && !wfail) { wfail = true; fsite = 5; }
        ph ^= 1u;
        tc::fence_after_sync();
#pragma unroll 1
        for (int l = 0; l < 2; ++l) {
          // D[hidden pt][env]: tanh(acc + b) into row env, column pt of HP
          const float b = *(const float *)(sm + C::OFF_BIAS + ((l == 0 ? BO_B1P : BO_B2P) + pt) * 4);
          for (int g = 0; g < npad; g += 16) {
            uint32_t z[16];
            tmem_ld16(tm + (uint32_t)g, z);
            tc::tmem_wait_ld();
#pragma unroll
            for (int c = 0; c < 16; ++c) {
              const int e = g + c;
              if (e < n_env) {
                const float h = tc::tanh_fast(__uint_as_float(z[c]) + b);
                *(uint16_t *)(sm + C::OFF_HP + sw128_off(e, pt, 128)) = bf16_bits(h);
              }
            }
          }
          tc::fence_async_smem();
          tc::fence_before_sync();
          bar_sync_n(my_bar_id, 128);
          if (issuer) {
            tc::fence_after_sync();
#pragma unroll
            for (int kb = 0; kb < 2; ++kb) {
#pragma unroll
              for (int kk = 0; kk < 4; ++kk) {
                const uint32_t ka = (uint32_t)(kb * 16384 + kk * 32);
                if (l == 0) {
                  // layer 2, swapped: A = W2^T [hidden][k], B = h1 [env][k]
                  const uint64_t da = tc::smem_desc(sb + C::OFF_W2P + ka, 16, 1024, tc::kSwizzle128B);
                  const uint64_t db = tc::smem_desc(hp_base + ka, 16, 1024, tc::kSwizzle128B);
                  tc::mma_bf16(tcol, da, db, idn, (kb | kk) != 0);
                } else {
                  // layer 3, normal: A = h2 [env rows][k], B = W3^T [class][k]
                  const uint64_t da = tc::smem_desc(hp_base + ka, 16, 1024, tc::kSwizzle128B);
                  const uint64_t db = tc::smem_desc(
                      sb + C::OFF_W3P + (uint32_t)(kb * kNPp * 128 + kk * 32), 16, 1024,
                      tc::kSwizzle128B);
                  tc::mma_bf16(tcol, da, db, id3, (kb | kk) != 0);
                }
              }
            }
            tc::mma_commit(bar);
          }
          if (!tc::mbar_wait(bar, ph, d.wait_ns) && !wfail) { wfail = true; fsite = 6 + (uint32_t)l; }
          ph ^= 1u;
          tc::fence_after_sync();
        }
        {
          uint32_t z[16];
          tmem_ld16(tm, z);
          tc::tmem_wait_ld();
          if (pt < n_env) {
            float lg[kNP];
#pragma unroll
            for (int c = 0; c < kNP; ++c)
              lg[c] = __uint_as_float(z[c]) + *(const float *)(sm + C::OFF_BIAS + (BO_B3P + c) * 4);
            const float u = u01(draw(seed, k, d.env_base + penv, kPlannerId, kTagAction, 0).x);
            float lp;
            const int tau = sample_cat<kNP>(lg, u, lp);
            ((int32_t *)d.r_act)[rowR * S + ps] = tau;
            d.r_logp[rowR * S + ps] = lp;
            if (d.dbg_logits) {
#pragma unroll
              for (int c = 0; c < kNP; ++c) d.pout[(size_t)penv * kNP + c] = lg[c];
#pragma unroll
              for (int c = 0; c < kNA; ++c)
                d.r_pout[(rowR * kNA + c) * S + ps] = c < kNP ? lg[c] : 0.f;
            }
            envi[pt].w = tau;
            const int t2 = t + 1;
            pdone = t2 >= (int)d.episode_limit;
            t = pdone ? 0 : t2;
          }
        }
        tc::fence_before_sync();
        ok = bar_all_n(kBarTax, C::THREADS, !wfail);
        if (!ok) break;
        bar_sync_n(kBarPool, C::THREADS);
      }
      if (ok && pt < n_env) d.t[penv] = t;
    }
    __syncthreads();
    if (!ok) break;
  }

  if (!ok) {
    if (r == 0 && (planner || tid < C::ROWS)) {
      // let any MMA still in flight finish before the columns are released
      tc::mma_commit(bars + AT + 1);
      tc::mbar_wait(bars + AT + 1, 0, tc::kDrainNs);
    }
    if (tid == 0) {
      atomicExch(d.err, 1u);
      atomicExch(d.err + 1, 300u + fsite);
    }
  }
  // the last CTA out resets the work queue for the next launch
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(d.queue + 1, 1u) == gridDim.x - 1) {
      d.queue[0] = 0u;
      d.queue[1] = 0u;
      __threadfence();
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tbase, C::TMEM_COLS);
  }
}

template <int AT>
struct Run {
  static cudaError_t go(const Dev &d, const void *packed, uint32_t n, int grid, cudaStream_t st) {
    k_econ_tc<AT><<<grid, EconTc<AT>::THREADS, EconTc<AT>::SMEM, st>>>(d, (const uint8_t *)packed, n);
    return cudaGetLastError();
  }
  static cudaError_t attr() {
    return cudaFuncSetAttribute(k_econ_tc<AT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                EconTc<AT>::SMEM);
  }
};

}  // namespace

bool econ_tc_supported(const PolicyShape &p, const PolicyShape &pp) {
  return p.w[0] == kEconF && p.w[1] == kH && p.w[2] == kH && p.w[3] == kNA && pp.w[0] == kEconF &&
         pp.w[1] == kH && pp.w[2] == kH && pp.w[3] == kNP;
}

size_t econ_tc_packed_bytes() { return (size_t)PACKED; }
int econ_tc_max_envs_per_item() { return kMaxEnvs; }

void launch_econ_tc_pack(const float *agent_params, const float *planner_params, void *packed,
                         cudaStream_t st) {
  k_econ_tc_pack<<<64, 256, 0, st>>>(agent_params, planner_params, (uint8_t *)packed);
}

void econ_tc_init() {
  Run<1>::attr();
  Run<2>::attr();
  Run<3>::attr();
}

cudaError_t launch_econ_tc(const Dev &d, const void *packed, uint32_t n_steps, int tiles, int grid,
                           cudaStream_t st) {
  if (tiles == 1) return Run<1>::go(d, packed, n_steps, grid, st);
  if (tiles == 2) return Run<2>::go(d, packed, n_steps, grid, st);
  if (tiles == 3) return Run<3>::go(d, packed, n_steps, grid, st);
  return cudaErrorInvalidValue;
}

}  // namespace ws
