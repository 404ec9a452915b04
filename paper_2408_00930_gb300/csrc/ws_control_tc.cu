// ws_control_tc.cu -- fused persistent BF16 tensor-core roll-out kernel of the
// classic-control envs (the cart-pole-like control env and the acrobot, paper
// App. C): one launch runs a whole chunk of steps for every env, with the env
// state held in registers and nothing but the transition records leaving the SM
// (paper Sec. 2 / App. B: roll-out, inference, reset and the in-place store all
// on the GPU; envs independent, policy referenced from GPU memory).  The two
// envs differ in the observation (4 state values; the acrobot's cos / sin of
// both angles and both velocities), the action count (2; 3) and the step
// (explicit Euler; RK4 of the two-link dynamics).
//
// Work split: a CTA holds two groups of 256 threads; each group owns a tile of
// 128 envs and 256 of the CTA's 512 TMEM columns.  Env row r of a tile is served
// by two threads ("halves" h = 0, 1; both in warps that may reach TMEM lane r),
// which split the row's hidden units by 64-unit blocks (by 32-unit halves of a
// 64-unit layer).  Per step and tile:
//   layer 1  z1 = o W1 + b1 on the tensor core, K = 16 (acrobot 32): the
//            operand row [o_hi, o_lo, o_hi, 1, 1, 0...] against [W1_hi; W1_hi;
//            W1_lo; b1_hi; b1_lo] keeps FP32-level accuracy (missing term
//            o_lo W1_lo ~ 2^-16); z1 lands in TMEM columns [0, H0)
//   act 1    h1 = tanh(z1) as packed bf16x2, written back into TMEM columns
//            [128, 128 + H0/2): the A operand of layer 2 stays in tensor memory
//            (two bf16 per 32-bit column), so it never touches shared memory
//   layer 2  z2 = h1 W2 + b2 in passes of up to 128 output units into TMEM
//            columns [0, 128): b2 by one K = 16 MMA of the K-chunk of the operand
//            row that holds its constant columns against [.., b2_hi, b2_lo, ..],
//            then H0 / 16 MMAs with A read from tensor memory and W2^T resident
//            in shared memory
//   layer 3  logits = tanh(z2) W3 + b3 on the CUDA cores after each pass: each
//            half reads its block of z2, applies tanh (FP32, SFU) and accumulates
//            its partial dot products with W3 (FP32, packed f32x2 FMAs, W3 read as
//            shared-memory broadcasts); half 1 hands its partial to half 0
//   then     half 0: categorical sample (Philox), env step, reward, done,
//            auto-reset, the time-major record write and the next operand row.
// Two threads per row give 16 warps per SM, so that one warp's MUFU/TMEM
// latency overlaps another's work, and the two groups' tensor and tanh phases
// interleave.  Tiles go to CTAs round-robin, group 0's turn first, so that
// every SM receives either floor or ceil of tiles / SMs.
#include "ws_acrobot.cuh"
#include "ws_kernels.cuh"
#include "ws_tc.cuh"

namespace ws {

namespace {

constexpr int kTile = 128;
constexpr int kGroups = 2;
constexpr int kGroupThreads = 2 * kTile;
constexpr int kThreads = kGroups * kGroupThreads;
constexpr uint32_t kTmemCols = 512;

// The two envs: observation width, actions, layer-1 K.
struct EnvCart {
  static constexpr int OBS = 4, NA = 2, K1 = 16;
};
struct EnvAcro {
  static constexpr int OBS = 6, NA = 3, K1 = 32;
};

template <typename E, int H0, int H1>
struct CtrlTc {
  static_assert(H0 == 64 || H0 == 128 || H0 == 256, "layer-2 K must be 64, 128 or 256");
  static_assert(H1 == 64 || H1 == 128 || H1 == 256, "layer-3 K (= H1) must be 64, 128 or 256");
  static constexpr int KB = H0 / 64;                // layer-2 K-blocks (1, 2 or 4)
  static constexpr int NP = H1 > 128 ? 2 : 1;       // layer-2 passes
  static constexpr int NPW = H1 / NP;               // output units per pass (64 or 128)
  static constexpr int KBP = NPW / 64;              // 64-unit blocks per pass (1 or 2)
  static constexpr uint32_t A_COL = 128;            // TMEM column of the layer-2 A operand
  static constexpr int K1 = E::K1;                  // layer-1 K (operand row length)
  static constexpr int KC = 3 * E::OBS;             // the operand row's first constant column
  static constexpr int W2_BYTES = KB * H1 * 128;    // B of layer 2, SW128, K-blocks of 64
  static constexpr int B1_BYTES = H0 * K1 * 2;      // B of layer 1, no swizzle
  static constexpr int BB_BYTES = H1 * 32;          // B of the b2 MMA, no swizzle, K = 16
  static constexpr int W3P = E::NA == 2 ? 16 : 32;  // W3 bytes per unit pair (FP32 float4s)
  static constexpr int W3_BYTES = H1 / 2 * W3P;
  static constexpr int B3V_BYTES = 16;              // b3
  // packed global image: [W2 | B1 | BB | W3 | b3]
  static constexpr int PK_W2 = 0;
  static constexpr int PK_B1 = PK_W2 + W2_BYTES;
  static constexpr int PK_BB = PK_B1 + B1_BYTES;
  static constexpr int PK_W3 = PK_BB + BB_BYTES;
  static constexpr int PK_B3V = PK_W3 + W3_BYTES;
  static constexpr int PACKED = PK_B3V + B3V_BYTES;
  // shared memory (from a 1024-aligned base)
  static constexpr int OFF_W2 = 0;
  static constexpr int OFF_A1 = OFF_W2 + W2_BYTES;  // [group] layer-1 operand [128][K1]
  static constexpr int OFF_B1 = OFF_A1 + kGroups * 128 * K1 * 2;
  static constexpr int OFF_BB = OFF_B1 + B1_BYTES;  // B1, BB, W3, b3 contiguous as packed
  static constexpr int OFF_W3 = OFF_BB + BB_BYTES;
  static constexpr int OFF_B3V = OFF_W3 + W3_BYTES;
  // [group][row] from half 1 to half 0: two logit partials, the action uniform,
  // the third logit partial (acrobot) and the four reset words (8 words, 32 B)
  static constexpr int OFF_XCH = OFF_B3V + B3V_BYTES;
  static constexpr int OFF_BAR = OFF_XCH + kGroups * 128 * 32;
  static constexpr int N_BAR = 3;  // per group: layer 1, layer-2 pass, error drain
  static constexpr int OFF_TOK = OFF_BAR + kGroups * N_BAR * 8;  // [group] SFU token barrier
  static constexpr int OFF_DONE = OFF_TOK + kGroups * 8;         // [group] finished flag
  static constexpr int OFF_TM = OFF_DONE + kGroups * 4;
  static constexpr int SMEM_NEED = OFF_TM + 16 + 1024;
  // at least 120 KB: one CTA per SM, so its 512 TMEM columns are uncontended
  static constexpr int SMEM = SMEM_NEED > 120 * 1024 ? SMEM_NEED : 120 * 1024;
  static_assert(SMEM_NEED <= 232448, "shared memory over the 227 KB per-CTA limit");
  static_assert(OFF_A1 % 1024 == 0 && OFF_B1 % 128 == 0 && OFF_BB % 128 == 0 && OFF_W3 % 16 == 0,
                "operand alignment");
  static_assert(A_COL + H0 / 2 <= 256, "the A operand must fit the group's TMEM columns");
};

__device__ __forceinline__ uint16_t bf16_bits(float f) {
  return (uint16_t)(tc::pack_bf16x2(f, 0.f) & 0xFFFFu);
}
__device__ __forceinline__ float bf16_val(float f) { return tc::bf16_lo(tc::pack_bf16x2(f, 0.f)); }

// Byte offset of element (row n, k) in a 128B-swizzled K-major operand of
// `rows` rows and K-blocks of 64 elements.
__device__ __forceinline__ int sw128_off(int n, int k, int rows) {
  const int kb = k >> 6, kk = k & 63;
  return kb * (rows * 128) + n * 128 + (((kk >> 3) ^ (n & 7)) << 4) + (kk & 7) * 2;
}
// Byte offset of element (row n, q) in an operand of K elements per row without
// swizzle (8-row core matrices of 16 B rows; K-adjacent core matrices 128 B apart).
__device__ __forceinline__ int kns_off(int n, int q, int K) {
  return (n >> 3) * (K * 16) + (q >> 3) * 128 + (n & 7) * 16 + (q & 7) * 2;
}

// Pack the FP32 policy into the byte images the kernel copies verbatim.
template <typename E, int H0, int H1>
__global__ void k_ctrl_tc_pack(const float *__restrict__ params, uint8_t *__restrict__ packed) {
  using C = CtrlTc<E, H0, H1>;
  constexpr int OBS = E::OBS, NA = E::NA;
  const float *W1 = params;          // [OBS][H0]
  const float *b1 = W1 + OBS * H0;   // [H0]
  const float *W2 = b1 + H0;         // [H0][H1]
  const float *b2 = W2 + H0 * H1;    // [H1]
  const float *W3 = b2 + H1;         // [H1][NA]
  const float *b3 = W3 + NA * H1;    // [NA]
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  // layer 2: B row n (output unit), K = input unit
  for (int i = tid; i < H0 * H1; i += stride) {
    const int n = i / H0, k = i % H0;
    *(uint16_t *)(packed + C::PK_W2 + sw128_off(n, k, H1)) = bf16_bits(W2[(size_t)k * H1 + n]);
  }
  // layer 3 per unit pair i (k = 2i): float4 {W3[k][0], W3[k+1][0], W3[k][1],
  // W3[k+1][1]}, and for three actions float4 {W3[k][2], W3[k+1][2], 0, 0}
  for (int i = tid; i < H1 / 2; i += stride) {
    const int k = 2 * i;
    *(float4 *)(packed + C::PK_W3 + C::W3P * i) =
        make_float4(W3[k * NA + 0], W3[(k + 1) * NA + 0], W3[k * NA + 1], W3[(k + 1) * NA + 1]);
    if (NA == 3)
      *(float4 *)(packed + C::PK_W3 + C::W3P * i + 16) =
          make_float4(W3[k * NA + 2], W3[(k + 1) * NA + 2], 0.f, 0.f);
  }
  // layer 1 row n: [W1_hi[.][n] | W1_hi[.][n] | W1_lo[.][n] | b1_hi, b1_lo | 0...]
  for (int i = tid; i < H0 * C::K1; i += stride) {
    const int n = i / C::K1, q = i % C::K1;
    float v = 0.f;
    if (q < 2 * OBS) {
      v = bf16_val(W1[(q % OBS) * H0 + n]);
    } else if (q < 3 * OBS) {
      const float w = W1[(q - 2 * OBS) * H0 + n];
      v = bf16_val(w - bf16_val(w));
    } else if (q == 3 * OBS) {
      v = bf16_val(b1[n]);
    } else if (q == 3 * OBS + 1) {
      v = bf16_val(b1[n] - bf16_val(b1[n]));
    }
    *(uint16_t *)(packed + C::PK_B1 + kns_off(n, q, C::K1)) = bf16_bits(v);
  }
  // b2 row n (K = 16, the chunk of the operand row with its constant columns):
  // b2_hi, b2_lo at the constant columns, 0 elsewhere
  for (int i = tid; i < H1 * 16; i += stride) {
    const int n = i / 16, q = i % 16;
    float v = 0.f;
    if (q == C::KC % 16) v = bf16_val(b2[n]);
    if (q == C::KC % 16 + 1) v = bf16_val(b2[n] - bf16_val(b2[n]));
    *(uint16_t *)(packed + C::PK_BB + kns_off(n, q, 16)) = bf16_bits(v);
  }
  if (tid == 0)
    *(float4 *)(packed + C::PK_B3V) = make_float4(b3[0], b3[1], NA == 3 ? b3[2] : 0.f, 0.f);
}

// 32 consecutive 32-bit TMEM columns of this thread's lane from registers.
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
      "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, "
      "%17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
      "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),
      "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]),
      "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]),
      "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// D[tmem] (+)= A[tmem] * B[smem]^T, issued by one thread.  A: M = 128 rows in
// the TMEM lanes, K along the columns, two bf16 per 32-bit column (lower K in
// the low half).
__device__ __forceinline__ void mma_bf16_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc,
                                            uint32_t idesc, bool accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
      "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"((uint32_t)accumulate)
      : "memory");
}

// 16 consecutive 32-bit TMEM columns of this thread's lane from registers.
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
      "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
      "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),
      "r"(r[15])
      : "memory");
}

// tanh of NC (32 or 64) accumulator columns at taddr, packed bf16x2 (32-column
// loads).
template <int NC>
__device__ __forceinline__ void tanh_block(uint32_t taddr, uint32_t (&hp)[NC / 2]) {
#pragma unroll
  for (int half = 0; half < NC / 32; ++half) {
    uint32_t z[32];
    tc::tmem_ld32(taddr + half * 32, z);
    tc::tmem_wait_ld();
#pragma unroll
    for (int i = 0; i < 16; ++i)
      hp[half * 16 + i] =
          tc::tanh_bf16x2(tc::pack_bf16x2(__uint_as_float(z[2 * i]), __uint_as_float(z[2 * i + 1])));
  }
}

__device__ __forceinline__ uint64_t f2(float lo, float hi) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ float2 unf2(uint64_t v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ float4 lds128f(uint32_t addr) {
  float4 v;
  asm("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(addr));
  return v;
}

// Layer 3 over one block of NC (32 or 64) units: tanh of the block's z2 columns (FP32 SFU
// tanh; the same SFU rate per value as the packed bf16x2 form, and no packing)
// against W3 in FP32.  acc0 / acc1 / acc2 hold (even-unit, odd-unit) partial
// sums of logits 0 / 1 / 2; w3 holds the block's unit pairs (W3P bytes each:
// float4 {W3[k][0], W3[k+1][0], W3[k][1], W3[k+1][1]}, k even, then for three
// actions float4 {W3[k][2], W3[k+1][2], 0, 0}).
template <int NA, int NC>
__device__ __forceinline__ void layer3_block(uint32_t taddr, uint32_t w3, uint64_t &acc0,
                                             uint64_t &acc1, uint64_t &acc2) {
  constexpr uint32_t W3P = NA == 2 ? 16u : 32u;
#pragma unroll
  for (int half = 0; half < NC / 32; ++half) {
    uint32_t z[32];
    tc::tmem_ld32(taddr + half * 32, z);
    tc::tmem_wait_ld();
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const uint32_t wa = w3 + W3P * (uint32_t)(half * 16 + j);
      const float4 q = lds128f(wa);
      const uint64_t hv = f2(tc::tanh_fast(__uint_as_float(z[2 * j])),
                             tc::tanh_fast(__uint_as_float(z[2 * j + 1])));
      acc0 = fma2(hv, f2(q.x, q.y), acc0);
      acc1 = fma2(hv, f2(q.z, q.w), acc1);
      if (NA == 3) {
        const float4 q2 = lds128f(wa + 16u);
        acc2 = fma2(hv, f2(q2.x, q2.y), acc2);
      }
    }
  }
}

// The SFU token.  The two groups of a CTA take turns in their layer-3 epilogues
// (tanh of z2 and the W3 dot products, after each layer-2 pass): one group's
// tanh work then runs while the other waits on its tensor-core pass, instead of
// both groups competing for the SFU at the same time.  (Measured: turns on the
// layer-3 epilogues alone beat turns on those plus act 1, and no turns at all,
// by 6 % and 25 %.)  tok[g] completes a phase when the other group's eight warps
// have handed the token over; a group that leaves its tile loop raises its done
// flag (and hands over once more), after which the other group runs alone.
struct SfuToken {
  uint32_t mine, theirs;       // shared addresses of tok[g], tok[1 - g]
  const volatile uint32_t *their_done;
  uint32_t ph;
  bool solo;
};
__device__ __forceinline__ void tok_take(SfuToken &t, uint64_t limit_ns) {
  if (t.solo) return;
  uint32_t res = 1;  // 1: token, 2: the other group finished, 0: wait limit reached
  if ((threadIdx.x & 31) == 0) {
    uint64_t *bar = (uint64_t *)__cvta_shared_to_generic(t.mine);
    if (!tc::mbar_try_wait(bar, t.ph)) {
      const uint64_t t0 = tc::global_ns();
      for (;;) {
        if (tc::mbar_try_wait(bar, t.ph)) break;
        if (*t.their_done) { res = 2; break; }
        if (tc::global_ns() - t0 > limit_ns) { res = 0; break; }
      }
    }
  }
  res = __shfl_sync(0xffffffffu, res, 0);
  if (res == 1) t.ph ^= 1u;
  else t.solo = true;  // the other group is gone (or stuck): no more turns to wait for
}
__device__ __forceinline__ void tok_give(const SfuToken &t) {
  __syncwarp();
  if ((threadIdx.x & 31) == 0)
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(t.theirs) : "memory");
}

// Barrier of the two warps (one per half) that serve the same 32 rows.
__device__ __forceinline__ void pair_sync(uint32_t id) {
  asm volatile("bar.sync %0, 64;" ::"r"(id) : "memory");
}

// Group-wide barrier (256 threads) and AND-vote.
__device__ __forceinline__ void grp_sync(uint32_t id) {
  asm volatile("bar.sync %0, 256;" ::"r"(id) : "memory");
}
__device__ __forceinline__ bool grp_all(uint32_t id, bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.and.pred q, %2, 256, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(id)
      : "memory");
  return r != 0;
}

template <typename E, int H0, int H1>
__global__ void __launch_bounds__(kThreads, 1)
    k_ctrl_tc(Dev d, const uint8_t *__restrict__ packed, uint32_t n_steps) {
  using C = CtrlTc<E, H0, H1>;
  constexpr bool ACRO = E::NA == 3;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = tc::smem_u32(smem_raw);
  uint8_t *sm = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
  const uint32_t sb = tc::smem_u32(sm);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int g = tid >> 8, h = (tid >> 7) & 1, r = tid & 127;
  uint64_t *bars = (uint64_t *)(sm + C::OFF_BAR) + g * C::N_BAR;
  uint64_t *bar_l1 = bars, *bar_l2 = bars + 1, *bar_drain = bars + 2;
  uint32_t *tm_holder = (uint32_t *)(sm + C::OFF_TM);

  // Stage the packed operands into shared memory.
  {
    const uint4 *src = (const uint4 *)(packed + C::PK_W2);
    uint4 *dst = (uint4 *)(sm + C::OFF_W2);
    for (int i = tid; i < C::W2_BYTES / 16; i += kThreads) dst[i] = __ldg(src + i);
    src = (const uint4 *)(packed + C::PK_B1);
    dst = (uint4 *)(sm + C::OFF_B1);  // B1, BB, W3, b3: contiguous in both
    constexpr int kSmall = (C::B1_BYTES + C::BB_BYTES + C::W3_BYTES + C::B3V_BYTES) / 16;
    for (int i = tid; i < kSmall; i += kThreads) dst[i] = __ldg(src + i);
  }
  if (tid == 0) {
    uint64_t *all = (uint64_t *)(sm + C::OFF_BAR);
    for (int i = 0; i < kGroups * C::N_BAR; ++i) tc::mbar_init(all + i, 1);
    for (int i = 0; i < kGroups; ++i) {
      tc::mbar_init((uint64_t *)(sm + C::OFF_TOK) + i, kGroupThreads / 32);
      ((volatile uint32_t *)(sm + C::OFF_DONE))[i] = 0u;
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tc::tmem_alloc(tm_holder, kTmemCols);
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();

  const uint32_t tmem = *tm_holder + (uint32_t)g * 256u;
  const uint32_t a_tm = tmem + C::A_COL;  // layer-2 A operand (h1), lane 0
  const uint32_t lane = (uint32_t)((warp & 3) * 32) << 16;
  const uint32_t bar_id = 1u + (uint32_t)g;
  const uint32_t pair_id = 3u + 4u * (uint32_t)g + (uint32_t)(warp & 3);
  const uint32_t a1 = sb + C::OFF_A1 + (uint32_t)g * 128 * (C::K1 * 2);
  const uint32_t a1_row = a1 + (uint32_t)(r >> 3) * (C::K1 * 16) + (uint32_t)(r & 7) * 16u;
  const uint32_t w3s = sb + C::OFF_W3;
  const uint32_t xch = sb + C::OFF_XCH + (uint32_t)g * 128 * 32 + (uint32_t)r * 32;
  const uint64_t desc_a1 = tc::smem_desc(a1, 128, C::K1 * 16, tc::kSwizzleNone);
  const uint64_t desc_b1 = tc::smem_desc(sb + C::OFF_B1, 128, C::K1 * 16, tc::kSwizzleNone);
  // the K = 16 chunk of the operand row that holds its constant columns (b2 MMA)
  const uint64_t desc_ac = tc::smem_desc(a1 + (uint32_t)(C::KC / 16) * 256u, 128, C::K1 * 16,
                                         tc::kSwizzleNone);
  const uint64_t desc_bb0 = tc::smem_desc(sb + C::OFF_BB, 128, 256, tc::kSwizzleNone);
  const uint64_t desc_w20 = tc::smem_desc(sb + C::OFF_W2, 16, 1024, tc::kSwizzle128B);
  constexpr uint32_t idesc1 = tc::idesc_bf16_f32(128, H0);
  constexpr uint32_t idesc2 = tc::idesc_bf16_f32(128, C::NPW);
  const float4 b3 = *(const float4 *)(sm + C::OFF_B3V);
  const bool issuer = (r == 0 && h == 0);

  uint32_t ph_l1 = 0u, ph_l2 = 0u;
  // group 0 holds the token first (parity 1 of a fresh barrier reads as complete)
  SfuToken tok{sb + C::OFF_TOK + 8u * (uint32_t)g, sb + C::OFF_TOK + 8u * (uint32_t)(g ^ 1),
               (const volatile uint32_t *)(sm + C::OFF_DONE) + (g ^ 1), g == 0 ? 1u : 0u, false};
  bool ok = true;
  uint32_t fail_site = 0;
  // Each thread waits on the MMA barriers itself; a wait that runs out is noted
  // and voted on once per step, at the group barrier that starts the next step
  // (reading TMEM columns an unfinished MMA still writes yields wrong values, not
  // a fault), so that the whole group leaves together.
  bool wfail = false;
  uint32_t fsite = 0;
  const uint64_t k0 = d.k[0];
  const uint64_t wlim = d.wait_ns;
  const uint32_t R = d.ring_steps;
  const uint32_t row0 = (uint32_t)(k0 % R);
  const uint32_t N = d.n_envs, S = d.n_slots;
  const int n_tiles = (int)((N + kTile - 1) / kTile);

  for (int tile = (int)blockIdx.x + (int)gridDim.x * g; ok && tile < n_tiles;
       tile += kGroups * (int)gridDim.x) {
    const uint32_t e = (uint32_t)tile * kTile + (uint32_t)r;
    const bool valid = e < N;
    float x = 0.f, v = 0.f, th = 0.f, w = 0.f;
    int tep = 0;
    if (valid && h == 0) {
      x = d.s[e];
      v = d.s[N + e];
      th = d.s[2 * N + e];
      w = d.s[3 * N + e];
      tep = d.t[e];
    }
    uint32_t row = row0;
    for (uint32_t j = 0; j < n_steps; ++j) {
      const uint32_t k = (uint32_t)(k0 + j);
      // ---- layer 1 operand row [o_hi | o_lo | o_hi | 1 1 0...] (half 0 holds the state)
      float ob[E::OBS];  // this step's observation (the record)
      if (h == 0) {
        if constexpr (ACRO) {
          acro_sincos<true>(x, &ob[1], &ob[0]);  // (th1, th2, w1, w2) in (x, v, th, w)
          acro_sincos<true>(v, &ob[3], &ob[2]);
          ob[4] = th;
          ob[5] = w;
          float oh[6];
#pragma unroll
          for (int i = 0; i < 6; ++i) oh[i] = bf16_val(ob[i]);
          const uint32_t h01 = tc::pack_bf16x2(oh[0], oh[1]), h23 = tc::pack_bf16x2(oh[2], oh[3]),
                         h45 = tc::pack_bf16x2(oh[4], oh[5]);
          const uint32_t l01 = tc::pack_bf16x2(ob[0] - oh[0], ob[1] - oh[1]);
          const uint32_t l23 = tc::pack_bf16x2(ob[2] - oh[2], ob[3] - oh[3]);
          const uint32_t l45 = tc::pack_bf16x2(ob[4] - oh[4], ob[5] - oh[5]);
          // K 0-7: h h h l | 8-15: l l h h | 16-23: h 1 0 0 | 24-31: 0
          tc::sts128(a1_row, h01, h23, h45, l01);
          tc::sts128(a1_row + 128, l23, l45, h01, h23);
          tc::sts128(a1_row + 256, h45, tc::pack_bf16x2(1.f, 1.f), 0u, 0u);
          tc::sts128(a1_row + 384, 0u, 0u, 0u, 0u);
        } else {
          ob[0] = x;
          ob[1] = v;
          ob[2] = th;
          ob[3] = w;
          const float xh = bf16_val(x), vh = bf16_val(v), thh = bf16_val(th), wh = bf16_val(w);
          const uint32_t hi01 = tc::pack_bf16x2(xh, vh), hi23 = tc::pack_bf16x2(thh, wh);
          tc::sts128(a1_row, hi01, hi23, tc::pack_bf16x2(x - xh, v - vh),
                     tc::pack_bf16x2(th - thh, w - wh));
          tc::sts128(a1_row + 128, hi01, hi23, tc::pack_bf16x2(1.f, 1.f), 0u);
        }
      }
      tc::fence_async_smem();
      tc::fence_before_sync();  // (also orders the last step's TMEM reads before the MMA)
      ok = grp_all(bar_id, !wfail);
      if (!ok) { fail_site = fsite ? fsite : 9u; break; }
      if (issuer) {
        tc::fence_after_sync();
#pragma unroll
        for (int q = 0; q < C::K1 / 16; ++q)
          tc::mma_bf16(tmem, desc_a1 + (uint64_t)(16 * q), desc_b1 + (uint64_t)(16 * q), idesc1,
                       q != 0);
        tc::mma_commit(bar_l1);
      }
      if (!tc::mbar_wait(bar_l1, ph_l1, wlim) && !wfail) { wfail = true; fsite = 1; }
      ph_l1 ^= 1u;
      tc::fence_after_sync();
      // ---- act 1: h1 block kb -> TMEM columns A_COL + 32 kb.  With H0 = 256, z1
      // blocks 2 and 3 share columns with the A operand: both halves read them
      // (and the pair barrier orders those reads) before anything is written.
      if (C::KB == 4) {
        uint32_t hp[32];
        tanh_block<64>(tmem + lane + (uint32_t)((h + 2) * 64), hp);
        pair_sync(pair_id);
        tmem_st32(a_tm + lane + (uint32_t)((h + 2) * 32), hp);
      }
      if (C::KB == 1) {
        // 64 units: each half takes 32 (the SFU work of a row on both threads)
        uint32_t hp[16];
        tanh_block<32>(tmem + lane + (uint32_t)(h * 32), hp);
        tmem_st16(a_tm + lane + (uint32_t)(h * 16), hp);
      } else if (h < C::KB) {
        uint32_t hp[32];
        tanh_block<64>(tmem + lane + (uint32_t)(h * 64), hp);
        tmem_st32(a_tm + lane + (uint32_t)(h * 32), hp);
      }
      tmem_wait_st();
      // ---- layer 2 in passes of NPW output units; layer 3 after each pass
      uint64_t acc0 = 0ull, acc1 = 0ull, acc2 = 0ull;  // (+0.f, +0.f) pairs
      float sin_th = 0.f, cos_th = 0.f;
#pragma unroll
      for (int p = 0; p < C::NP; ++p) {
        tc::fence_before_sync();
        grp_sync(bar_id);  // A complete (p = 0) / the last pass's columns read (p = 1)
        if (issuer) {
          tc::fence_after_sync();
          // descriptors as base + offset (the start address field is the low 14 bits,
          // in 16 B units); the empty asm keeps the compiler from holding all of them
          // in registers across the step loop
          uint64_t dbb = desc_bb0, dw2 = desc_w20;
          asm volatile("" : "+l"(dbb), "+l"(dw2));
          tc::mma_bf16(tmem, desc_ac, dbb + (uint64_t)((p * C::NPW * 32) >> 4), idesc2,
                       false);  // b2
#pragma unroll
          for (int kb = 0; kb < C::KB; ++kb) {
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
              mma_bf16_ts(tmem, a_tm + (uint32_t)(kb * 32 + kk * 8),
                          dw2 + (uint64_t)((kb * (H1 * 128) + p * C::NPW * 128 + kk * 32) >> 4),
                          idesc2, true);
          }
          tc::mma_commit(bar_l2);
        }
        if (p == 0) {
          // while the pass runs: half 1 draws this step's action uniform and reset
          // words for half 0; half 0 takes sin / cos of the pole angle
          if (h == 1) {
            const float ud = u01(draw(d.seed, k, d.env_base + e, 0, kTagAction, 0).x);
            const uint4 rr = draw(d.seed, k, d.env_base + e, 0, kTagReset, 0);
            asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(xch + 16), "r"(rr.x),
                         "r"(rr.y), "r"(rr.z), "r"(rr.w)
                         : "memory");
            asm volatile("st.shared.f32 [%0], %1;" ::"r"(xch + 8), "f"(ud) : "memory");
          } else if constexpr (!ACRO) {
            sin_th = sinf(th);
            cos_th = cosf(th);
          }
        }
        if (!tc::mbar_wait(bar_l2, ph_l2, wlim) && !wfail) { wfail = true; fsite = 2 + (uint32_t)p; }
        ph_l2 ^= 1u;
        tc::fence_after_sync();
        tok_take(tok, wlim);
        if (C::NPW == 64)  // 64 units per pass: each half takes 32
          layer3_block<E::NA, 32>(tmem + lane + (uint32_t)(h * 32),
                                  w3s + (uint32_t)((p * C::NPW + h * 32) / 2 * C::W3P), acc0, acc1,
                                  acc2);
        else if (h < C::KBP)
          layer3_block<E::NA, 64>(tmem + lane + (uint32_t)(h * 64),
                                  w3s + (uint32_t)((p * C::NPW + h * 64) / 2 * C::W3P), acc0,
                                  acc1, acc2);
        tok_give(tok);
      }
      const float2 pa = unf2(acc0), pb = unf2(acc1), pc = unf2(acc2);
      const float p0 = pa.x + pa.y, p1 = pb.x + pb.y, p2 = pc.x + pc.y;
      if (h == 1) {
        asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(xch), "f"(p0), "f"(p1) : "memory");
        if (ACRO) asm volatile("st.shared.f32 [%0], %1;" ::"r"(xch + 12), "f"(p2) : "memory");
      }
      pair_sync(pair_id);
      if (h == 0) {
        float q0, q1, q2 = 0.f, u;
        asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(q0), "=f"(q1) : "r"(xch) : "memory");
        asm volatile("ld.shared.f32 %0, [%1];" : "=f"(u) : "r"(xch + 8) : "memory");
        if (ACRO) asm volatile("ld.shared.f32 %0, [%1];" : "=f"(q2) : "r"(xch + 12) : "memory");
        const float l0 = (p0 + q0) + b3.x, l1v = (p1 + q1) + b3.y, l2 = (p2 + q2) + b3.z;
        // ---- sample by inverse CDF: a = min{ i : u S < C_i } (C_i running sums
        // of exp(l - max), S the total), as the per-step sampler
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
        // ---- env step, reward, done, auto-reset
        float ns[4];
        float rew;
        bool done;
        const int t2 = tep + 1;
        if constexpr (ACRO) {
          // RK4 of the two-link dynamics, dt = 0.2, torque a - 1
          ns[0] = x;
          ns[1] = v;
          ns[2] = th;
          ns[3] = w;
          acro_step<true>(ns, (float)(a - 1), 0.2f);
          const bool term = acro_terminal<true>(ns);
          rew = term ? 0.0f : -1.0f;
          done = term || t2 >= (int)d.episode_limit;
        } else {
          // explicit Euler, dt = 0.02
          const float uf = a ? 10.0f : -10.0f;
          const float xacc = uf - 0.5f * x - 0.1f * v;
          const float thacc = 9.8f * sin_th - 0.3f * cos_th * uf;
          ns[0] = x + 0.02f * v;
          ns[1] = v + 0.02f * xacc;
          ns[2] = th + 0.02f * w;
          ns[3] = w + 0.02f * thacc;
          rew = 1.0f;
          done = fabsf(ns[0]) > 2.4f || fabsf(ns[2]) > 0.21f || t2 >= (int)d.episode_limit;
        }
        if (valid) {
          const float lp = (la - m) - logf(Ssum);
          const size_t o = (size_t)row * S + e;
          float *obr = d.r_obs + (size_t)row * E::OBS * S + e;
#pragma unroll
          for (int i = 0; i < E::OBS; ++i) obr[(size_t)i * S] = ob[i];
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
        if (done) {
          uint4 rr;
          asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];"
                       : "=r"(rr.x), "=r"(rr.y), "=r"(rr.z), "=r"(rr.w)
                       : "r"(xch + 16)
                       : "memory");
          const float lim = ACRO ? 0.1f : 0.05f;
          x = uniform(rr.x, -lim, lim);
          v = uniform(rr.y, -lim, lim);
          th = uniform(rr.z, -lim, lim);
          w = uniform(rr.w, -lim, lim);
          tep = 0;
        } else {
          x = ns[0];
          v = ns[1];
          th = ns[2];
          w = ns[3];
          tep = t2;
        }
      }
      row = (row + 1 == R) ? 0 : row + 1;
    }
    if (valid && h == 0) {
      d.s[e] = x;
      d.s[N + e] = v;
      d.s[2 * N + e] = th;
      d.s[3 * N + e] = w;
      d.t[e] = tep;
    }
  }
  // a wait that ran out in the last step of the last tile
  if (ok) {
    ok = grp_all(bar_id, !wfail);
    if (!ok) fail_site = fsite ? fsite : 9u;
  }
  // this group is finished: release the other group from the turn-taking
  __syncwarp();
  if ((tid & 31) == 0) {
    ((volatile uint32_t *)(sm + C::OFF_DONE))[g] = 1u;
    __threadfence_block();
  }
  tok_give(tok);
  if (!ok && issuer) {
    // let any MMA still in flight finish before the columns are released
    tc::mma_commit(bar_drain);
    tc::mbar_wait(bar_drain, 0, tc::kDrainNs);
    atomicExch(d.err, 1u);
    atomicExch(d.err + 1, 100u + fail_site);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(*tm_holder, kTmemCols);
  }
}

template <typename E, int H0, int H1>
struct Shape {
  using C = CtrlTc<E, H0, H1>;
  static constexpr size_t packed_bytes = C::PACKED;
  static void pack(const Dev &d, void *packed, cudaStream_t st) {
    k_ctrl_tc_pack<E, H0, H1><<<64, 256, 0, st>>>(d.params, (uint8_t *)packed);
  }
  static cudaError_t run(const Dev &d, const void *packed, uint32_t n, int grid, cudaStream_t st) {
    k_ctrl_tc<E, H0, H1><<<grid, kThreads, C::SMEM, st>>>(d, (const uint8_t *)packed, n);
    return cudaGetLastError();
  }
  static cudaError_t attr() {
    return cudaFuncSetAttribute(k_ctrl_tc<E, H0, H1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                C::SMEM);
  }
};

template <typename E, typename F>
bool dispatch_env(const PolicyShape &sh, F &&f) {
  if (sh.w[1] == 256 && sh.w[2] == 256) return f(Shape<E, 256, 256>()), true;
  if (sh.w[1] == 128 && sh.w[2] == 128) return f(Shape<E, 128, 128>()), true;
  if (sh.w[1] == 64 && sh.w[2] == 64) return f(Shape<E, 64, 64>()), true;
  return false;
}

// The policy's input and output widths name the env: 4 -> 2 the control env,
// 6 -> 3 the acrobot.
template <typename F>
bool dispatch(const PolicyShape &sh, F &&f) {
  if (sh.w[0] == EnvCart::OBS && sh.w[3] == EnvCart::NA) return dispatch_env<EnvCart>(sh, f);
  if (sh.w[0] == EnvAcro::OBS && sh.w[3] == EnvAcro::NA) return dispatch_env<EnvAcro>(sh, f);
  return false;
}

}  // namespace

size_t control_tc_packed_bytes(const PolicyShape &sh) {
  size_t n = 0;
  dispatch(sh, [&](auto s) { n = decltype(s)::packed_bytes; });
  return n;
}

bool control_tc_supported(const PolicyShape &sh) {
  return dispatch(sh, [](auto) {});
}

void launch_control_tc_pack(const Dev &d, void *packed, cudaStream_t st) {
  dispatch(d.pol, [&](auto s) { s.pack(d, packed, st); });
}

cudaError_t launch_control_tc(const Dev &d, const void *packed, uint32_t n_steps, int grid,
                              cudaStream_t st) {
  cudaError_t e = cudaErrorNotSupported;
  dispatch(d.pol, [&](auto s) { e = s.run(d, packed, n_steps, grid, st); });
  return e;
}

int control_tc_default_grid(const Dev &d) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  dispatch(d.pol, [](auto s) { s.attr(); });
  const int tiles = (int)((d.n_envs + kTile - 1) / kTile);
  return tiles < sms ? tiles : sms;
}

}  // namespace ws
