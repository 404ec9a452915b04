// ws_land_tc.cu -- fused persistent BF16 tensor-core roll-out kernel of the
// reaction-path landscape: one launch runs a whole chunk of steps for every
// env, keeping each env's coordinates in registers.
//
// Paper grounding: App. C (catalytic reactions) has the agent move atoms on a
// first-principles energy landscape and be rewarded by the energy change; App.
// B / Sec. 2 keep roll-out, inference and reset on the GPU.  The stand-in
// landscape is a sum of M Gaussians, E(x) = sum_m a_m exp(-|x - c_m|^2 / (2 w_m^2)).
//
// A tile of 128 envs is served by a cluster of CL CTAs (CL = 1 or 2; a launch
// parameter).  Every CTA of the cluster runs the same policy and sampling for
// the tile (identical inputs and instruction streams give identical results)
// and sweeps its own 1/CL of the Gaussians; the partial energies meet through
// distributed shared memory.  Per step:
//   policy   24-256-256-48 on tcgen05: layer 1 from the coordinates (K = 32,
//            the bias in two constant columns), h1 and h2 written back to tensor
//            memory as the A operand of the next layer (packed BF16), W2^T / W3^T
//            resident in shared memory
//   sample   diagonal Gaussian head: mean, log sigma clamped to [-5, 2],
//            dx = clip(mean + sigma z) with Philox normals; log-probability of the
//            unclipped sample
//   energy   E(y) at y = x + dx, whole exponents on tcgen05: with q_m =
//            -log2(e) / (2 w_m^2), q_m |y - c_m|^2 + log2|a_m| = -2 q_m y.c_m +
//            (q_m |c_m|^2 + log2|a_m|) + q_m |y|^2 is one dot product of the
//            operand row [y, 1, |y|^2] with the Gaussian row [-2 q c,
//            q |c|^2 + log2|a|, q], every product split BF16 hi+lo (FP32
//            accumulate).  The Gaussians are grouped by the sign of a_m, so the
//            epilogue is one ex2 per pair summed into a positive and a negative
//            part (each sign group padded to 128 Gaussians).  The operand row
//            sits in tensor memory as the A operand; blocks of 128 Gaussians
//            stream through two shared-memory buffers (a loader warp that
//            polls each block's MMA completion) into three 128-column TMEM
//            accumulators (two MMA warps taking the even and the odd blocks,
//            one M = 128, N = 128 MMA per K step); the two threads of a row
//            take the blocks of even and odd index.
//   step     observed energy with Philox noise, reward Eobs(x) - Eobs(x'), done
//            at the episode limit or when E(y) falls below the energy target
//            (the product basin of App. C), reset to U(-3, 3)^D and a second
//            sweep for the fresh state's energy when a tile has a reset
// Threads: warps 0-3 own the env rows (state, sampling, records); warps 4-7
// take the other half of every tanh and exp epilogue; warp 8 loads the energy
// blocks, warps 9 and 10 issue the energy MMAs.  The step's Philox normals are
// drawn while the layer-2 MMA runs.  Every wait is bounded; a wait that
// runs out sets the error flag and the CTA leaves its loops at the next step
// boundary.
#include "ws_kernels.cuh"
#include "ws_tc.cuh"

namespace ws {

namespace {

constexpr int kRows = 128;
constexpr int kH = 256;                       // hidden width of both layers
constexpr int kMaxD = 24;                     // coordinates (a multiple of 8, <= 24)
constexpr int kN3 = 48;                       // layer-3 N (2 D, padded to 48)
constexpr int kK1 = 32;                       // layer-1 K: D coordinates, 1, 1, zeros
constexpr int kKE = 80;                       // energy K: 3 D + 5 <= 80, five K16 steps
constexpr int kBlk = 64;                      // Gaussians per block of the energy image
constexpr int kBlkBytes = kBlk * kKE * 2;     // block image, K = 80 without swizzle
constexpr int kEB = 128;                      // Gaussians per energy MMA of the roll-out sweep
constexpr int kEBBytes = kEB * kKE * 2;       // two consecutive image blocks
constexpr int kNS = 2;                        // shared-memory sweep-block buffers
constexpr int kNT = 3;                        // TMEM accumulators of the sweep (128 columns each)
constexpr int kHdr = 256;                     // energy image header: {blocks, positive blocks}
constexpr int kEpi = 256, kThreads = kEpi + 64;  // + a loader warp and an MMA warp
// The roll-out kernel issues its sweep MMAs from two warps that take the even
// and the odd blocks, so that one warp's waits run while the other's MMAs
// keep the tensor core busy.
constexpr int kMmaWarps = 2;
constexpr int kRollThreads = kEpi + 32 * (1 + kMmaWarps);
constexpr uint64_t kWaitNs = 2000000000ull;

// Packed policy image (copied verbatim to shared memory offset 0):
//   W2^T SW128 [256 n][256 k] | W3^T SW128 [48 n][256 k] | W1^T [256 n][32 k]
//   (no swizzle; columns D, D+1 hold b1_hi, b1_lo) | b2 f32 [256] | b3 f32 [64]
constexpr int PK_W2 = 0;
constexpr int PK_W3 = PK_W2 + 4 * kH * 128;
constexpr int PK_W1 = PK_W3 + 4 * kN3 * 128;
constexpr int PK_B2 = PK_W1 + kH * kK1 * 2;
constexpr int PK_B3 = PK_B2 + kH * 4;
constexpr int POLICY = PK_B3 + 64 * 4;

// shared memory
constexpr int OFF_AE = POLICY;                    // layer-1 A [128][32] (the energy A is in TMEM)
constexpr int OFF_BE = OFF_AE + kRows * kK1 * 2;  // kNS energy B blocks of kEB Gaussians
constexpr int OFF_XCH = OFF_BE + kNS * kEBBytes;  // f32 [128] each: partial energy, log-probability,
                                                  // |y|^2 of half 0 and of half 1
constexpr int OFF_RECV = OFF_XCH + 4 * kRows * 4; // f32 [2][128] the cluster partner's partials
constexpr int OFF_BAR = OFF_RECV + 2 * kRows * 4;
constexpr int N_BAR = 5 + kNS + 2 * kNT;  // ae, b[kNS], mma[kNT], epi[kNT], pol, x, drain, drain_pol
// [0] sweep command, [1] end flag, [2] blocks loaded, [4 + w] blocks MMA warp w passed
constexpr int OFF_CMD = OFF_BAR + N_BAR * 8;
constexpr int OFF_TM = OFF_CMD + 32;
constexpr int SMEM = OFF_TM + 16 + 1024;
static_assert(SMEM <= 232448, "shared memory over the 227 KB per-CTA limit");
static_assert(PK_W3 % 1024 == 0 && (4 * kN3 * 128) % 1024 == 0 && (kN3 * 128) % 1024 == 0,
              "SW128 alignment");
static_assert(OFF_AE % 128 == 0 && OFF_BE % 16 == 0 && OFF_BAR % 8 == 0, "alignment");

constexpr uint32_t TM_H = 256;   // TMEM columns of h1 / h2 (packed BF16 A operand)
constexpr uint32_t TM_A = 448;   // TMEM columns of the energy A operand [128][80] (BF16 pairs)
constexpr uint32_t TM_E = 0;     // TMEM columns of the energy accumulators (during a sweep the
                                 // policy's columns are free)
static_assert(TM_E + kNT * kEB <= TM_A && TM_A + kKE / 2 <= 512, "energy accumulators and A");
static_assert(TM_H + kH / 2 <= TM_A, "the policy's A operand below the energy A");

__device__ __forceinline__ uint16_t bf16_bits(float f) {
  return (uint16_t)(tc::pack_bf16x2(f, 0.f) & 0xFFFFu);
}
__device__ __forceinline__ float bf16_val(float f) { return tc::bf16_lo(tc::pack_bf16x2(f, 0.f)); }
__device__ __forceinline__ int sw128_off(int n, int k, int rows) {
  const int kb = k >> 6, kk = k & 63;
  return kb * (rows * 128) + n * 128 + (((kk >> 3) ^ (n & 7)) << 4) + (kk & 7) * 2;
}
// Element (row n, k) of a K-major operand without swizzle with K elements per
// row: 8-row core matrices of 16-byte rows, K-adjacent core matrices 128 B apart.
__device__ __forceinline__ int ns_off(int n, int k, int K) {
  return (n >> 3) * (K * 16) + (k >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2;
}

__global__ void k_land_tc_pack_policy(const float *__restrict__ p, int D, uint8_t *__restrict__ out) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  const float *W1 = p, *b1 = W1 + D * kH, *W2 = b1 + kH, *b2 = W2 + kH * kH;
  const float *W3 = b2 + kH, *b3 = W3 + kH * 2 * D;
  for (int i = tid; i < kH * kH; i += stride) {
    const int n = i / kH, k = i % kH;
    *(uint16_t *)(out + PK_W2 + sw128_off(n, k, kH)) = bf16_bits(W2[k * kH + n]);
  }
  for (int i = tid; i < kN3 * kH; i += stride) {
    const int n = i / kH, k = i % kH;
    *(uint16_t *)(out + PK_W3 + sw128_off(n, k, kN3)) = bf16_bits(n < 2 * D ? W3[k * 2 * D + n] : 0.f);
  }
  for (int i = tid; i < kH * kK1; i += stride) {
    const int n = i / kK1, q = i % kK1;
    float v = 0.f;
    if (q < D) v = W1[q * kH + n];
    else if (q == D) v = bf16_val(b1[n]);
    else if (q == D + 1) v = b1[n] - bf16_val(b1[n]);
    *(uint16_t *)(out + PK_W1 + ns_off(n, q, kK1)) = bf16_bits(v);
  }
  for (int i = tid; i < kH; i += stride) ((float *)(out + PK_B2))[i] = b2[i];
  for (int i = tid; i < 64; i += stride) ((float *)(out + PK_B3))[i] = i < 2 * D ? b3[i] : 0.f;
}

// Energy image: a header {block count (even), blocks of non-negative
// amplitude}, the slot order (Gaussian index per slot, -1 for padding), then per
// block of 64 slots the B operand rows (K = 80, no swizzle)
//   [v_hi (D) | v_lo (D) | v_hi (D) | s_hi, s_lo | q_hi, q_lo, q_hi | 0...]
// with v = -2 q c, q = -log2(e) / (2 w^2) and s = q |c|^2 + log2 |a|, against the
// operand row [y_hi | y_hi | y_lo | 1, 1 | yy_hi, yy_hi, yy_lo | 0...] (yy = |y|^2):
// the dot product is log2(|a_m| exp(-|y - c_m|^2 / (2 w_m^2))).  Gaussians with
// a >= 0 fill the first blocks and those with a < 0 the rest (each group padded
// to whole sweep blocks of kEB = 2 image blocks, the block count a multiple of 4
// so that the two CTAs of a pair sweep whole sweep blocks), so that a sweep
// block's sign is one flag; padding slots carry s = -200 (2^-200 flushes to
// zero).  The header counts image blocks of 64.
inline int land_slots(int M) { return ((M + kBlk - 1) / kBlk + 8) * kBlk; }
inline size_t land_order_off() { return (size_t)kHdr; }
inline size_t land_blocks_off(int M) { return kHdr + ((size_t)land_slots(M) * 4 + 255) / 256 * 256; }

__global__ void k_land_tc_order(const float *__restrict__ a, int M, int slots,
                                int32_t *__restrict__ hdr, int32_t *__restrict__ order) {
  __shared__ int cnt[1024], base_p[1024], base_n[1024];
  const int t = threadIdx.x, T = blockDim.x;
  const int per = (M + T - 1) / T, lo = t * per, hi = min(M, lo + per);
  int np = 0;
  for (int m = lo; m < hi; ++m) np += a[m] >= 0.f;
  cnt[t] = np;
  for (int s = t; s < slots; s += T) order[s] = -1;
  __syncthreads();
  if (t == 0) {  // exclusive scans of the group counts, in thread order (stable)
    int p = 0, n = 0;
    for (int i = 0; i < T; ++i) {
      const int li = min(M, i * per), hi_i = min(M, li + per), len = max(0, hi_i - li);
      base_p[i] = p;
      base_n[i] = n;
      p += cnt[i];
      n += len - cnt[i];
    }
    const int pb = (p + kEB - 1) / kEB * 2, nb = (n + kEB - 1) / kEB * 2;
    hdr[0] = (pb + nb + 3) / 4 * 4;
    hdr[1] = pb;
    cnt[0] = pb * kBlk;  // first slot of the negative group
  }
  __syncthreads();
  const int neg0 = cnt[0];
  int ip = base_p[t], in = base_n[t];
  for (int m = lo; m < hi; ++m) {
    if (a[m] >= 0.f) order[ip++] = m;
    else order[neg0 + in++] = m;
  }
}

__global__ void k_land_tc_pack_energy(const float *__restrict__ c, const float *__restrict__ w,
                                      const float *__restrict__ a, int D, int slots,
                                      const int32_t *__restrict__ order, uint8_t *__restrict__ img) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  for (int i = tid; i < slots * kKE; i += stride) {
    const int sl = i / kKE, k = i % kKE, m = order[sl];
    float v = 0.f;
    if (m < 0) {
      if (k == 3 * D) v = -200.f;
    } else if (k < 3 * D + 5) {
      const float q = -1.4426950408889634f / (2.0f * w[m] * w[m]);
      if (k < 3 * D) {
        const float x = -2.0f * q * c[(size_t)m * D + (k % D)];
        v = (k / D == 1) ? x - bf16_val(x) : x;
      } else if (k < 3 * D + 2) {
        float s = 0.f;
        for (int j = 0; j < D; ++j) s = fmaf(c[(size_t)m * D + j], c[(size_t)m * D + j], s);
        const float x = fmaf(q, s, fmaxf(log2f(fabsf(a[m])), -200.f));
        v = k == 3 * D ? x : x - bf16_val(x);
      } else {
        v = k == 3 * D + 3 ? q - bf16_val(q) : q;
      }
    }
    *(uint16_t *)(img + (size_t)(sl / kBlk) * kBlkBytes + ns_off(sl % kBlk, k, kKE)) = bf16_bits(v);
  }
}

// ---- helpers ---------------------------------------------------------------------
__device__ __forceinline__ void bar_sync_n(uint32_t id, uint32_t n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
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
__device__ __forceinline__ bool bar_any_n(uint32_t id, uint32_t n, bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.or.pred q, %2, %3, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(id), "r"(n)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(tc::smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}
__device__ __forceinline__ float ex2_fast(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// Exponentials of 32 accumulator columns summed into s[0..3] (by column mod 4).
__device__ __forceinline__ void ex2_sum32(const uint32_t (&z)[32], float (&s)[4]) {
#pragma unroll
  for (int c = 0; c < 32; ++c) s[c & 3] += ex2_fast(__uint_as_float(z[c]));
}
// tcgen05.wait::ld with the loaded registers as operands, so that no use of
// them can be scheduled before the wait.
__device__ __forceinline__ void tmem_wait_ld_regs(uint32_t (&z)[32]) {
  asm volatile(
      "tcgen05.wait::ld.sync.aligned;"
      : "+r"(z[0]), "+r"(z[1]), "+r"(z[2]), "+r"(z[3]), "+r"(z[4]), "+r"(z[5]), "+r"(z[6]),
        "+r"(z[7]), "+r"(z[8]), "+r"(z[9]), "+r"(z[10]), "+r"(z[11]), "+r"(z[12]), "+r"(z[13]),
        "+r"(z[14]), "+r"(z[15]), "+r"(z[16]), "+r"(z[17]), "+r"(z[18]), "+r"(z[19]), "+r"(z[20]),
        "+r"(z[21]), "+r"(z[22]), "+r"(z[23]), "+r"(z[24]), "+r"(z[25]), "+r"(z[26]), "+r"(z[27]),
        "+r"(z[28]), "+r"(z[29]), "+r"(z[30]), "+r"(z[31])
      :
      : "memory");
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
// NC consecutive 32-bit TMEM columns of this thread's lane from registers.
template <int NC>
__device__ __forceinline__ void tmem_st_cols(uint32_t taddr, const uint32_t (&w)[NC]) {
  int c = 0;
#pragma unroll
  for (; c + 4 <= NC; c += 4)
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr + c),
                 "r"(w[c]), "r"(w[c + 1]), "r"(w[c + 2]), "r"(w[c + 3])
                 : "memory");
#pragma unroll
  for (; c + 2 <= NC; c += 2)
    asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1, %2};" ::"r"(taddr + c), "r"(w[c]),
                 "r"(w[c + 1])
                 : "memory");
#pragma unroll
  for (; c < NC; ++c)
    asm volatile("tcgen05.st.sync.aligned.32x32b.x1.b32 [%0], {%1};" ::"r"(taddr + c), "r"(w[c])
                 : "memory");
}
// D[tmem] (+)= A[tmem] * B[smem]^T (A: 128 lanes, two bf16 per column).
__device__ __forceinline__ void mma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc,
                                      uint32_t idesc, bool acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
      "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"((uint32_t)acc)
      : "memory");
}
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}
__device__ __forceinline__ uint32_t mapa(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
__device__ __forceinline__ void st_cluster_f32(uint32_t addr, float v) {
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}
__device__ __forceinline__ void arrive_remote(uint32_t addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(addr) : "memory");
}
// Bounded wait with cluster-scope acquire (for arrivals from the partner CTA).
__device__ __forceinline__ bool mbar_wait_cluster(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
  const uint32_t a = tc::smem_u32(bar);
  const bool short_lim = limit_ns < tc::kShortWaitNs;
  uint64_t t0 = 0;
  for (int it = 0;; ++it) {
    uint32_t ok;
    if (short_lim)  // a poll that never suspends (see tc::mbar_test_wait)
      asm volatile(
          "{\n\t.reg .pred p;\n\t"
          "mbarrier.test_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
          "selp.u32 %0, 1, 0, p;\n\t}"
          : "=r"(ok)
          : "r"(a), "r"(parity)
          : "memory");
    else
      asm volatile(
          "{\n\t.reg .pred p;\n\t"
          "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
          "selp.u32 %0, 1, 0, p;\n\t}"
          : "=r"(ok)
          : "r"(a), "r"(parity)
          : "memory");
    if (ok) return true;
    if (short_lim) {  // the SM clock, 2 cycles per ns
      if (it == 0) t0 = tc::sm_clock();
      else if (tc::sm_clock() - t0 > 2 * limit_ns) return false;
    } else if (it == 0) {
      t0 = tc::global_ns();
    } else if ((it & 255) == 0 && tc::global_ns() - t0 > limit_ns) {
      return false;
    }
  }
}

// Barrier ids: 1 the 256 epilogue threads; 2 + w the two warps (w, w + 4) of rows
// 32w..; 6 the producer warps.
constexpr uint32_t kBarEpi = 1, kBarPair0 = 2, kBarProd = 6;

template <int D, int CL>
__global__ void __launch_bounds__(kRollThreads, 1)
    k_land_tc(Dev d, const uint8_t *__restrict__ pol, const uint8_t *__restrict__ eimg,
              const uint8_t *__restrict__ blocks, uint32_t n_steps) {
  constexpr int DH = D / 2;  // coordinates per thread of a row (two threads per row)
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = tc::smem_u32(smem_raw);
  uint8_t *sm = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
  const uint32_t sb = tc::smem_u32(sm);
  const int tid = threadIdx.x, warp = tid >> 5;
  uint64_t *bars = (uint64_t *)(sm + OFF_BAR);
  uint64_t *bar_ae = bars, *bar_b = bars + 1, *bar_mma = bar_b + kNS, *bar_epi = bar_mma + kNT;
  uint64_t *bar_pol = bar_epi + kNT, *bar_x = bar_pol + 1, *bar_drain = bar_x + 1;
  uint64_t *bar_drain_pol = bar_drain + 1;
  volatile uint32_t *cmd = (volatile uint32_t *)(sm + OFF_CMD);
  uint32_t *tm_holder = (uint32_t *)(sm + OFF_TM);
  const uint32_t rank = CL > 1 ? cluster_rank() : 0u;

  {
    const uint4 *src = (const uint4 *)pol;
    uint4 *dst = (uint4 *)sm;
    for (int i = tid; i < POLICY / 16; i += kRollThreads) dst[i] = __ldg(src + i);
  }
  if (tid == 0) {
    tc::mbar_init(bar_ae, kEpi);
    for (int i = 0; i < kNS; ++i) tc::mbar_init(bar_b + i, 1);
    for (int i = 0; i < kNT; ++i) {
      tc::mbar_init(bar_mma + i, 1);
      tc::mbar_init(bar_epi + i, kRows);  // the half that evaluates the block
    }
    tc::mbar_init(bar_pol, 1);
    tc::mbar_init(bar_x, kRows);
    tc::mbar_init(bar_drain, kMmaWarps);
    tc::mbar_init(bar_drain_pol, 1);
    cmd[0] = 0u;
    cmd[1] = 0u;
    cmd[2] = 0u;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tc::tmem_alloc(tm_holder, 512);
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (CL > 1) cluster_sync_all();  // the partner's barriers exist before any remote arrive
  const uint32_t tbase = *tm_holder;
  const uint32_t N = d.n_envs;
  const int n_tiles = (int)((N + kRows - 1) / kRows);
  const int n_clus = (int)gridDim.x / CL, cid = (int)blockIdx.x / CL;
  // in sweep blocks of kEB Gaussians (two image blocks each)
  const int n_blk = ((const int32_t *)eimg)[0] / 2 / CL;  // this CTA's blocks per sweep
  const int nb_pos = ((const int32_t *)eimg)[1] / 2;       // blocks before the first a < 0 block
  const int blk0 = (int)rank * n_blk;                      // this CTA's first block
  const uint64_t wlim = d.wait_ns;
  bool fail = false;

  if (tid >= kEpi) {
    // ===================== producer warps =====================
    // Block g of this CTA's sweep sequence lands in shared-memory buffer g % kNS
    // and accumulates in TMEM buffer g % kNT.  The loader (warp 8) refills a
    // shared-memory buffer as soon as the MMA that read it has completed, ahead of
    // the sweeps (blocks do not depend on the env rows); MMA warp w (warp 9 + w)
    // issues the blocks g = w mod 2 once their bytes have landed, their
    // accumulator has been read out, and the sweep's operand rows are ready.
    // The epilogue thus finds up to kNT blocks already multiplied.  A block's
    // phase on one of these barriers is (g / buffers) & 1: no later phase can
    // complete before the waiter acts (block g + kNT reuses g's accumulator only
    // after the epilogue has read g, which follows g's completion, whichever
    // warp issued either).
    volatile uint32_t *endf = cmd + 1, *s_gl = cmd + 2;
    const int lane = tid & 31;
    if (warp == kEpi / 32) {
      if (lane == 0) {
        const uint8_t *src0 = blocks + (size_t)blk0 * kEBBytes;
        uint32_t gl = 0;
        for (;;) {
          if (gl >= (uint32_t)kNS) {  // the MMA of block gl - kNS has read its buffer, or the end
            // Polled with test_wait, which never suspends the thread, so that the
            // copy starts within a few cycles of the MMA's completion (the next
            // blocks' MMAs wait on it); the limit is counted on the SM clock
            // (2 cycles per ns).
            const uint32_t gp = gl - kNS;
            bool got = false;
            const uint64_t c0 = tc::sm_clock();
            for (;;) {
              if (tc::mbar_test_wait(bar_mma + gp % kNT, (gp / kNT) & 1u)) { got = true; break; }
              if (*endf) break;
              if (tc::sm_clock() - c0 > 2 * wlim) { fail = true; break; }
            }
            if (!got) break;
          }
          const uint32_t sbuf = gl % kNS;
          mbar_expect_tx(bar_b + sbuf, kEBBytes);
          bulk_g2s(sb + OFF_BE + sbuf * kEBBytes, src0 + (size_t)(gl % (uint32_t)n_blk) * kEBBytes,
                   kEBBytes, bar_b + sbuf);
          ++gl;
        }
        *s_gl = gl;
      }
      __syncwarp();
      bar_sync_n(kBarProd, 32 * (1 + kMmaWarps));
    } else {
      const uint32_t mw = (uint32_t)(warp - kEpi / 32 - 1);  // this MMA warp
      uint32_t g = 0;  // blocks passed (issued by either warp) in the sweep sequence
      if (lane == 0) {
        constexpr uint32_t idesc = tc::idesc_bf16_f32(128, kEB);
        uint32_t pa = 0;
        while (!fail) {
          if (!tc::mbar_wait(bar_ae, pa, wlim)) { fail = true; break; }
          pa ^= 1u;
          if (*cmd == 0u) break;
          for (int i = 0; i < n_blk && !fail; ++i, ++g) {
            if (g % kMmaWarps != mw) continue;  // the other warp's block
            const uint32_t sbuf = g % kNS, t = g % kNT;
            if (!tc::mbar_wait(bar_b + sbuf, (g / kNS) & 1u, wlim)) { fail = true; break; }
            if (g >= (uint32_t)kNT &&
                !tc::mbar_wait(bar_epi + t, ((g - kNT) / kNT) & 1u, wlim)) { fail = true; break; }
            tc::fence_after_sync();
#pragma unroll
            for (int s = 0; s < kKE / 16; ++s) {
              const uint64_t db = tc::smem_desc(sb + OFF_BE + sbuf * kEBBytes + (uint32_t)s * 256u,
                                                128, kKE * 16, tc::kSwizzleNone);
              mma_ts(tbase + TM_E + t * kEB, tbase + TM_A + (uint32_t)(8 * s), db, idesc, s != 0);
            }
            tc::mma_commit(bar_mma + t);
          }
        }
        cmd[4 + mw] = g;
      }
      __syncwarp();
      bar_sync_n(kBarProd, 32 * (1 + kMmaWarps));
      if (lane == 0) {
        if (mw == 0) {
          // blocks loaded ahead whose MMA was never issued (the sweeps' end, or
          // a wait that ran out): their copies finish before shared memory goes
          // away, on every path.  Block q belongs to warp q mod 2, which issued
          // it if q is below the count that warp passed; a block never issued
          // is the last one loaded into its buffer, so its phase is exact.
          const uint32_t gl = *s_gl;
          uint32_t g_min = cmd[4];
          for (int w = 1; w < kMmaWarps; ++w) g_min = min(g_min, cmd[4 + w]);
          for (uint32_t q = g_min; q < gl; ++q)
            if (q >= cmd[4 + q % kMmaWarps])
              tc::mbar_wait(bar_b + q % kNS, (q / kNS) & 1u, tc::kDrainNs);
        }
        tc::mma_commit(bar_drain);
        tc::mbar_wait(bar_drain, 0, tc::kDrainNs);
      }
    }
    if (fail && (tid & 31) == 0) {
      atomicExch(d.err, 1u);
      atomicExch(d.err + 1, 500u);
    }
  } else {
    // ===================== epilogue: env rows =====================
    // Row r is served by thread r (half 0: the env's record writer, its energy
    // and observed energy) and thread r + 128 (half 1); each half holds and
    // samples D / 2 of the row's coordinates and takes half of every tanh and
    // exp epilogue.
    const int r = tid & 127, h = tid >> 7;
    const bool own = h == 0;
    const int j0 = h * DH;
    const uint32_t lane_sel = (uint32_t)((warp & 3) * 32) << 16;
    const uint32_t pair = kBarPair0 + (uint32_t)(warp & 3);
    float *xch_e = (float *)(sm + OFF_XCH), *xch_lp = xch_e + kRows, *xch_yy = xch_lp + kRows;
    float *recv = (float *)(sm + OFF_RECV);
    const uint64_t seed = d.seed;
    const uint64_t k0 = d.k[0];
    const uint32_t R = d.ring_steps;
    const size_t S = d.n_slots;
    const float sig_n = d.noise_sigma, clip = d.step_clip;
    const float half_log_2pi = 0.91893853320467274f;
    constexpr uint32_t id_pol = tc::idesc_bf16_f32(128, kH);
    constexpr uint32_t id_out = tc::idesc_bf16_f32(128, kN3);
    uint32_t pp = 0, ge = 0, px = 0, par = 0;
    // After a wait has run out no other wait is attempted: the CTA runs on to the
    // vote at the next step boundary and leaves together.
    auto wait = [&](uint64_t *bar, uint32_t parity) {
      if (!fail && !tc::mbar_wait(bar, parity, wlim)) fail = true;
    };
    const uint32_t partner = rank ^ 1u;
    const uint32_t recv_remote = CL > 1 ? mapa(sb + OFF_RECV, partner) : 0u;
    const uint32_t barx_remote = CL > 1 ? mapa(tc::smem_u32(bar_x), partner) : 0u;
    const uint32_t a1_row = sb + OFF_AE + (uint32_t)(r >> 3) * (kK1 * 16) + (uint32_t)(r & 7) * 16u;
    const uint32_t ae_tm = tbase + lane_sel + TM_A;  // this row's energy operand (TMEM lane r)
    // byte offset of element k within a row of a K-major operand without swizzle
    auto kofs = [](int k) -> uint32_t { return (uint32_t)((k >> 3) * 128 + (k & 7) * 2); };

    // One energy sweep over this CTA's Gaussians at the rows of the energy
    // operand; returns the whole-landscape energy (the same bits on both halves
    // and on both CTAs of a pair).
    auto sweep = [&]() -> float {
      if (tid == 0) *cmd = 1u;
      tmem_wait_st();  // the operand rows are in tensor memory before the MMAs read them
      tc::fence_before_sync();
      mbar_arrive(bar_ae);
      // Half h evaluates the blocks of parity h, all kEB columns of each, so that
      // the two warps of an SMSP work on different blocks (one's TMEM load and
      // waits overlap the other's exponentials).  A block holds Gaussians of one
      // sign; the two signs are summed apart.  The loads are pipelined over the
      // block's four 32-column chunks: each chunk loads while the one before it
      // is exponentiated (two 32-register buffers), the next block's first
      // chunk while the last is.
      float ap = 0.f, an = 0.f;
      uint32_t za[32], zb[32];
      const uint32_t tm_e = tbase + lane_sel + TM_E;
      if (h < n_blk) {
        const uint32_t gb = ge + (uint32_t)h, t = gb % kNT;
        wait(bar_mma + t, (gb / kNT) & 1u);
        tc::fence_after_sync();
        tc::tmem_ld32(tm_e + t * kEB, za);
        tmem_wait_ld_regs(za);
      }
      for (int i = h; i < n_blk; i += 2) {
        const uint32_t gb = ge + (uint32_t)i, t = gb % kNT;
        const uint32_t col = tm_e + t * kEB;
        float sv[4] = {0.f, 0.f, 0.f, 0.f};
        tc::tmem_ld32(col + 32u, zb);
        ex2_sum32(za, sv);
        tmem_wait_ld_regs(zb);
        tc::tmem_ld32(col + 64u, za);
        ex2_sum32(zb, sv);
        tmem_wait_ld_regs(za);
        tc::tmem_ld32(col + 96u, zb);
        ex2_sum32(za, sv);
        tmem_wait_ld_regs(zb);
        tc::fence_before_sync();
        mbar_arrive(bar_epi + t);  // the accumulator is read out
        const int in = i + 2;
        if (in < n_blk) {
          const uint32_t gn = ge + (uint32_t)in, tn = gn % kNT;
          wait(bar_mma + tn, (gn / kNT) & 1u);
          tc::fence_after_sync();
          tc::tmem_ld32(tm_e + tn * kEB, za);
        }
        ex2_sum32(zb, sv);
        if (in < n_blk) tmem_wait_ld_regs(za);
        const float bs = (sv[0] + sv[1]) + (sv[2] + sv[3]);
        if (blk0 + i < nb_pos) ap += bs;
        else an += bs;
      }
      ge += (uint32_t)n_blk;
      const float part = ap - an;
      if (!own) xch_e[r] = part;
      bar_sync_n(pair, 64);
      float E = 0.f;
      if (own) {
        E = part + xch_e[r];
        if (CL > 1) {
          st_cluster_f32(recv_remote + (par * kRows + (uint32_t)r) * 4u, E);
          arrive_remote(barx_remote);
          if (!fail && !mbar_wait_cluster(bar_x, px, wlim)) fail = true;
          const float other = recv[par * kRows + r];
          E = rank == 0 ? E + other : other + E;
        }
        xch_e[r] = E;
      }
      px ^= 1u;
      par ^= 1u;
      bar_sync_n(pair, 64);
      if (!own) E = xch_e[r];  // half 1 writes xch_e next only after this read
      return E;
    };
    // The energy operand row [v_hi | v_hi | v_lo | 1, 1 | vv_hi, vv_hi, vv_lo | 0]
    // (K = 80) in tensor memory, the A operand of the sweep's MMAs: element k in
    // column k / 2 of the row's lane (the lower k in the low half).  Each half
    // writes its coordinates' columns of the three copies; after the two halves'
    // sums of squares meet, half 1 writes the constant and |v|^2 columns and the
    // zero tail.  lp (half 1's log-probability part) rides along to half 0.
    auto write_ae = [&](const float (&v)[DH], float lp_part) {
      float yy = 0.f;
      uint32_t hw[DH / 2], lw[DH / 2];
#pragma unroll
      for (int q = 0; q < DH / 2; ++q) {
        const float a0 = v[2 * q], a1 = v[2 * q + 1];
        yy = fmaf(a0, a0, yy);
        yy = fmaf(a1, a1, yy);
        hw[q] = tc::pack_bf16x2(a0, a1);
        lw[q] = tc::pack_bf16x2(a0 - tc::bf16_lo(hw[q]), a1 - tc::bf16_hi(hw[q]));
      }
      tmem_st_cols<DH / 2>(ae_tm + (uint32_t)(j0 / 2), hw);
      tmem_st_cols<DH / 2>(ae_tm + (uint32_t)((D + j0) / 2), hw);
      tmem_st_cols<DH / 2>(ae_tm + (uint32_t)((2 * D + j0) / 2), lw);
      if (!own) xch_lp[r] = lp_part;
      xch_yy[h * kRows + r] = yy;
      bar_sync_n(pair, 64);
      if (!own) {
        const float vv = xch_yy[r] + xch_yy[kRows + r];
        const uint32_t hv = tc::pack_bf16x2(vv, 0.f) & 0xFFFFu;
        const uint32_t lv = tc::pack_bf16x2(vv - __uint_as_float(hv << 16), 0.f) & 0xFFFFu;
        constexpr int NT = kKE / 2 - 3 * D / 2;  // [1, 1 | vv_hi, vv_hi | vv_lo, 0 | 0 ...]
        uint32_t tw[NT];
#pragma unroll
        for (int c = 0; c < NT; ++c) tw[c] = 0u;
        tw[0] = tc::pack_bf16x2(1.f, 1.f);
        tw[1] = hv | (hv << 16);
        tw[2] = lv;
        tmem_st_cols<NT>(ae_tm + (uint32_t)(3 * D / 2), tw);
      }
    };

    for (int tile = cid; tile < n_tiles && !fail; tile += n_clus) {
      const uint32_t e = (uint32_t)tile * kRows + (uint32_t)r;
      const bool valid = e < N;
      float x[DH];
      float eobs = 0.f;
      int t = 0;
#pragma unroll
      for (int i = 0; i < DH; ++i) x[i] = valid ? d.s[(size_t)(j0 + i) * N + e] : 0.f;
      if (valid) {
        t = d.t[e];
        if (own) eobs = d.eobs[e];
      }
      const bool rec = valid && rank == 0;  // this thread writes its part of the records
      for (uint32_t s = 0; s < n_steps; ++s) {
        const uint32_t k = (uint32_t)(k0 + s);
        const size_t rowR = (size_t)((k0 + s) % R);
        // ---- observation record and the layer-1 operand row [x, 1, 1, 0...]
        if (rec)
#pragma unroll
          for (int i = 0; i < DH; ++i) d.r_obs[(rowR * D + (size_t)(j0 + i)) * S + e] = x[i];
#pragma unroll
        for (int q = 0; q < DH / 4; ++q) {
          const uint32_t a = tc::pack_bf16x2(x[4 * q], x[4 * q + 1]);
          const uint32_t b = tc::pack_bf16x2(x[4 * q + 2], x[4 * q + 3]);
          asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(a1_row + kofs(j0 + 4 * q)), "r"(a), "r"(b) : "memory");
        }
        if (!own) {
#pragma unroll
          for (int c = D / 8; c < kK1 / 8; ++c)
            tc::sts128(a1_row + (uint32_t)c * 128u, c == D / 8 ? tc::pack_bf16x2(1.f, 1.f) : 0u, 0u, 0u, 0u);
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        if (!bar_all_n(kBarEpi, kEpi, !fail)) { fail = true; break; }
        // ---- layer 1
        if (tid == 0) {
          tc::fence_after_sync();
#pragma unroll
          for (int q = 0; q < kK1 / 16; ++q) {
            const uint64_t da = tc::smem_desc(sb + OFF_AE + (uint32_t)q * 256u, 128, kK1 * 16, tc::kSwizzleNone);
            const uint64_t db = tc::smem_desc(sb + PK_W1 + (uint32_t)q * 256u, 128, kK1 * 16, tc::kSwizzleNone);
            tc::mma_bf16(tbase, da, db, id_pol, q != 0);
          }
          tc::mma_commit(bar_pol);
        }
        // The step's Philox normals (this half's action coordinates, and the
        // observation noise of the candidate) do not depend on the policy: they
        // are drawn while the layer-2 MMA runs.
        float zn[DH];
        float zo = 0.f;
#pragma unroll 1
        for (int l = 0; l < 3; ++l) {
          if (l == 1) {
#pragma unroll
            for (int q = 0; q < DH / 4; ++q) {
              const uint4 rw = draw(seed, k, d.env_base + e, 0, kTagAction, (uint32_t)((j0 + 4 * q) >> 2));
              const float2 p = box_muller(rw.x, rw.y), p2 = box_muller(rw.z, rw.w);
              zn[4 * q] = p.x;
              zn[4 * q + 1] = p.y;
              zn[4 * q + 2] = p2.x;
              zn[4 * q + 3] = p2.y;
            }
            if (own) {
              const uint4 rn = draw(seed, k, d.env_base + e, 0, kTagNoise, 0);
              zo = box_muller(rn.x, rn.y).x;
            }
          }
          wait(bar_pol, pp);
          pp ^= 1u;
          tc::fence_after_sync();
          if (l == 2) break;
          // ---- tanh epilogue of layer l + 1: columns [128 h, 128 h + 128) -> packed h
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            uint32_t hp[32];
#pragma unroll
            for (int hf = 0; hf < 2; ++hf) {
              const uint32_t c0 = (uint32_t)(128 * h + 64 * q + 32 * hf);
              uint32_t z[32];
              tc::tmem_ld32(tbase + lane_sel + c0, z);
              tc::tmem_wait_ld();
#pragma unroll
              for (int i = 0; i < 16; ++i) {
                float z0 = __uint_as_float(z[2 * i]), z1 = __uint_as_float(z[2 * i + 1]);
                if (l == 1) {
                  const float2 bb = *(const float2 *)(sm + PK_B2 + (c0 + 2 * i) * 4);
                  z0 += bb.x;
                  z1 += bb.y;
                }
                hp[hf * 16 + i] = tc::pack_bf16x2(tc::tanh_fast(z0), tc::tanh_fast(z1));
              }
            }
            tmem_st32(tbase + lane_sel + TM_H + (uint32_t)(64 * h + 32 * q), hp);
          }
          tmem_wait_st();
          tc::fence_before_sync();
          bar_sync_n(kBarEpi, kEpi);
          if (tid == 0) {
            tc::fence_after_sync();
            // layer 2 (l = 0): N = 256 into columns [0, 256); layer 3 (l = 1): N = 48
#pragma unroll
            for (int q = 0; q < kH / 16; ++q) {
              const int kb = q >> 2, kk = q & 3;
              const uint32_t boff = l == 0 ? (uint32_t)(PK_W2 + kb * kH * 128 + kk * 32)
                                           : (uint32_t)(PK_W3 + kb * kN3 * 128 + kk * 32);
              const uint64_t db = tc::smem_desc(sb + boff, 16, 1024, tc::kSwizzle128B);
              mma_ts(tbase, tbase + TM_H + (uint32_t)(8 * q), db, l == 0 ? id_pol : id_out, q != 0);
            }
            tc::mma_commit(bar_pol);
          }
        }
        // ---- sample this half's coordinates of the Gaussian head, y = x + dx
        float y[DH];
        float lp = 0.f;
        {
          float out[2 * D];
#pragma unroll
          for (int q = 0; q < kN3 / 16; ++q) {
            uint32_t z[16];
            tmem_ld16(tbase + lane_sel + (uint32_t)(16 * q), z);
            tc::tmem_wait_ld();
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const int c = 16 * q + i;
              if (c < 2 * D) out[c] = __uint_as_float(z[i]) + *(const float *)(sm + PK_B3 + c * 4);
            }
          }
          if (rec && own && d.dbg_logits) {
#pragma unroll
            for (int c = 0; c < 2 * D; ++c) d.out[(size_t)e * 2 * D + c] = out[c];
#pragma unroll
            for (int c = 0; c < 2 * D; ++c) d.r_pout[(rowR * 2 * D + c) * S + e] = out[c];
          }
          float mu[DH], lsr[DH];
#pragma unroll
          for (int i = 0; i < DH; ++i) {
            mu[i] = own ? out[i] : out[DH + i];
            lsr[i] = own ? out[D + i] : out[D + DH + i];
          }
          float *act = (float *)d.r_act + rowR * (size_t)D * S + e;
#pragma unroll
          for (int q = 0; q < DH / 4; ++q) {
            const int j = j0 + 4 * q;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const int u = 4 * q + i;
              const float zz = zn[u];
              const float ls = fminf(fmaxf(lsr[u], -5.0f), 2.0f);
              const float smp = mu[u] + expf(ls) * zz;
              const float dx = fminf(fmaxf(smp, -clip), clip);
              if (rec) act[(size_t)(j + i) * S] = dx;
              lp += -0.5f * zz * zz - ls - half_log_2pi;
              y[u] = x[u] + dx;
            }
          }
        }
#pragma unroll
        for (int i = 0; i < DH; ++i) x[i] = y[i];  // the candidate; the old state is recorded
        // pass 0: energy of the candidate, the step; pass 1 (only when the tile has
        // a reset; the same vote on every CTA of the cluster, whose states are
        // identical): energy of the fresh states
        const int t2 = t + 1;
        bool done = false;
#pragma unroll 1
        for (int pass = 0; pass < 2; ++pass) {
          write_ae(x, lp);
          if (pass == 0 && own && rec) d.r_logp[rowR * S + e] = lp + xch_lp[r];
          const float E = sweep();
          // the step limit, or the product basin reached (both halves and both
          // CTAs of a pair hold the same E, so they take the same decision)
          if (pass == 0) done = valid && (t2 >= (int)d.episode_limit || E < d.energy_target);
          if (pass == 1) {
            if (own && done) {
              const uint4 rn = draw(seed, k, d.env_base + e, 0, kTagNoise, 1);
              eobs = E + sig_n * box_muller(rn.x, rn.y).x;
            }
            break;
          }
          // ---- step: observed energy, reward, done, auto-reset
          if (own) {
            const float eobs2 = E + sig_n * zo;
            if (rec) {
              const size_t o = rowR * S + e;
              d.r_energy[o] = E;
              d.r_rew[o] = eobs - eobs2;
              d.r_done[o] = (uint8_t)done;
            }
            if (!done) eobs = eobs2;
          }
          if (done) {
#pragma unroll
            for (int q = 0; q < DH / 4; ++q) {
              const uint4 rr = draw(seed, k, d.env_base + e, 0, kTagReset, (uint32_t)((j0 + 4 * q) >> 2));
              x[4 * q] = uniform(rr.x, -3.0f, 3.0f);
              x[4 * q + 1] = uniform(rr.y, -3.0f, 3.0f);
              x[4 * q + 2] = uniform(rr.z, -3.0f, 3.0f);
              x[4 * q + 3] = uniform(rr.w, -3.0f, 3.0f);
            }
            t = 0;
          } else {
            t = t2;
          }
          lp = 0.f;
          if (!bar_any_n(kBarEpi, kEpi, done)) break;
        }
      }
      if (rec && !fail) {
#pragma unroll
        for (int i = 0; i < DH; ++i) d.s[(size_t)(j0 + i) * N + e] = x[i];
        if (own) {
          d.eobs[e] = eobs;
          d.t[e] = t;
          d.needs_energy[e] = 0;
        }
      }
    }
    // stop the producer warps (a wait of the last step that ran out on any
    // epilogue thread counts: the vote makes every thread see it)
    fail = !bar_all_n(kBarEpi, kEpi, !fail);
    if (tid == 0) {
      *cmd = 0u;
      cmd[1] = 1u;  // the loader stops waiting
    }
    mbar_arrive(bar_ae);
    if (fail && tid == 0) {
      // a policy MMA may still be in flight after a wait that ran out: the
      // commit on a barrier not used before completes once all of them have
      tc::mma_commit(bar_drain_pol);
      tc::mbar_wait(bar_drain_pol, 0, tc::kDrainNs);
      atomicExch(d.err, 1u);
      atomicExch(d.err + 1, 501u);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (CL > 1) cluster_sync_all();  // no remote access to this CTA's memory after this point
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tbase, 512);
  }
}

// =====================================================================
// Force of recorded transitions on the tensor cores (ws_forces, BF16 path).
// F(y) = -grad E(y) = sum_m s_m P_m (y - c_m) / w_m^2 with P_m = |a_m| e_m and
// s_m the sign of a_m:
//   F_j = y_j * sum_m P_m f_m  -  sum_m P_m f_m c_mj,   f_m = s_m / w_m^2.
// Per 128-row tile of (step, env) rows: each 64-Gaussian block's whole
// exponents log2 P_m come from the energy image exactly as in the roll-out
// sweep (one MMA, K = 80, into one of four TMEM accumulators); the epilogue
// turns them into P = 2^z (one ex2 per pair) and writes P as BF16 hi + lo into
// a shared-memory A operand [128 rows][64 Gaussians]; a second MMA multiplies
// it with the block's force image [32 columns][64 Gaussians] = (f c_m, f, 0...)
// (hi + lo; three products hi.hi + lo.hi + hi.lo) into one FP32 accumulator of
// 32 columns per row.  The sign and 1 / w^2 ride in the force image, so the
// epilogue is the exponential and the split alone.
constexpr int kFN = 32;                          // force columns: D coordinates, the sum, zeros
constexpr int kFImgBytes = kFN * kBlk * 2;       // one plane of a block's force image
constexpr int kFBlkBytes = 2 * kFImgBytes;       // hi plane | lo plane
constexpr int kFS = 4;                           // shared-memory stages (energy + force block)
constexpr int kFStage = kBlkBytes + kFBlkBytes;
constexpr int kFZ = 4;                           // TMEM exponent accumulators
constexpr int kFP = 3;                           // P operand buffers
constexpr int kPPlane = kRows * kBlk * 2;        // one plane of P [128][64]
constexpr uint32_t TM_F = kFZ * kBlk;            // TMEM columns of the force accumulator
constexpr int FOFF_AE = 0;
constexpr int FOFF_ST = FOFF_AE + kRows * kKE * 2;
constexpr int FOFF_P = FOFF_ST + kFS * kFStage;
constexpr int FOFF_BAR = FOFF_P + kFP * 2 * kPPlane;
constexpr int F_NBAR = 1 + 2 * kFS + 2 * kFZ + 2 * kFP + 2;  // ae, b, sf, z, zf, p, pf, f, drain
constexpr int FOFF_CMD = FOFF_BAR + F_NBAR * 8;
constexpr int FOFF_TM = FOFF_CMD + 16;
constexpr int FSMEM = FOFF_TM + 16 + 1024;
static_assert(FSMEM <= 232448, "force kernel shared memory");
static_assert(FOFF_ST % 16 == 0 && FOFF_P % 16 == 0 && FOFF_BAR % 8 == 0, "alignment");
static_assert(TM_F + kFN <= 512, "force accumulator");

inline size_t force_img_bytes(int M) { return (size_t)(land_slots(M) / kBlk) * kFBlkBytes; }

// Block b's force image: planes hi and lo of [32 n][64 k] (K-major, no swizzle),
// n < D: f_m c_mn, n = D: f_m, else 0; padding slots all 0.
__global__ void k_force_tc_pack(const float *__restrict__ c, const float *__restrict__ w,
                                const float *__restrict__ a, int D, int slots,
                                const int32_t *__restrict__ order, uint8_t *__restrict__ img) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  for (int i = tid; i < slots * kFN; i += stride) {
    const int sl = i / kFN, n = i % kFN, m = order[sl];
    float v = 0.f;
    if (m >= 0 && n <= D) {
      const float f = (a[m] >= 0.f ? 1.0f : -1.0f) / (w[m] * w[m]);
      v = n < D ? f * c[(size_t)m * D + n] : f;
    }
    uint8_t *blk = img + (size_t)(sl / kBlk) * kFBlkBytes;
    const int off = ns_off(n, sl % kBlk, kBlk);
    *(uint16_t *)(blk + off) = bf16_bits(v);
    *(uint16_t *)(blk + kFImgBytes + off) = bf16_bits(v - bf16_val(v));
  }
}

template <int D>
__global__ void __launch_bounds__(kThreads, 1)
    k_force_tc(Dev d, const uint8_t *__restrict__ eimg, const uint8_t *__restrict__ eblocks,
               const uint8_t *__restrict__ fblocks, uint32_t n) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = tc::smem_u32(smem_raw);
  uint8_t *sm = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
  const uint32_t sb = tc::smem_u32(sm);
  const int tid = threadIdx.x, warp = tid >> 5;
  uint64_t *bars = (uint64_t *)(sm + FOFF_BAR);
  uint64_t *bar_ae = bars, *bar_b = bar_ae + 1, *bar_sf = bar_b + kFS, *bar_z = bar_sf + kFS;
  uint64_t *bar_zf = bar_z + kFZ, *bar_p = bar_zf + kFZ, *bar_pf = bar_p + kFP;
  uint64_t *bar_f = bar_pf + kFP, *bar_drain = bar_f + 1;
  volatile uint32_t *cmd = (volatile uint32_t *)(sm + FOFF_CMD);
  uint32_t *tm_holder = (uint32_t *)(sm + FOFF_TM);
  if (tid == 0) {
    tc::mbar_init(bar_ae, kRows);  // half 0 writes the operand rows
    for (int i = 0; i < kFS; ++i) {
      tc::mbar_init(bar_b + i, 1);
      tc::mbar_init(bar_sf + i, 1);
    }
    for (int i = 0; i < kFZ; ++i) {
      tc::mbar_init(bar_z + i, 1);
      tc::mbar_init(bar_zf + i, kEpi);
    }
    for (int i = 0; i < kFP; ++i) {
      tc::mbar_init(bar_p + i, kEpi);
      tc::mbar_init(bar_pf + i, 1);
    }
    tc::mbar_init(bar_f, 1);
    tc::mbar_init(bar_drain, 1);
    cmd[0] = 0u;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tc::tmem_alloc(tm_holder, 512);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tm_holder;
  const size_t N = d.n_envs, S = d.n_slots, rows = (size_t)n * N;
  const int n_tiles = (int)((rows + kRows - 1) / kRows);
  const int nb = ((const int32_t *)eimg)[0];  // blocks per tile (all Gaussians)
  int my_tiles = 0;
  for (int t = (int)blockIdx.x; t < n_tiles; t += (int)gridDim.x) ++my_tiles;
  const uint32_t total = (uint32_t)my_tiles * (uint32_t)nb;
  bool fail = false;

  if (tid >= kEpi) {
    // ===================== producer warps =====================
    // Block g (counted over this CTA's tiles) sits in stage g % kFS, its
    // exponents in TMEM accumulator g % kFZ, its P in buffer g % kFP.  The MMA
    // warp issues the exponent MMA of block g, then the force MMA of block g - 1,
    // so the tensor core works on g while the epilogue exponentiates g - 1.
    const int lane = tid & 31;
    if (warp == kEpi / 32) {
      if (lane == 0) {
        uint32_t gl = 0;
        for (; gl < total && !fail; ++gl) {
          const uint32_t st = gl % kFS;
          if (gl >= (uint32_t)kFS &&
              !tc::mbar_wait(bar_sf + st, ((gl - kFS) / kFS) & 1u, kWaitNs)) { fail = true; break; }
          const uint32_t b = gl % (uint32_t)nb;
          mbar_expect_tx(bar_b + st, kFStage);
          bulk_g2s(sb + FOFF_ST + st * kFStage, eblocks + (size_t)b * kBlkBytes, kBlkBytes, bar_b + st);
          bulk_g2s(sb + FOFF_ST + st * kFStage + kBlkBytes, fblocks + (size_t)b * kFBlkBytes,
                   kFBlkBytes, bar_b + st);
        }
        cmd[0] = gl;
      }
      __syncwarp();
      bar_sync_n(kBarProd, 64);
    } else {
      uint32_t g = 0;
      if (lane == 0) {
        constexpr uint32_t id_e = tc::idesc_bf16_f32(128, kBlk), id_f = tc::idesc_bf16_f32(128, kFN);
        // force MMA of block q: three products of P (hi, lo) and the image (hi, lo)
        auto force_mma = [&](uint32_t q, bool first) -> bool {
          const uint32_t pb = q % kFP, st = q % kFS;
          if (!tc::mbar_wait(bar_p + pb, (q / kFP) & 1u, kWaitNs)) return false;
          tc::fence_after_sync();
          const uint32_t pa = sb + FOFF_P + pb * 2u * kPPlane;
          const uint32_t fb = sb + FOFF_ST + st * kFStage + kBlkBytes;
#pragma unroll
          for (int prod = 0; prod < 3; ++prod) {
            const uint32_t a0 = pa + (prod == 1 ? (uint32_t)kPPlane : 0u);
            const uint32_t b0 = fb + (prod == 2 ? (uint32_t)kFImgBytes : 0u);
#pragma unroll
            for (int s = 0; s < kBlk / 16; ++s) {
              const uint64_t da = tc::smem_desc(a0 + (uint32_t)s * 256u, 128, kBlk * 16, tc::kSwizzleNone);
              const uint64_t db = tc::smem_desc(b0 + (uint32_t)s * 256u, 128, kBlk * 16, tc::kSwizzleNone);
              tc::mma_bf16(tbase + TM_F, da, db, id_f, !(first && prod == 0 && s == 0));
            }
          }
          tc::mma_commit(bar_pf + pb);
          tc::mma_commit(bar_sf + st);
          return true;
        };
        uint32_t pa = 0;
        for (int t = 0; t < my_tiles && !fail; ++t) {
          if (!tc::mbar_wait(bar_ae, pa, kWaitNs)) { fail = true; break; }
          pa ^= 1u;
          for (int i = 0; i < nb; ++i, ++g) {
            const uint32_t st = g % kFS, z = g % kFZ;
            if (!tc::mbar_wait(bar_b + st, (g / kFS) & 1u, kWaitNs)) { fail = true; break; }
            if (g >= (uint32_t)kFZ &&
                !tc::mbar_wait(bar_zf + z, ((g - kFZ) / kFZ) & 1u, kWaitNs)) { fail = true; break; }
            tc::fence_after_sync();
#pragma unroll
            for (int s = 0; s < kKE / 16; ++s) {
              const uint64_t da = tc::smem_desc(sb + FOFF_AE + (uint32_t)s * 256u, 128, kKE * 16,
                                                tc::kSwizzleNone);
              const uint64_t db = tc::smem_desc(sb + FOFF_ST + st * kFStage + (uint32_t)s * 256u, 128,
                                                kKE * 16, tc::kSwizzleNone);
              tc::mma_bf16(tbase + z * kBlk, da, db, id_e, s != 0);
            }
            tc::mma_commit(bar_z + z);
            if (i > 0 && !force_mma(g - 1, i == 1)) { fail = true; break; }
          }
          if (fail) break;
          if (!force_mma(g - 1, nb == 1)) { fail = true; break; }
          tc::mma_commit(bar_f);
        }
      }
      __syncwarp();
      bar_sync_n(kBarProd, 64);
      if (lane == 0) {
        // copies issued ahead of a wait that ran out land before shared memory goes away
        if (fail) {
          const uint32_t gl = cmd[0];
          for (uint32_t q = g; q < gl; ++q) tc::mbar_wait(bar_b + q % kFS, (q / kFS) & 1u, kWaitNs);
        }
        tc::mma_commit(bar_drain);
        tc::mbar_wait(bar_drain, 0, kWaitNs);
      }
    }
    if (fail && (tid & 31) == 0) {
      atomicExch(d.err, 1u);
      atomicExch(d.err + 1, 510u);
    }
  } else {
    // ===================== epilogue =====================
    // Row r of a tile: thread r (half 0) holds y, writes the operand row and the
    // force; threads r and r + 128 exponentiate columns [32 h, 32 h + 32) of
    // every block.
    const int r = tid & 127, h = tid >> 7;
    const uint32_t lane_sel = (uint32_t)((warp & 3) * 32) << 16;
    const uint32_t ae_row = sb + FOFF_AE + (uint32_t)(r >> 3) * (kKE * 16) + (uint32_t)(r & 7) * 16u;
    auto kofs = [](int k) -> uint32_t { return (uint32_t)((k >> 3) * 128 + (k & 7) * 2); };
    const uint64_t k_end = d.k[0];
    uint32_t g = 0, pf = 0;
    for (int tile = (int)blockIdx.x; tile < n_tiles && !fail; tile += (int)gridDim.x) {
      const size_t q = (size_t)tile * kRows + (size_t)r;
      const bool valid = q < rows;
      const uint32_t i = valid ? (uint32_t)(q / N) : 0u, e = valid ? (uint32_t)(q % N) : 0u;
      const size_t rowR = (size_t)((k_end - n + i) % d.ring_steps);
      float y[D];
      if (h == 0) {
        const float *obs = d.r_obs + rowR * D * S + e;
        const float *act = (const float *)d.r_act + rowR * D * S + e;
        float yy = 0.f;
#pragma unroll
        for (int j = 0; j < D; ++j) {
          y[j] = valid ? obs[(size_t)j * S] + act[(size_t)j * S] : 0.f;
          yy = fmaf(y[j], y[j], yy);
        }
        // [y_hi | y_hi | y_lo | 1, 1 | yy_hi, yy_hi, yy_lo | 0...]
#pragma unroll
        for (int q4 = 0; q4 < D / 4; ++q4) {
          const float a0 = y[4 * q4], a1 = y[4 * q4 + 1], a2 = y[4 * q4 + 2], a3 = y[4 * q4 + 3];
          const uint32_t h01 = tc::pack_bf16x2(a0, a1), h23 = tc::pack_bf16x2(a2, a3);
          const uint32_t l01 = tc::pack_bf16x2(a0 - tc::bf16_lo(h01), a1 - tc::bf16_hi(h01));
          const uint32_t l23 = tc::pack_bf16x2(a2 - tc::bf16_lo(h23), a3 - tc::bf16_hi(h23));
          const int j = 4 * q4;
          asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(ae_row + kofs(j)), "r"(h01), "r"(h23) : "memory");
          asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(ae_row + kofs(D + j)), "r"(h01), "r"(h23) : "memory");
          asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(ae_row + kofs(2 * D + j)), "r"(l01), "r"(l23) : "memory");
        }
        const uint32_t hv = tc::pack_bf16x2(yy, 0.f) & 0xFFFFu;
        const uint32_t lv = tc::pack_bf16x2(yy - __uint_as_float(hv << 16), 0.f) & 0xFFFFu;
#pragma unroll
        for (int c = 3 * D / 8; c < kKE / 8; ++c) {
          if (c == 3 * D / 8)
            tc::sts128(ae_row + (uint32_t)c * 128u, tc::pack_bf16x2(1.f, 1.f), hv | (hv << 16), lv, 0u);
          else
            tc::sts128(ae_row + (uint32_t)c * 128u, 0u, 0u, 0u, 0u);
        }
        tc::fence_async_smem();
        mbar_arrive(bar_ae);
      }
      // ---- the blocks: P = 2^z as BF16 hi + lo into the A operand of the force MMA
      const uint32_t p_row = (uint32_t)(r >> 3) * (kBlk * 16) + (uint32_t)(r & 7) * 16u;
      for (int b = 0; b < nb; ++b, ++g) {
        const uint32_t z = g % kFZ, pb = g % kFP;
        if (!tc::mbar_wait(bar_z + z, (g / kFZ) & 1u, kWaitNs)) { fail = true; break; }
        tc::fence_after_sync();
        uint32_t v[32];
        tc::tmem_ld32(tbase + lane_sel + z * kBlk + (uint32_t)(32 * h), v);
        tc::tmem_wait_ld();
        tc::fence_before_sync();
        mbar_arrive(bar_zf + z);
        if (g >= (uint32_t)kFP &&
            !tc::mbar_wait(bar_pf + pb, ((g - kFP) / kFP) & 1u, kWaitNs)) { fail = true; break; }
        const uint32_t pbase = sb + FOFF_P + pb * 2u * kPPlane + p_row;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          uint32_t hi[4], lo[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float p0 = ex2_fast(__uint_as_float(v[8 * c + 2 * u]));
            const float p1 = ex2_fast(__uint_as_float(v[8 * c + 2 * u + 1]));
            hi[u] = tc::pack_bf16x2(p0, p1);
            lo[u] = tc::pack_bf16x2(p0 - tc::bf16_lo(hi[u]), p1 - tc::bf16_hi(hi[u]));
          }
          const uint32_t off = (uint32_t)((4 * h + c) * 128);
          tc::sts128(pbase + off, hi[0], hi[1], hi[2], hi[3]);
          tc::sts128(pbase + kPPlane + off, lo[0], lo[1], lo[2], lo[3]);
        }
        tc::fence_async_smem();
        mbar_arrive(bar_p + pb);
      }
      if (fail) break;
      // ---- the tile's force: F_j = y_j * acc[D] - acc[j]
      if (h == 0) {
        if (!tc::mbar_wait(bar_f, pf, kWaitNs)) { fail = true; break; }
        tc::fence_after_sync();
        uint32_t acc[32];
        tc::tmem_ld32(tbase + lane_sel + TM_F, acc);
        tc::tmem_wait_ld();
        tc::fence_before_sync();
        if (valid) {
          const float sp = __uint_as_float(acc[D]);
          float *out = d.r_force + rowR * D * S + e;
#pragma unroll
          for (int j = 0; j < D; ++j) out[(size_t)j * S] = fmaf(y[j], sp, -__uint_as_float(acc[j]));
        }
      }
      pf ^= 1u;
    }
    if (fail && tid == 0) {
      atomicExch(d.err, 1u);
      atomicExch(d.err + 1, 511u);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tbase, 512);
  }
}

template <int D>
cudaError_t launch_force_d(const Dev &d, const uint8_t *eimg, const uint8_t *fimg, uint32_t n,
                           cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_force_tc<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, FSMEM);
    attr = true;
  }
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t rows = (size_t)n * d.n_envs;
  const int n_tiles = (int)((rows + kRows - 1) / kRows);
  const int grid = n_tiles < sms ? n_tiles : sms;
  k_force_tc<D><<<grid, kThreads, FSMEM, st>>>(d, eimg, eimg + land_blocks_off((int)d.n_gauss), fimg, n);
  return cudaGetLastError();
}

}  // namespace

bool land_tc_supported(int D, int M, const PolicyShape &p) {
  return D >= 8 && D <= kMaxD && D % 8 == 0 && M >= 1 && p.w[0] == D && p.w[1] == kH &&
         p.w[2] == kH && p.w[3] == 2 * D;
}
size_t land_tc_policy_bytes() { return (size_t)POLICY; }
size_t land_tc_energy_bytes(int M) {
  return land_blocks_off(M) + (size_t)(land_slots(M) / kBlk) * kBlkBytes;
}
size_t force_tc_bytes(int M) { return force_img_bytes(M); }

// Needs the energy image packed first (its slot order).
void launch_force_tc_pack(const Dev &d, const void *energy_img, void *force_img, cudaStream_t st) {
  const int M = (int)d.n_gauss, slots = land_slots(M);
  const int32_t *order = (const int32_t *)((const uint8_t *)energy_img + land_order_off());
  k_force_tc_pack<<<128, 256, 0, st>>>(d.centres, d.widths, d.amps, (int)d.dim, slots, order,
                                       (uint8_t *)force_img);
}

cudaError_t launch_force_tc(const Dev &d, const void *energy_img, const void *force_img,
                            uint32_t n_steps, cudaStream_t st) {
  const uint8_t *e = (const uint8_t *)energy_img, *f = (const uint8_t *)force_img;
  if (n_steps == 0) return cudaSuccess;
  if (d.dim == 8) return launch_force_d<8>(d, e, f, n_steps, st);
  if (d.dim == 16) return launch_force_d<16>(d, e, f, n_steps, st);
  if (d.dim == 24) return launch_force_d<24>(d, e, f, n_steps, st);
  return cudaErrorInvalidValue;
}

void launch_land_tc_pack(const Dev &d, void *policy_img, void *energy_img, cudaStream_t st) {
  const int M = (int)d.n_gauss, slots = land_slots(M);
  uint8_t *img = (uint8_t *)energy_img;
  int32_t *order = (int32_t *)(img + land_order_off());
  k_land_tc_pack_policy<<<64, 256, 0, st>>>(d.params, (int)d.dim, (uint8_t *)policy_img);
  k_land_tc_order<<<1, 1024, 0, st>>>(d.amps, M, slots, (int32_t *)img, order);
  k_land_tc_pack_energy<<<128, 256, 0, st>>>(d.centres, d.widths, d.amps, (int)d.dim, slots, order,
                                             img + land_blocks_off(M));
}

template <int D>
void land_attr() {
  cudaFuncSetAttribute(k_land_tc<D, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
  cudaFuncSetAttribute(k_land_tc<D, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
}

void land_tc_init() {
  land_attr<8>();
  land_attr<16>();
  land_attr<24>();
}

template <int D>
cudaError_t launch_land_d(const Dev &d, const uint8_t *pol, const uint8_t *eimg, uint32_t n_steps,
                          int tile_ctas, cudaStream_t st) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int n_tiles = (int)((d.n_envs + kRows - 1) / kRows);
  const uint8_t *blocks = eimg + land_blocks_off((int)d.n_gauss);
  if (tile_ctas == 1) {
    const int grid = n_tiles < sms ? n_tiles : sms;
    k_land_tc<D, 1><<<grid, kRollThreads, SMEM, st>>>(d, pol, eimg, blocks, n_steps);
    return cudaGetLastError();
  }
  if (tile_ctas != 2) return cudaErrorInvalidValue;
  const int clusters = n_tiles < sms / 2 ? n_tiles : sms / 2;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(2 * clusters));
  cfg.blockDim = dim3(kRollThreads);
  cfg.dynamicSmemBytes = SMEM;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_land_tc<D, 2>, d, pol, eimg, blocks, n_steps);
}

// tile_ctas = CTAs per 128-env tile (1, or 2 as a cluster splitting the Gaussians).
cudaError_t launch_land_tc(const Dev &d, const void *policy_img, const void *energy_img,
                           uint32_t n_steps, int tile_ctas, cudaStream_t st) {
  const uint8_t *p = (const uint8_t *)policy_img, *e = (const uint8_t *)energy_img;
  if (d.dim == 8) return launch_land_d<8>(d, p, e, n_steps, tile_ctas, st);
  if (d.dim == 16) return launch_land_d<16>(d, p, e, n_steps, tile_ctas, st);
  if (d.dim == 24) return launch_land_d<24>(d, p, e, n_steps, tile_ctas, st);
  return cudaErrorInvalidValue;
}

}  // namespace ws
