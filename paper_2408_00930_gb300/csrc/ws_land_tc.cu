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
//   energy   E(y) at y = x + dx: the cross-term y.c on tcgen05 as
//            [y_hi, y_hi, y_lo] . [c_hi, c_lo, c_hi] (BF16 hi+lo, FP32 accumulate)
//            in blocks of 64 Gaussians streamed by a producer warp (bulk copies
//            into two buffers, MMAs into two TMEM accumulators), and the epilogue
//            a_m 2^(q_m (|y|^2 + |c_m|^2 - 2 y.c_m)) summed per env
//   step     observed energy with Philox noise, reward Eobs(x) - Eobs(x'), done
//            at the episode limit, reset to U(-3, 3)^D and a second sweep for the
//            fresh state's energy when a tile has a reset
// Threads: warps 0-3 own the env rows (state, sampling, records); warps 4-7
// take the other half of every tanh and exp epilogue; warp 8 is the producer.
// Every wait is bounded; a wait that runs out sets the error flag and the CTA
// leaves its loops at the next step boundary.
#include "ws_kernels.cuh"
#include "ws_tc.cuh"

namespace ws {

namespace {

constexpr int kRows = 128;
constexpr int kH = 256;                       // hidden width of both layers
constexpr int kMaxD = 24;                     // coordinates (a multiple of 8, <= 24)
constexpr int kN3 = 48;                       // layer-3 N (2 D, padded to 48)
constexpr int kK1 = 32;                       // layer-1 K: D coordinates, 1, 1, zeros
constexpr int kKE = 80;                       // energy K: 3 D <= 72, five K16 steps
constexpr int kBlk = 64;                      // Gaussians per energy MMA block
constexpr int kBlkImg = kBlk * kKE * 2;       // block image, K = 80 without swizzle
constexpr int kBlkBytes = kBlkImg + kBlk * 16;  // + {|c|^2, q, a, 0} per Gaussian
constexpr int kEpi = 256, kThreads = kEpi + 32;
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
constexpr int OFF_AE = POLICY;                    // energy A [128][80] (also the layer-1 A [128][32])
constexpr int OFF_BE = OFF_AE + kRows * kKE * 2;  // two energy B blocks
constexpr int OFF_XCH = OFF_BE + 2 * kBlkBytes;   // f32 [128] partial energies, [128] |y|^2
constexpr int OFF_RECV = OFF_XCH + 2 * kRows * 4; // f32 [2][128] the cluster partner's partials
constexpr int OFF_BAR = OFF_RECV + 2 * kRows * 4;
constexpr int N_BAR = 10;  // ae, b[2], mma[2], epi[2], pol, x, drain
constexpr int OFF_CMD = OFF_BAR + N_BAR * 8;
constexpr int OFF_TM = OFF_CMD + 16;
constexpr int SMEM = OFF_TM + 16 + 1024;
static_assert(SMEM <= 232448, "shared memory over the 227 KB per-CTA limit");
static_assert(PK_W3 % 1024 == 0 && (4 * kN3 * 128) % 1024 == 0 && (kN3 * 128) % 1024 == 0,
              "SW128 alignment");
static_assert(OFF_AE % 128 == 0 && OFF_BE % 16 == 0 && OFF_BAR % 8 == 0, "alignment");

constexpr uint32_t TM_H = 256;   // TMEM columns of h1 / h2 (packed BF16 A operand)
constexpr uint32_t TM_E = 384;   // TMEM columns of the two energy accumulators

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

// Energy image: per block of 64 Gaussians, the B operand rows
// [c_hi (D), c_lo (D), c_hi (D), 0...] (K = 80, no swizzle) followed by the
// table {|c|^2, q = -log2(e) / (2 w^2), a, 0}; Gaussians beyond M have a = 0.
__global__ void k_land_tc_pack_energy(const float *__restrict__ c, const float *__restrict__ w,
                                      const float *__restrict__ a, int D, int M, int Mp,
                                      uint8_t *__restrict__ img) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  for (int i = tid; i < Mp * kKE; i += stride) {
    const int m = i / kKE, k = i % kKE;
    float v = 0.f;
    if (m < M && k < 3 * D) {
      const float x = c[(size_t)m * D + (k % D)];
      const float hi = bf16_val(x);
      v = (k / D == 1) ? x - hi : x;
    }
    const int blk = m / kBlk, n = m % kBlk;
    *(uint16_t *)(img + (size_t)blk * kBlkBytes + ns_off(n, k, kKE)) = bf16_bits(v);
  }
  for (int m = tid; m < Mp; m += stride) {
    float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
    if (m < M) {
      float s = 0.f;
      for (int j = 0; j < D; ++j) s = fmaf(c[(size_t)m * D + j], c[(size_t)m * D + j], s);
      t.x = s;
      t.y = -1.4426950408889634f / (2.0f * w[m] * w[m]);
      t.z = a[m];
    }
    *(float4 *)(img + (size_t)(m / kBlk) * kBlkBytes + kBlkImg + (m % kBlk) * 16) = t;
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
__device__ __forceinline__ bool mbar_wait_cluster(uint64_t *bar, uint32_t parity) {
  const uint32_t a = tc::smem_u32(bar);
  uint64_t t0 = 0;
  for (int it = 0;; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
    if (it == 0) t0 = tc::global_ns();
    else if ((it & 255) == 0 && tc::global_ns() - t0 > kWaitNs) return false;
  }
}

// Barrier ids: 1 the 256 epilogue threads; 2 + w the two warps (w, w + 4) of rows 32w..
constexpr uint32_t kBarEpi = 1, kBarPair0 = 2;

template <int D, int CL>
__global__ void __launch_bounds__(kThreads, 1)
    k_land_tc(Dev d, const uint8_t *__restrict__ pol, const uint8_t *__restrict__ eimg, int n_blk,
              uint32_t n_steps) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = tc::smem_u32(smem_raw);
  uint8_t *sm = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
  const uint32_t sb = tc::smem_u32(sm);
  const int tid = threadIdx.x, warp = tid >> 5;
  uint64_t *bars = (uint64_t *)(sm + OFF_BAR);
  uint64_t *bar_ae = bars, *bar_b = bars + 1, *bar_mma = bars + 3, *bar_epi = bars + 5;
  uint64_t *bar_pol = bars + 7, *bar_x = bars + 8, *bar_drain = bars + 9;
  volatile uint32_t *cmd = (volatile uint32_t *)(sm + OFF_CMD);
  uint32_t *tm_holder = (uint32_t *)(sm + OFF_TM);
  const uint32_t rank = CL > 1 ? cluster_rank() : 0u;

  {
    const uint4 *src = (const uint4 *)pol;
    uint4 *dst = (uint4 *)sm;
    for (int i = tid; i < POLICY / 16; i += kThreads) dst[i] = __ldg(src + i);
  }
  if (tid == 0) {
    tc::mbar_init(bar_ae, kEpi);
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(bar_b + i, 1);
      tc::mbar_init(bar_mma + i, 1);
      tc::mbar_init(bar_epi + i, kEpi);
    }
    tc::mbar_init(bar_pol, 1);
    tc::mbar_init(bar_x, kRows);
    tc::mbar_init(bar_drain, 1);
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
  bool fail = false;

  if (tid >= kEpi) {
    // ===================== producer: energy blocks in, MMAs out =====================
    if (tid == kEpi) {
      const uint8_t *src0 = eimg + (size_t)rank * n_blk * kBlkBytes;
      constexpr uint32_t idesc = tc::idesc_bf16_f32(128, kBlk);
      uint32_t g = 0, pa = 0;
      auto load = [&](uint32_t gg) -> bool {
        const uint32_t b = gg & 1u;
        if (gg >= 2 && !tc::mbar_wait(bar_epi + b, ((gg >> 1) - 1u) & 1u, kWaitNs)) return false;
        mbar_expect_tx(bar_b + b, kBlkBytes);
        bulk_g2s(sb + OFF_BE + b * kBlkBytes, src0 + (size_t)(gg % (uint32_t)n_blk) * kBlkBytes,
                 kBlkBytes, bar_b + b);
        return true;
      };
      bool loaded = load(0);
      fail = !loaded;
      while (!fail) {
        if (!tc::mbar_wait(bar_ae, pa, kWaitNs)) { fail = true; break; }
        pa ^= 1u;
        if (*cmd == 0u) break;
        for (int i = 0; i < n_blk && !fail; ++i, ++g) {
          const uint32_t b = g & 1u;
          if (!tc::mbar_wait(bar_b + b, (g >> 1) & 1u, kWaitNs)) { fail = true; loaded = false; break; }
          tc::fence_after_sync();
#pragma unroll
          for (int s = 0; s < kKE / 16; ++s) {
            const uint64_t da = tc::smem_desc(sb + OFF_AE + (uint32_t)s * 256u, 128, kKE * 16,
                                              tc::kSwizzleNone);
            const uint64_t db = tc::smem_desc(sb + OFF_BE + b * kBlkBytes + (uint32_t)s * 256u, 128,
                                              kKE * 16, tc::kSwizzleNone);
            tc::mma_bf16(tbase + TM_E + b * kBlk, da, db, idesc, s != 0);
          }
          tc::mma_commit(bar_mma + b);
          if (!load(g + 1)) { fail = true; loaded = false; }
        }
      }
      // the prefetched block g is in flight: wait for it before shared memory goes away
      if (loaded) tc::mbar_wait(bar_b + (g & 1u), (g >> 1) & 1u, kWaitNs);
      tc::mma_commit(bar_drain);
      tc::mbar_wait(bar_drain, 0, kWaitNs);
      if (fail) {
        atomicExch(d.err, 1u);
        atomicExch(d.err + 1, 500u);
      }
    }
  } else {
    // ===================== epilogue: env rows =====================
    const int r = tid & 127, h = tid >> 7;
    const bool own = h == 0;  // warps 0-3 hold the env state
    const uint32_t lane_sel = (uint32_t)((warp & 3) * 32) << 16;
    const uint32_t pair = kBarPair0 + (uint32_t)(warp & 3);
    float *xch_e = (float *)(sm + OFF_XCH), *xch_y = xch_e + kRows;
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
      if (!fail && !tc::mbar_wait(bar, parity, kWaitNs)) fail = true;
    };
    const uint32_t partner = rank ^ 1u;
    const uint32_t recv_remote = CL > 1 ? mapa(sb + OFF_RECV, partner) : 0u;
    const uint32_t barx_remote = CL > 1 ? mapa(tc::smem_u32(bar_x), partner) : 0u;

    // One energy sweep over this CTA's Gaussians at the rows written to the
    // energy operand; returns the whole-landscape energy on the owner threads.
    auto sweep = [&](float yy) -> float {
      if (tid == 0) *cmd = 1u;
      tc::fence_async_smem();
      mbar_arrive(bar_ae);
      float part = 0.f;
      for (int i = 0; i < n_blk; ++i, ++ge) {
        const uint32_t b = ge & 1u;
        wait(bar_mma + b, (ge >> 1) & 1u);
        // the block's table arrived by bulk copy: observe its completion before
        // reading it with ordinary loads (its phase is the one the MMA waited on)
        wait(bar_b + b, (ge >> 1) & 1u);
        tc::fence_after_sync();
        uint32_t z[32];
        tc::tmem_ld32(tbase + lane_sel + TM_E + b * kBlk + (uint32_t)(32 * h), z);
        tc::tmem_wait_ld();
        const uint32_t tab = sb + OFF_BE + b * kBlkBytes + kBlkImg + (uint32_t)(32 * h) * 16u;
#pragma unroll
        for (int c = 0; c < 32; ++c) {
          const float4 t = lds128f(tab + 16u * (uint32_t)c);
          const float d2 = fmaf(-2.0f, __uint_as_float(z[c]), yy + t.x);
          part = fmaf(t.z, ex2_fast(d2 * t.y), part);
        }
        tc::fence_before_sync();
        mbar_arrive(bar_epi + b);
      }
      if (!own) xch_e[r] = part;
      bar_sync_n(pair, 64);
      float E = 0.f;
      if (own) {
        E = part + xch_e[r];
        if (CL > 1) {
          st_cluster_f32(recv_remote + (par * kRows + (uint32_t)r) * 4u, E);
          arrive_remote(barx_remote);
          if (!fail && !mbar_wait_cluster(bar_x, px)) fail = true;
          const float other = recv[par * kRows + r];
          E = rank == 0 ? E + other : other + E;
        }
      }
      px ^= 1u;
      par ^= 1u;
      bar_sync_n(pair, 64);  // xch_e is free again
      return E;
    };
    // Energy operand row [y_hi | y_hi | y_lo | 0] (K = 80) of the owner's row;
    // |y|^2 (FP32) goes to both threads of the row.
    auto write_ae = [&](const float (&y)[kMaxD]) -> float {
      float yy = 0.f;
      if (own) {
        uint32_t hi[kMaxD / 2], lo[kMaxD / 2];
#pragma unroll
        for (int j = 0; j < kMaxD; j += 2) {
          const float a0 = j < D ? y[j] : 0.f, a1 = j + 1 < D ? y[j + 1] : 0.f;
          yy = fmaf(a0, a0, yy);
          yy = fmaf(a1, a1, yy);
          const uint32_t hp = tc::pack_bf16x2(a0, a1);
          hi[j / 2] = hp;
          lo[j / 2] = tc::pack_bf16x2(a0 - tc::bf16_lo(hp), a1 - tc::bf16_hi(hp));
        }
        const uint32_t row = sb + OFF_AE + (uint32_t)(r >> 3) * (kKE * 16) + (uint32_t)(r & 7) * 16u;
        constexpr int nc = D / 8;  // chunks of 8 per third
#pragma unroll
        for (int c = 0; c < kKE / 8; ++c) {
          uint32_t q0 = 0u, q1 = 0u, q2 = 0u, q3 = 0u;
          const int third = c / nc, cc = c % nc;
          if (c < 3 * nc) {
            // thirds 0 and 1: y_hi; third 2: y_lo
#pragma unroll
            for (int u = 0; u < kMaxD / 8; ++u) {
              if (u == cc) {
                const uint32_t *src = third == 2 ? lo : hi;
                q0 = src[4 * u];
                q1 = src[4 * u + 1];
                q2 = src[4 * u + 2];
                q3 = src[4 * u + 3];
              }
            }
          }
          tc::sts128(row + (uint32_t)c * 128u, q0, q1, q2, q3);
        }
        xch_y[r] = yy;
      }
      bar_sync_n(pair, 64);
      if (!own) yy = xch_y[r];
      return yy;
    };

    for (int tile = cid; tile < n_tiles && !fail; tile += n_clus) {
      const uint32_t e = (uint32_t)tile * kRows + (uint32_t)r;
      const bool valid = e < N;
      float x[kMaxD];
      float eobs = 0.f;
      int t = 0;
#pragma unroll
      for (int j = 0; j < kMaxD; ++j) x[j] = (own && valid && j < D) ? d.s[(size_t)j * N + e] : 0.f;
      if (own && valid) {
        eobs = d.eobs[e];
        t = d.t[e];
      }
      const bool rec = own && valid && rank == 0;
      for (uint32_t s = 0; s < n_steps; ++s) {
        const uint32_t k = (uint32_t)(k0 + s);
        const size_t rowR = (size_t)((k0 + s) % R);
        // ---- observation record and the layer-1 operand row [x, 1, 1, 0...]
        if (own) {
          if (rec)
            for (int j = 0; j < D; ++j) d.r_obs[(rowR * D + (size_t)j) * S + e] = x[j];
          const uint32_t row = sb + OFF_AE + (uint32_t)(r >> 3) * (kK1 * 16) + (uint32_t)(r & 7) * 16u;
#pragma unroll
          for (int c = 0; c < kK1 / 8; ++c) {
            uint32_t q[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int j = 8 * c + 2 * u;
              const float a0 = j < D ? x[j < kMaxD ? j : 0] : (j == D ? 1.f : 0.f);
              const float a1 = j + 1 < D ? x[j + 1 < kMaxD ? j + 1 : 0] : (j + 1 == D + 1 ? 1.f : 0.f);
              q[u] = tc::pack_bf16x2(a0, a1);
            }
            tc::sts128(row + (uint32_t)c * 128u, q[0], q[1], q[2], q[3]);
          }
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
#pragma unroll 1
        for (int l = 0; l < 3; ++l) {
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
        // ---- sample the Gaussian head, candidate y = x + dx
        float y[kMaxD];
#pragma unroll
        for (int j = 0; j < kMaxD; ++j) y[j] = x[j];
        if (own) {
          float out[kN3];
#pragma unroll
          for (int q = 0; q < kN3 / 16; ++q) {
            uint32_t z[16];
            tmem_ld16(tbase + lane_sel + (uint32_t)(16 * q), z);
            tc::tmem_wait_ld();
#pragma unroll
            for (int i = 0; i < 16; ++i)
              out[16 * q + i] = __uint_as_float(z[i]) + *(const float *)(sm + PK_B3 + (16 * q + i) * 4);
          }
          float lp = 0.f;
          float *act = (float *)d.r_act + rowR * (size_t)D * S + e;
#pragma unroll
          for (int j = 0; j < kMaxD; j += 4) {
            if (j < D) {
              const uint4 rw = draw(seed, k, e, 0, kTagAction, (uint32_t)(j >> 2));
              const float2 p = box_muller(rw.x, rw.y), q2 = box_muller(rw.z, rw.w);
              const float z4[4] = {p.x, p.y, q2.x, q2.y};
#pragma unroll
              for (int i = 0; i < 4; ++i) {
                const float mu = out[j + i], lsr = out[D + j + i];
                const float zz = z4[i];
                const float ls = fminf(fmaxf(lsr, -5.0f), 2.0f);
                const float smp = mu + expf(ls) * zz;
                const float dx = fminf(fmaxf(smp, -clip), clip);
                if (rec) act[(size_t)(j + i) * S] = dx;
                lp += -0.5f * zz * zz - ls - half_log_2pi;
                y[j + i] = x[j + i] + dx;
              }
            }
          }
          if (rec) d.r_logp[rowR * S + e] = lp;
          if (rec && d.dbg_logits) {
#pragma unroll
            for (int i = 0; i < 2 * D; ++i) d.out[(size_t)e * 2 * D + i] = out[i];
          }
        }
        const float yy = write_ae(y);
        const float E2 = sweep(yy);
        // ---- step: observed energy, reward, done, auto-reset
        bool done = false;
        if (own) {
          const uint4 rn = draw(seed, k, e, 0, kTagNoise, 0);
          const float eobs2 = E2 + sig_n * box_muller(rn.x, rn.y).x;
          const int t2 = t + 1;
          done = valid && t2 >= (int)d.episode_limit;
          if (rec) {
            const size_t o = rowR * S + e;
            d.r_energy[o] = E2;
            d.r_rew[o] = eobs - eobs2;
            d.r_done[o] = (uint8_t)done;
          }
          if (done) {
#pragma unroll
            for (int j = 0; j < kMaxD; j += 4) {
              if (j < D) {
                const uint4 rr = draw(seed, k, e, 0, kTagReset, (uint32_t)(j >> 2));
                x[j] = uniform(rr.x, -3.0f, 3.0f);
                if (j + 1 < D) x[j + 1] = uniform(rr.y, -3.0f, 3.0f);
                if (j + 2 < D) x[j + 2] = uniform(rr.z, -3.0f, 3.0f);
                if (j + 3 < D) x[j + 3] = uniform(rr.w, -3.0f, 3.0f);
              }
            }
            t = 0;
          } else {
#pragma unroll
            for (int j = 0; j < kMaxD; ++j) x[j] = y[j];
            eobs = eobs2;
            t = t2;
          }
        }
        // a tile with a reset sweeps again at the fresh states (identical vote on
        // every CTA of the cluster: they hold identical states)
        if (bar_any_n(kBarEpi, kEpi, done)) {
          const float xx = write_ae(x);
          const float E0 = sweep(xx);
          if (own && done) {
            const uint4 rn = draw(seed, k, e, 0, kTagNoise, 1);
            eobs = E0 + sig_n * box_muller(rn.x, rn.y).x;
          }
        }
      }
      if (rec && !fail) {
        for (int j = 0; j < D; ++j) d.s[(size_t)j * N + e] = x[j];
        d.eobs[e] = eobs;
        d.t[e] = t;
        d.needs_energy[e] = 0;
      }
    }
    // stop the producer
    bar_sync_n(kBarEpi, kEpi);
    if (tid == 0) *cmd = 0u;
    mbar_arrive(bar_ae);
    if (fail && tid == 0) {
      // a policy MMA may still be in flight after a wait that ran out
      tc::mma_commit(bar_pol);
      tc::mbar_wait(bar_pol, pp, kWaitNs);
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

}  // namespace

bool land_tc_supported(int D, int M, const PolicyShape &p) {
  return D >= 8 && D <= kMaxD && D % 8 == 0 && M >= 1 && p.w[0] == D && p.w[1] == kH &&
         p.w[2] == kH && p.w[3] == 2 * D;
}
size_t land_tc_policy_bytes() { return (size_t)POLICY; }
int land_tc_padded_gauss(int M) { return (M + 2 * kBlk - 1) / (2 * kBlk) * (2 * kBlk); }
size_t land_tc_energy_bytes(int M) { return (size_t)(land_tc_padded_gauss(M) / kBlk) * kBlkBytes; }

void launch_land_tc_pack(const Dev &d, void *policy_img, void *energy_img, cudaStream_t st) {
  k_land_tc_pack_policy<<<64, 256, 0, st>>>(d.params, (int)d.dim, (uint8_t *)policy_img);
  k_land_tc_pack_energy<<<128, 256, 0, st>>>(d.centres, d.widths, d.amps, (int)d.dim, (int)d.n_gauss,
                                             land_tc_padded_gauss((int)d.n_gauss),
                                             (uint8_t *)energy_img);
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
  const int Mp = land_tc_padded_gauss((int)d.n_gauss);
  if (tile_ctas == 1) {
    const int grid = n_tiles < sms ? n_tiles : sms;
    k_land_tc<D, 1><<<grid, kThreads, SMEM, st>>>(d, pol, eimg, Mp / kBlk, n_steps);
    return cudaGetLastError();
  }
  if (tile_ctas != 2) return cudaErrorInvalidValue;
  const int clusters = n_tiles < sms / 2 ? n_tiles : sms / 2;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(2 * clusters));
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = SMEM;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_land_tc<D, 2>, d, pol, eimg, Mp / kBlk / 2, n_steps);
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
