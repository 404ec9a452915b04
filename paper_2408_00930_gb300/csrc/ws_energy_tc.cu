// ws_energy_tc.cu -- Gaussian-sum energy of the reaction landscape with the
// distance cross-term on the tcgen05 tensor cores (BF16 path).
//
//   E(y) = sum_m a_m exp(-|y - c_m|^2 / (2 w_m^2)),
//   |y - c_m|^2 = |y|^2 + |c_m|^2 - 2 y.c_m,
//
// y.c_m for 128 envs x 256 Gaussians per MMA group, in BF16 with a hi+lo split
// that restores FP32-level accuracy of the product: the operand row of env y
// is [y_hi, y_hi, y_lo] against [c_hi, c_lo, c_hi] for Gaussian m (the missing
// term y_lo.c_lo is ~2^-18 |y||c|).  |y|^2 and |c|^2 stay FP32.  The epilogue
// (one TMEM row per thread) evaluates a_m 2^(q_m d2) with q_m = -log2(e)/(2w^2)
// and sums over the chunk's Gaussians; partial sums go to the same per-chunk
// buffer the FP32 path uses, so the env step combines them in fixed order.
//
// Warp roles: warps 0-3 build the operand rows and run the epilogue; warp 4
// (one lane) streams 256-Gaussian blocks of the packed centre image into two
// shared-memory buffers with 1-D bulk copies and issues the MMAs into two
// 256-column TMEM accumulators, so the MMA of block j+1 overlaps the epilogue
// of block j.
#include "ws_kernels.cuh"
#include "ws_tc.cuh"

namespace ws {

namespace {

constexpr int kRows = 128;               // envs per CTA tile
constexpr int kThreads = kRows + 32;     // 4 epilogue warps + 1 producer warp
constexpr int kBlockG = 256;             // Gaussians per MMA group (N)
constexpr int kKB = 2;                   // K-blocks of 64: 3 D <= 128
constexpr int kABytes = kKB * kRows * 128;
constexpr int kBBytes = kKB * kBlockG * 128;
constexpr uint64_t kWaitNs = 2000000000ull;
constexpr uint32_t kTmemCols = 512;
// Gaussian chunks per env tile (1, 2 or 4; a launch parameter the tuner
// picks): each CTA sweeps Mp / chunks Gaussians in 256-wide blocks through its
// double-buffered pipeline (long enough to amortise its set-up); partial sums
// land in the first `chunks` of the kEnergyChunks slots, whose others are kept
// at zero.  Mp is padded for the largest count, so one image serves all.
constexpr int kMaxTcChunks = 4;

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
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

// Packed centre image, per padded Gaussian row m: [c_hi (D), c_lo (D), c_hi (D),
// zeros] in 128B-swizzled K-major layout, K-block-major ([kb][m][128 B]); and
// the table {|c_m|^2, q_m, a_m, 0}.  Rows beyond M are zero (a_m = 0).
__global__ void k_energy_tc_pack(const float *__restrict__ c, const float *__restrict__ w,
                                 const float *__restrict__ a, int D, int M, int Mp,
                                 uint8_t *__restrict__ img, float4 *__restrict__ tab) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  for (int i = tid; i < Mp * kKB * 64; i += stride) {
    const int m = i / (kKB * 64), k = i % (kKB * 64);
    float v = 0.f;
    if (m < M && k < 3 * D) {
      const float x = c[(size_t)m * D + (k % D)];
      const float hi = tc::bf16_lo(tc::pack_bf16x2(x, 0.f));
      v = (k / D == 1) ? x - hi : x;  // the pack below rounds to bf16
    }
    const int kb = k >> 6, kk = k & 63;
    const size_t off = (size_t)kb * Mp * 128 + (size_t)m * 128 + (((kk >> 3) ^ (m & 7)) << 4) + (kk & 7) * 2;
    *(uint16_t *)(img + off) = (uint16_t)(tc::pack_bf16x2(v, 0.f) & 0xFFFFu);
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
    tab[m] = t;
  }
}

// grid (env tiles, chunks); block 160.  mode 0: y = x + dx; mode 1: y = x for
// envs flagged needs_energy (tiles without one return at once).
__global__ void __launch_bounds__(kThreads, 1)
    k_energy_tc(Dev d, uint32_t off, int mode, const uint8_t *__restrict__ img,
                const float4 *__restrict__ tab, int Mp, int per_chunk) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = tc::smem_u32(smem_raw);
  uint8_t *sm = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
  const uint32_t sb = tc::smem_u32(sm);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int D = (int)d.dim;
  const uint32_t e = blockIdx.x * kRows + (uint32_t)(tid & 127);
  const bool epi = tid < kRows;
  const bool valid = epi && e < d.n_envs;
  const bool want = valid && (mode == 0 || d.needs_energy[e]);
  if (!__syncthreads_or(want)) return;

  const uint32_t off_a = 0, off_b = kABytes;  // A, then two B buffers
  float4 *stab = (float4 *)(sm + kABytes + 2 * kBBytes);
  uint64_t *bars = (uint64_t *)(sm + kABytes + 2 * kBBytes + per_chunk * 16);
  uint64_t *bar_a = bars, *bar_b = bars + 1, *bar_mma = bars + 3, *bar_epi = bars + 5;
  uint64_t *bar_drain = bars + 7;
  uint32_t *tm_holder = (uint32_t *)(bars + 8);
  const int g0 = blockIdx.y * per_chunk;
  const int nblk = per_chunk / kBlockG;

  for (int i = tid; i < per_chunk; i += kThreads) stab[i] = tab[g0 + i];
  if (tid == 0) {
    tc::mbar_init(bar_a, kRows);
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(bar_b + i, 1);
      tc::mbar_init(bar_mma + i, 1);
      tc::mbar_init(bar_epi + i, kRows);
    }
    tc::mbar_init(bar_drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tc::tmem_alloc(tm_holder, kTmemCols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tm_holder;
  bool ok = true;

  if (!epi) {
    // ---------------- producer: centre blocks in, MMAs out ----------------
    if (tid == kRows) {
      constexpr uint32_t idesc = tc::idesc_bf16_f32(128, kBlockG);
      const int ksteps = (3 * D + 15) / 16;
      uint32_t ph_b[2] = {0, 0}, ph_e[2] = {0, 0};
      ok = tc::mbar_wait(bar_a, 0, kWaitNs);
      for (int j = 0; ok && j < nblk; ++j) {
        const int b = j & 1;
        if (j >= 2) {  // accumulator and buffer b free once block j-2 is consumed
          ok = tc::mbar_wait(bar_epi + b, ph_e[b], kWaitNs);
          ph_e[b] ^= 1u;
          if (!ok) break;
        }
        const uint32_t dst = sb + off_b + (uint32_t)b * kBBytes;
        mbar_expect_tx(bar_b + b, kBBytes);
        for (int kb = 0; kb < kKB; ++kb)
          bulk_g2s(dst + kb * (kBlockG * 128),
                   img + (size_t)kb * Mp * 128 + (size_t)(g0 + j * kBlockG) * 128, kBlockG * 128,
                   bar_b + b);
        ok = tc::mbar_wait(bar_b + b, ph_b[b], kWaitNs);
        ph_b[b] ^= 1u;
        if (!ok) break;
        tc::fence_after_sync();
        for (int s = 0; s < ksteps; ++s) {
          const int kb = s >> 2, kk = s & 3;
          const uint64_t da = tc::smem_desc(sb + off_a + kb * (kRows * 128) + kk * 32, 16, 1024,
                                            tc::kSwizzle128B);
          const uint64_t db = tc::smem_desc(dst + kb * (kBlockG * 128) + kk * 32, 16, 1024,
                                            tc::kSwizzle128B);
          tc::mma_bf16(tmem + (uint32_t)b * 256u, da, db, idesc, s != 0);
        }
        tc::mma_commit(bar_mma + b);
      }
      if (!ok) {
        atomicExch(d.err, 1u);
        atomicExch(d.err + 1, 300u);
      }
      // make sure no MMA is still writing TMEM when the columns are released
      tc::mma_commit(bar_drain);
      tc::mbar_wait(bar_drain, 0, kWaitNs);
    }
  } else {
    // ---------------- epilogue warps: operand rows, then exp-sums ----------------
    const int r = tid;
    const uint32_t lane = (uint32_t)((warp & 3) * 32) << 16;
    float yy = 0.f;
    {
      // operand row [y_hi, y_hi, y_lo, 0...] over kKB K-blocks of 64, written
      // element by element at its 128B-swizzled position
      const uint32_t ra = sb + off_a + (uint32_t)r * 128u;
      const uint32_t swz = (uint32_t)(r & 7);
#pragma unroll
      for (int kb = 0; kb < kKB; ++kb)
#pragma unroll
        for (int ch = 0; ch < 8; ++ch) tc::sts128(ra + kb * (kRows * 128) + (ch << 4), 0u, 0u, 0u, 0u);
      const uint32_t row = (uint32_t)((d.k[0] + off) % d.ring_steps);
      const float *act = (const float *)d.r_act + (size_t)row * D * d.n_slots;
#pragma unroll
      for (int j = 0; j < 40; ++j) {
        if (j < D) {
          float v = 0.f;
          if (valid) {
            v = d.s[(size_t)j * d.n_envs + e];
            if (mode == 0) v = v + act[(size_t)j * d.n_slots + e];
          }
          yy = fmaf(v, v, yy);
          const uint32_t hv = tc::pack_bf16x2(v, 0.f) & 0xFFFFu;
          const uint32_t lv = tc::pack_bf16x2(v - __uint_as_float(hv << 16), 0.f) & 0xFFFFu;
          const int ks[3] = {j, D + j, 2 * D + j};
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            const int k = ks[q], kb = k >> 6, kk = k & 63;
            const uint32_t addr = ra + kb * (kRows * 128) + ((((uint32_t)kk >> 3) ^ swz) << 4) + (kk & 7) * 2;
            const uint32_t bits = q == 2 ? lv : hv;
            asm volatile("st.shared.u16 [%0], %1;" ::"r"(addr), "h"((unsigned short)bits) : "memory");
          }
        }
      }
    }
    tc::fence_async_smem();
    mbar_arrive(bar_a);
    float sum = 0.f;
    uint32_t ph_m[2] = {0, 0};
    for (int j = 0; j < nblk; ++j) {
      const int b = j & 1;
      ok = tc::mbar_wait(bar_mma + b, ph_m[b], kWaitNs);
      ph_m[b] ^= 1u;
      if (!ok) break;
      tc::fence_after_sync();
      const float4 *t = stab + j * kBlockG;
      for (int c0 = 0; c0 < kBlockG; c0 += 32) {
        uint32_t z[32];
        tc::tmem_ld32(tmem + lane + (uint32_t)b * 256u + (uint32_t)c0, z);
        tc::tmem_wait_ld();
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const float4 g = t[c0 + i];
          const float d2 = fmaf(-2.0f, __uint_as_float(z[i]), yy + g.x);
          sum = fmaf(g.z, ex2_fast(d2 * g.y), sum);
        }
      }
      tc::fence_before_sync();
      mbar_arrive(bar_epi + b);
    }
    if (!ok) {
      atomicExch(d.err, 1u);
      atomicExch(d.err + 1, 301u);
    }
    if (want) {
      d.epart[((size_t)blockIdx.y * 2 + 0) * d.n_envs + e] = sum;
      d.epart[((size_t)blockIdx.y * 2 + 1) * d.n_envs + e] = 0.f;
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(*tm_holder, kTmemCols);
  }
}

size_t smem_for(int per_chunk) {
  return (size_t)kABytes + 2 * kBBytes + (size_t)per_chunk * 16 + 10 * 8 + 1024;
}

}  // namespace

// Padded Gaussian count (a multiple of 4 * 256) and the chunk size for `chunks`.
void energy_tc_shape(int M, int chunks, int *Mp, int *per_chunk) {
  const int blk = kMaxTcChunks * kBlockG;
  *Mp = (M + blk - 1) / blk * blk;
  *per_chunk = *Mp / chunks;
}

size_t energy_tc_bytes(int D, int M) {
  int Mp, pc;
  energy_tc_shape(M, kMaxTcChunks, &Mp, &pc);
  (void)D;
  return (size_t)Mp * kKB * 128 + (size_t)Mp * 16;
}

bool energy_tc_supported(int D, int M) {
  int Mp, pc;
  energy_tc_shape(M, kMaxTcChunks, &Mp, &pc);
  return D >= 1 && 3 * D <= kKB * 64 && D <= 40 && smem_for(pc) <= 232448;
}

bool energy_tc_chunks_ok(int M, int chunks) {
  if (chunks != 1 && chunks != 2 && chunks != 4) return false;
  int Mp, pc;
  energy_tc_shape(M, chunks, &Mp, &pc);
  return smem_for(pc) <= 232448;
}

void launch_energy_tc_pack(const Dev &d, void *buf, cudaStream_t st) {
  int Mp, pc;
  energy_tc_shape((int)d.n_gauss, kMaxTcChunks, &Mp, &pc);
  uint8_t *img = (uint8_t *)buf;
  float4 *tab = (float4 *)(img + (size_t)Mp * kKB * 128);
  k_energy_tc_pack<<<256, 256, 0, st>>>(d.centres, d.widths, d.amps, (int)d.dim, (int)d.n_gauss, Mp,
                                         img, tab);
}

void energy_tc_init(int M) {
  int Mp, pc = 0;
  for (int c = 1; c <= kMaxTcChunks; c *= 2) {
    if (!energy_tc_chunks_ok(M, c)) continue;
    energy_tc_shape(M, c, &Mp, &pc);
    break;  // the smallest supported count has the largest chunk
  }
  cudaFuncSetAttribute(k_energy_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_for(pc));
}

void launch_energy_tc(const Dev &d, const void *buf, uint32_t off, int mode, cudaStream_t st) {
  int Mp, pc;
  const int chunks = d.energy_chunks > 0 ? d.energy_chunks : 2;
  energy_tc_shape((int)d.n_gauss, chunks, &Mp, &pc);
  const uint8_t *img = (const uint8_t *)buf;
  const float4 *tab = (const float4 *)(img + (size_t)Mp * kKB * 128);
  dim3 grid((d.n_envs + kRows - 1) / kRows, chunks);
  k_energy_tc<<<grid, kThreads, smem_for(pc), st>>>(d, off, mode, img, tab, Mp, pc);
}

}  // namespace ws
