// ws_dense_tc.cu -- one policy layer on the tcgen05 tensor cores:
//   Y[M][N] = act(X[M][K] W[K][N] + b)  with BF16 operands, FP32 accumulation
// in TMEM, bias and tanh in the epilogue.  Used per layer by the BF16 paths of
// the economy and the landscape (paper App. B: every agent thread runs policy
// inference on the model held in global memory; here 128 agents form one MMA
// tile, two tiles per CTA, persistent over the rows).
//
// W^T (N rows padded to a multiple of 16, K padded to 64) stays resident in
// shared memory as a 128B-swizzled K-major operand; each thread converts its
// own row of X (FP32 in any stride, or BF16 row-major) into the A operand, one
// K-block of 64 at a time through two 16 KB slots per warpgroup.
#include "ws_kernels.cuh"
#include "ws_tc.cuh"

namespace ws {

namespace {

constexpr int kTile = 128;
constexpr int kWG = 2;
constexpr int kThreads = kTile * kWG;
constexpr uint64_t kWaitNs = 2000000000ull;
constexpr uint32_t kTmemCols = 512;
constexpr int kSlot = 128 * 128;

struct DenseArgs {
  const void *X;
  long ldr, ldc;      // FP32 input addressing X[row * ldr + k * ldc]
  int x_bf16;         // 1: X is BF16 row-major [M][K]
  int K, N, Np, KB;   // true K, N; N padded to 16; K-blocks of 64
  const uint8_t *packed;
  void *Y;
  int y_bf16;         // 1: Y is BF16 row-major [M][N], else FP32 row-major
  int act;            // 1: tanh
  long M;
  uint32_t *err;
};

inline int pad16(int n) { return (n + 15) / 16 * 16; }

__device__ __forceinline__ uint16_t bf16_bits(float f) {
  return (uint16_t)(tc::pack_bf16x2(f, 0.f) & 0xFFFFu);
}

// W [K][N] row-major FP32 -> B image (Np rows, K-blocks of 64, SW128) + bias [Np].
__global__ void k_dense_tc_pack(const float *__restrict__ W, const float *__restrict__ b, int K,
                                int N, int Np, int KB, uint8_t *__restrict__ packed) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  const int Kp = KB * 64;
  for (int i = tid; i < Np * Kp; i += stride) {
    const int n = i / Kp, k = i % Kp;
    const float v = (n < N && k < K) ? W[(size_t)k * N + n] : 0.f;
    const int kb = k >> 6, kk = k & 63;
    const int off = kb * (Np * 128) + n * 128 + (((kk >> 3) ^ (n & 7)) << 4) + (kk & 7) * 2;
    *(uint16_t *)(packed + off) = bf16_bits(v);
  }
  float *bias = (float *)(packed + (size_t)KB * Np * 128);
  for (int n = tid; n < Np; n += stride) bias[n] = n < N ? b[n] : 0.f;
}

__device__ __forceinline__ void store_row_sw128(uint32_t row_addr, uint32_t swz,
                                                const uint32_t (&p)[32]) {
#pragma unroll
  for (int ch = 0; ch < 8; ++ch)
    tc::sts128(row_addr + (((uint32_t)ch ^ swz) << 4), p[ch * 4 + 0], p[ch * 4 + 1], p[ch * 4 + 2],
               p[ch * 4 + 3]);
}

// This thread's row of X, K-block kb, as 32 packed bf16 pairs.
__device__ __forceinline__ void load_row(const DenseArgs &a, long row, bool valid, int kb,
                                         uint32_t (&p)[32]) {
  const int k0 = kb * 64;
  if (a.x_bf16) {
    const uint4 *src = (const uint4 *)((const uint16_t *)a.X + row * a.K + k0);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      uint4 v = make_uint4(0, 0, 0, 0);
      if (valid && k0 + c * 8 < a.K) v = __ldg(src + c);
      p[c * 4 + 0] = v.x;
      p[c * 4 + 1] = v.y;
      p[c * 4 + 2] = v.z;
      p[c * 4 + 3] = v.w;
    }
  } else {
    const float *X = (const float *)a.X;
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      const int k = k0 + 2 * i;
      const float lo = (valid && k < a.K) ? __ldg(X + row * a.ldr + (long)k * a.ldc) : 0.f;
      const float hi = (valid && k + 1 < a.K) ? __ldg(X + row * a.ldr + (long)(k + 1) * a.ldc) : 0.f;
      p[i] = tc::pack_bf16x2(lo, hi);
    }
  }
}

__global__ void __launch_bounds__(kThreads, 1) k_dense_tc(DenseArgs a) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = tc::smem_u32(smem_raw);
  uint8_t *sm = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
  const uint32_t sb = tc::smem_u32(sm);
  const int tid = threadIdx.x, wg = tid >> 7, r = tid & 127, warp = tid >> 5;
  const int b_bytes = a.KB * a.Np * 128;
  const int off_slots = b_bytes;
  const int off_bias = off_slots + kWG * 2 * kSlot;
  const int off_bar = off_bias + a.Np * 4;
  const int off_tm = off_bar + kWG * 3 * 8;
  uint64_t *bars = (uint64_t *)(sm + off_bar) + wg * 3;
  uint64_t *bar_slot = bars, *bar_drain = bars + 2;
  uint32_t *tm_holder = (uint32_t *)(sm + off_tm);
  {
    const uint4 *src = (const uint4 *)a.packed;
    uint4 *dst = (uint4 *)sm;
    for (int i = tid; i < b_bytes / 16; i += kThreads) dst[i] = __ldg(src + i);
    const float *bsrc = (const float *)(a.packed + b_bytes);
    float *bdst = (float *)(sm + off_bias);
    for (int i = tid; i < a.Np; i += kThreads) bdst[i] = bsrc[i];
  }
  if (tid == 0) {
    uint64_t *all = (uint64_t *)(sm + off_bar);
    for (int i = 0; i < kWG * 3; ++i) tc::mbar_init(all + i, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tc::tmem_alloc(tm_holder, kTmemCols);
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();

  const uint32_t tmem = *tm_holder + (uint32_t)wg * 256u;
  const uint32_t lane = (uint32_t)((warp & 3) * 32) << 16;
  const uint32_t bar_id = 1u + (uint32_t)wg;
  const uint32_t slots = sb + off_slots + wg * 2 * kSlot;
  const uint32_t swz = (uint32_t)(r & 7);
  const uint32_t idesc = tc::idesc_bf16_f32(128, (uint32_t)a.Np);
  const float *bias = (const float *)(sm + off_bias);
  uint32_t ph[2] = {0, 0};
  bool ok = true;
  uint32_t fail_site = 0;
  const long n_tiles = (a.M + kTile - 1) / kTile;

  // warpgroup wg of CTA b takes tiles b + wg * grid, + 2 grid, ...: with fewer
  // tiles than SMs every tile gets an SM of its own
  for (long tile = (long)blockIdx.x + (long)wg * gridDim.x; ok && tile < n_tiles;
       tile += (long)gridDim.x * kWG) {
    const long row = tile * kTile + r;
    const bool valid = row < a.M;
    for (int kb = 0; kb < a.KB; ++kb) {
      const int s = kb & 1;
      uint32_t p[32];
      load_row(a, row, valid, kb, p);
      if (kb >= 2) {
        ok = tc::wg_all(bar_id, tc::mbar_wait(bar_slot + s, ph[s], kWaitNs));
        ph[s] ^= 1u;
        if (!ok) { fail_site = 1; break; }
      }
      const uint32_t slot = slots + (uint32_t)s * kSlot;
      store_row_sw128(slot + (uint32_t)r * 128u, swz, p);
      tc::fence_async_smem();
      tc::fence_before_sync();
      tc::wg_sync(bar_id);
      if (r == 0) {
        tc::fence_after_sync();
        // only the K16 steps that hold real K (the rest of the block is zero)
        const int kk_n = min(4, (a.K - kb * 64 + 15) / 16);
        for (int kk = 0; kk < kk_n; ++kk) {
          const uint64_t da = tc::smem_desc(slot + kk * 32, 16, 1024, tc::kSwizzle128B);
          const uint64_t db = tc::smem_desc(sb + kb * (a.Np * 128) + kk * 32, 16, 1024,
                                            tc::kSwizzle128B);
          tc::mma_bf16(tmem, da, db, idesc, (kb | kk) != 0);
        }
        tc::mma_commit(bar_slot + s);
      }
    }
    if (!ok) break;
    // drain the (at most two) outstanding slot commits
    if (a.KB >= 2) {
      const int s = (a.KB - 2) & 1;
      ok = tc::wg_all(bar_id, tc::mbar_wait(bar_slot + s, ph[s], kWaitNs));
      ph[s] ^= 1u;
      if (!ok) { fail_site = 2; break; }
    }
    {
      const int s = (a.KB - 1) & 1;
      ok = tc::wg_all(bar_id, tc::mbar_wait(bar_slot + s, ph[s], kWaitNs));
      ph[s] ^= 1u;
      if (!ok) { fail_site = 3; break; }
    }
    tc::fence_after_sync();
    for (int c0 = 0; c0 < a.Np; c0 += 32) {
      uint32_t z[32];
      if (c0 + 32 <= a.Np) {
        tc::tmem_ld32(tmem + lane + (uint32_t)c0, z);
      } else {  // a 16-column tail
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
            "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
            : "=r"(z[0]), "=r"(z[1]), "=r"(z[2]), "=r"(z[3]), "=r"(z[4]), "=r"(z[5]), "=r"(z[6]),
              "=r"(z[7]), "=r"(z[8]), "=r"(z[9]), "=r"(z[10]), "=r"(z[11]), "=r"(z[12]),
              "=r"(z[13]), "=r"(z[14]), "=r"(z[15])
            : "r"(tmem + lane + (uint32_t)c0));
#pragma unroll
        for (int i = 16; i < 32; ++i) z[i] = 0u;
      }
      tc::tmem_wait_ld();
      if (!valid) continue;
      if (a.y_bf16) {
        uint32_t q[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int c = c0 + 2 * i;
          const float v0 = __uint_as_float(z[2 * i]) + bias[c];
          const float v1 = __uint_as_float(z[2 * i + 1]) + bias[c + 1 < a.Np ? c + 1 : c];
          q[i] = tc::pack_bf16x2(v0, v1);
          if (a.act) q[i] = tc::tanh_bf16x2(q[i]);
        }
        uint4 *dst = (uint4 *)((uint16_t *)a.Y + row * a.N + c0);
#pragma unroll
        for (int c = 0; c < 4; ++c)
          if (c0 + c * 8 < a.N) dst[c] = make_uint4(q[c * 4], q[c * 4 + 1], q[c * 4 + 2], q[c * 4 + 3]);
      } else {
        float *dst = (float *)a.Y + row * a.N;
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const int c = c0 + i;
          if (c < a.N) {
            float v = __uint_as_float(z[i]) + bias[c];
            if (a.act) v = tc::tanh_fast(v);
            dst[c] = v;
          }
        }
      }
    }
    tc::fence_before_sync();  // TMEM reads precede the next tile's MMAs (next sync)
  }
  if (!ok && r == 0) {
    tc::mma_commit(bar_drain);
    tc::mbar_wait(bar_drain, 0, kWaitNs);
    atomicExch(a.err, 1u);
    atomicExch(a.err + 1, 200u + fail_site);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(*tm_holder, kTmemCols);
  }
}

size_t smem_bytes(int KB, int Np) {
  return (size_t)KB * Np * 128 + kWG * 2 * kSlot + Np * 4 + kWG * 3 * 8 + 16 + 1024;
}

}  // namespace

// Raise the kernel's shared-memory limit (once per process and device, before
// any graph capture).
void dense_tc_init() {
  cudaFuncSetAttribute(k_dense_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
}

size_t dense_tc_packed_bytes(int K, int N) {
  const int KB = (K + 63) / 64, Np = pad16(N);
  return (size_t)KB * Np * 128 + (size_t)Np * 4;
}

bool dense_tc_supported(int K, int N) {
  if (K < 1 || N < 1 || pad16(N) > 256 || K > 4096) return false;
  const int KB = (K + 63) / 64;
  return smem_bytes(KB, pad16(N)) <= 232448;
}

void launch_dense_tc_pack(const float *W, const float *b, int K, int N, void *packed,
                          cudaStream_t st) {
  const int KB = (K + 63) / 64, Np = pad16(N);
  k_dense_tc_pack<<<64, 256, 0, st>>>(W, b, K, N, Np, KB, (uint8_t *)packed);
}

cudaError_t launch_dense_tc(const void *X, long ldr, long ldc, int x_bf16, int K,
                            const void *packed, int N, void *Y, int y_bf16, int act, long M,
                            uint32_t *err, cudaStream_t st) {
  if (M <= 0) return cudaSuccess;
  DenseArgs a;
  a.X = X;
  a.ldr = ldr;
  a.ldc = ldc;
  a.x_bf16 = x_bf16;
  a.K = K;
  a.N = N;
  a.Np = pad16(N);
  a.KB = (K + 63) / 64;
  a.packed = (const uint8_t *)packed;
  a.Y = Y;
  a.y_bf16 = y_bf16;
  a.act = act;
  a.M = M;
  a.err = err;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long tiles = (M + kTile - 1) / kTile;
  const long grid = tiles < sms ? tiles : sms;
  size_t smem = smem_bytes(a.KB, a.Np);
  if (smem < 120 * 1024) smem = 120 * 1024;  // one CTA per SM: its 512 TMEM columns uncontended
  k_dense_tc<<<(unsigned)grid, kThreads, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace ws
