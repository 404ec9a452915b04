// ws_mlp3_tc.cu -- a whole three-layer policy MLP per 128-row tile on the
// tcgen05 tensor cores, for policies whose three weight images fit in shared
// memory next to the operand slots (the economy's 16-128-128-20 agent and
// 16-128-128-10 planner policies):
//   out = tanh(tanh(X W1 + b1) W2 + b2) W3 + b3
// with BF16 operands and FP32 accumulation (paper App. B: every agent runs
// inference on the policy held in GPU memory).  The hidden activations never
// leave the SM: each layer's accumulator is read from TMEM, biased, passed
// through tanh as packed bf16x2 and written straight into the next layer's
// 128B-swizzled A slots (hidden widths up to 128 = two K-blocks, so the slots
// never need to be waited on within a layer).  One thread per row, two
// 128-row tiles (warpgroups) per CTA, persistent over the rows.
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

inline int pad16(int n) { return (n + 15) / 16 * 16; }

struct Mlp3Shape {
  int K0, N1, N2, N3;         // true widths
  int N1p, N2p, N3p;          // padded to 16
  int KB1, KB2, KB3;          // K-blocks of 64 per layer
  int b1_off, b2_off, b3_off; // byte offsets of the B images in the packed block
  int bias_off;               // fp32 biases b1 | b2 | b3 (padded widths)
  int bytes;                  // packed block size
};

Mlp3Shape mlp3_shape(const PolicyShape &p) {
  Mlp3Shape s;
  s.K0 = p.w[0];
  s.N1 = p.w[1];
  s.N2 = p.w[2];
  s.N3 = p.w[3];
  s.N1p = pad16(s.N1);
  s.N2p = pad16(s.N2);
  s.N3p = pad16(s.N3);
  s.KB1 = (s.K0 + 63) / 64;
  s.KB2 = (s.N1 + 63) / 64;
  s.KB3 = (s.N2 + 63) / 64;
  s.b1_off = 0;
  s.b2_off = s.b1_off + s.KB1 * s.N1p * 128;
  s.b3_off = s.b2_off + s.KB2 * s.N2p * 128;
  s.bias_off = s.b3_off + s.KB3 * s.N3p * 128;
  s.bytes = s.bias_off + (s.N1p + s.N2p + s.N3p) * 4;
  s.bytes = (s.bytes + 1023) / 1024 * 1024;
  return s;
}

size_t smem_of(const Mlp3Shape &s) {
  return (size_t)s.bytes + kWG * 2 * kSlot + kWG * 2 * 8 + 16 + 1024;
}

__device__ __forceinline__ uint16_t bf16_bits(float f) {
  return (uint16_t)(tc::pack_bf16x2(f, 0.f) & 0xFFFFu);
}

// W [K][N] row-major FP32 -> SW128 K-major image of Np rows, KB K-blocks.
__device__ void pack_layer(const float *W, int K, int N, int Np, int KB, uint8_t *img, int tid,
                           int stride) {
  const int Kp = KB * 64;
  for (int i = tid; i < Np * Kp; i += stride) {
    const int n = i / Kp, k = i % Kp;
    const float v = (n < N && k < K) ? W[(size_t)k * N + n] : 0.f;
    const int kb = k >> 6, kk = k & 63;
    const int off = kb * (Np * 128) + n * 128 + (((kk >> 3) ^ (n & 7)) << 4) + (kk & 7) * 2;
    *(uint16_t *)(img + off) = bf16_bits(v);
  }
}

__global__ void k_mlp3_tc_pack(const float *__restrict__ params, Mlp3Shape s,
                               uint8_t *__restrict__ out) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  const float *W1 = params, *b1 = W1 + (size_t)s.K0 * s.N1;
  const float *W2 = b1 + s.N1, *b2 = W2 + (size_t)s.N1 * s.N2;
  const float *W3 = b2 + s.N2, *b3 = W3 + (size_t)s.N2 * s.N3;
  pack_layer(W1, s.K0, s.N1, s.N1p, s.KB1, out + s.b1_off, tid, stride);
  pack_layer(W2, s.N1, s.N2, s.N2p, s.KB2, out + s.b2_off, tid, stride);
  pack_layer(W3, s.N2, s.N3, s.N3p, s.KB3, out + s.b3_off, tid, stride);
  float *bias = (float *)(out + s.bias_off);
  for (int i = tid; i < s.N1p + s.N2p + s.N3p; i += stride) {
    float v = 0.f;
    if (i < s.N1p) {
      v = i < s.N1 ? b1[i] : 0.f;
    } else if (i < s.N1p + s.N2p) {
      const int j = i - s.N1p;
      v = j < s.N2 ? b2[j] : 0.f;
    } else {
      const int j = i - s.N1p - s.N2p;
      v = j < s.N3 ? b3[j] : 0.f;
    }
    bias[i] = v;
  }
}

__device__ __forceinline__ void store_row_sw128(uint32_t row_addr, uint32_t swz,
                                                const uint32_t (&p)[32]) {
#pragma unroll
  for (int ch = 0; ch < 8; ++ch)
    tc::sts128(row_addr + (((uint32_t)ch ^ swz) << 4), p[ch * 4 + 0], p[ch * 4 + 1], p[ch * 4 + 2],
               p[ch * 4 + 3]);
}

// One layer's MMAs: K-blocks kb < KB from slots kb (KB <= 2), B image at bimg.
__device__ __forceinline__ void issue_layer(uint32_t tmem, uint32_t slots, uint32_t bimg, int KB,
                                            int Np, int K, uint32_t idesc) {
  for (int kb = 0; kb < KB; ++kb) {
    const int kk_n = min(4, (K - kb * 64 + 15) / 16);
    for (int kk = 0; kk < kk_n; ++kk) {
      const uint64_t da = tc::smem_desc(slots + kb * kSlot + kk * 32, 16, 1024, tc::kSwizzle128B);
      const uint64_t db = tc::smem_desc(bimg + kb * (Np * 128) + kk * 32, 16, 1024,
                                        tc::kSwizzle128B);
      tc::mma_bf16(tmem, da, db, idesc, (kb | kk) != 0);
    }
  }
}

// tanh(acc + bias) of accumulator columns [c0, c0 + 64) as 32 packed bf16x2.
__device__ __forceinline__ void act_block(uint32_t taddr, const float *bias, int c0, int Np,
                                          uint32_t (&hp)[32]) {
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    const int cb = c0 + half * 32;
    uint32_t z[32];
    if (cb < Np) {
      tc::tmem_ld32(taddr + (uint32_t)cb, z);
      tc::tmem_wait_ld();
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int c = cb + 2 * i;
      uint32_t q = 0u;
      if (c < Np)
        q = tc::tanh_bf16x2(tc::pack_bf16x2(__uint_as_float(z[2 * i]) + bias[c],
                                            __uint_as_float(z[2 * i + 1]) + bias[c + 1]));
      hp[half * 16 + i] = q;
    }
  }
}

__global__ void __launch_bounds__(kThreads, 1)
    k_mlp3_tc(const float *__restrict__ X, long ldr, long ldc, const uint8_t *__restrict__ packed,
              Mlp3Shape s, float *__restrict__ out, long M, uint32_t *err) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = tc::smem_u32(smem_raw);
  uint8_t *sm = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
  const uint32_t sb = tc::smem_u32(sm);
  const int tid = threadIdx.x, wg = tid >> 7, r = tid & 127, warp = tid >> 5;
  const int off_slots = s.bytes;
  const int off_bar = off_slots + kWG * 2 * kSlot;
  uint64_t *bar = (uint64_t *)(sm + off_bar) + wg * 2;  // [layer done, drain]
  uint32_t *tm_holder = (uint32_t *)(sm + off_bar + kWG * 2 * 8);
  {
    const uint4 *src = (const uint4 *)packed;
    uint4 *dst = (uint4 *)sm;
    for (int i = tid; i < s.bytes / 16; i += kThreads) dst[i] = __ldg(src + i);
  }
  if (tid == 0) {
    uint64_t *all = (uint64_t *)(sm + off_bar);
    for (int i = 0; i < kWG * 2; ++i) tc::mbar_init(all + i, 1);
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
  const uint32_t slots = sb + off_slots + (uint32_t)wg * 2 * kSlot;
  const uint32_t swz = (uint32_t)(r & 7);
  const uint32_t my_row = (uint32_t)r * 128u;
  const float *bias1 = (const float *)(sm + s.bias_off);
  const float *bias2 = bias1 + s.N1p;
  const float *bias3 = bias2 + s.N2p;
  const uint32_t id1 = tc::idesc_bf16_f32(128, (uint32_t)s.N1p);
  const uint32_t id2 = tc::idesc_bf16_f32(128, (uint32_t)s.N2p);
  const uint32_t id3 = tc::idesc_bf16_f32(128, (uint32_t)s.N3p);
  uint32_t ph = 0u;
  bool ok = true;
  const long n_tiles = (M + kTile - 1) / kTile;

  for (long tile = (long)blockIdx.x + (long)wg * gridDim.x; ok && tile < n_tiles;
       tile += (long)gridDim.x * kWG) {
    const long row = tile * kTile + r;
    const bool valid = row < M;
    // ---- layer-1 operand from X (FP32, any stride), at most two K-blocks
    for (int kb = 0; kb < s.KB1; ++kb) {
      uint32_t p[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const int k = kb * 64 + 2 * i;
        const float lo = (valid && k < s.K0) ? __ldg(X + row * ldr + (long)k * ldc) : 0.f;
        const float hi = (valid && k + 1 < s.K0) ? __ldg(X + row * ldr + (long)(k + 1) * ldc) : 0.f;
        p[i] = tc::pack_bf16x2(lo, hi);
      }
      store_row_sw128(slots + (uint32_t)kb * kSlot + my_row, swz, p);
    }
    // ---- three layers: MMA, then bias + tanh into the next layer's slots
    for (int l = 0; l < 3; ++l) {
      tc::fence_async_smem();
      tc::fence_before_sync();
      tc::wg_sync(bar_id);
      if (r == 0) {
        tc::fence_after_sync();
        if (l == 0) issue_layer(tmem, slots, sb + s.b1_off, s.KB1, s.N1p, s.K0, id1);
        if (l == 1) issue_layer(tmem, slots, sb + s.b2_off, s.KB2, s.N2p, s.N1, id2);
        if (l == 2) issue_layer(tmem, slots, sb + s.b3_off, s.KB3, s.N3p, s.N2, id3);
        tc::mma_commit(bar);
      }
      ok = tc::wg_all(bar_id, tc::mbar_wait(bar, ph, kWaitNs));
      ph ^= 1u;
      if (!ok) break;
      tc::fence_after_sync();
      if (l < 2) {
        const int Np = l == 0 ? s.N1p : s.N2p;
        const float *bias = l == 0 ? bias1 : bias2;
        const int KBn = l == 0 ? s.KB2 : s.KB3;
        for (int kb = 0; kb < KBn; ++kb) {
          uint32_t hp[32];
          act_block(tmem + lane, bias, kb * 64, Np, hp);
          store_row_sw128(slots + (uint32_t)kb * kSlot + my_row, swz, hp);
        }
      } else {
        // logits: acc + b3, FP32 row-major [M][N3]
        for (int c0 = 0; c0 < s.N3p; c0 += 16) {
          uint32_t z[16];
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
              "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
              : "=r"(z[0]), "=r"(z[1]), "=r"(z[2]), "=r"(z[3]), "=r"(z[4]), "=r"(z[5]),
                "=r"(z[6]), "=r"(z[7]), "=r"(z[8]), "=r"(z[9]), "=r"(z[10]), "=r"(z[11]),
                "=r"(z[12]), "=r"(z[13]), "=r"(z[14]), "=r"(z[15])
              : "r"(tmem + lane + (uint32_t)c0));
          tc::tmem_wait_ld();
          if (valid) {
#pragma unroll
            for (int i = 0; i < 16; ++i)
              if (c0 + i < s.N3) out[row * s.N3 + c0 + i] = __uint_as_float(z[i]) + bias3[c0 + i];
          }
        }
        tc::fence_before_sync();  // TMEM reads precede the next tile's MMAs
      }
    }
  }
  if (!ok && r == 0) {
    tc::mma_commit(bar + 1);
    tc::mbar_wait(bar + 1, 0, kWaitNs);
    atomicExch(err, 1u);
    atomicExch(err + 1, 400u);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(*tm_holder, kTmemCols);
  }
}

}  // namespace

bool mlp3_tc_supported(const PolicyShape &p) {
  const Mlp3Shape s = mlp3_shape(p);
  return s.K0 >= 1 && s.K0 <= 128 && s.N1 <= 128 && s.N2 <= 128 && s.N3p <= 256 &&
         smem_of(s) <= 232448;
}

size_t mlp3_tc_packed_bytes(const PolicyShape &p) { return (size_t)mlp3_shape(p).bytes; }

void launch_mlp3_tc_pack(const float *params, const PolicyShape &p, void *packed, cudaStream_t st) {
  k_mlp3_tc_pack<<<64, 256, 0, st>>>(params, mlp3_shape(p), (uint8_t *)packed);
}

void mlp3_tc_init() {
  cudaFuncSetAttribute(k_mlp3_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
}

void launch_mlp3_tc(const float *X, long ldr, long ldc, const void *packed, const PolicyShape &p,
                    float *out, long M, uint32_t *err, cudaStream_t st) {
  if (M <= 0) return;
  const Mlp3Shape s = mlp3_shape(p);
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long tiles = (M + kTile - 1) / kTile;
  const long grid = tiles < sms ? tiles : sms;
  size_t smem = smem_of(s);
  if (smem < 120 * 1024) smem = 120 * 1024;  // one CTA per SM: 512 TMEM columns uncontended
  k_mlp3_tc<<<(unsigned)grid, kThreads, smem, st>>>(X, ldr, ldc, (const uint8_t *)packed, s, out,
                                                    M, err);
}

}  // namespace ws
