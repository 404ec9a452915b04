// ws_gemm_tc.cu -- FP32-accurate GEMMs of the actor-critic update on the
// tensor cores (tcgen05).
//
// Paper grounding: Sec. 2 and App. B keep training on the GPU, fed in place by
// the roll-out store; the update's three hidden-by-hidden products per network
// (the forward of layer 2, its data gradient, its weight gradient) are its
// dense part.  The update keeps FP32 semantics: every FP32 operand is split
// into two BF16 parts, x = x_hi + x_lo (x_hi = bf16(x), x_lo = bf16(x - x_hi)),
// and a product takes the three terms x_hi y_hi + x_hi y_lo + x_lo y_hi into
// one FP32 accumulator in tensor memory.  The dropped x_lo y_lo and the split's
// rounding leave about 2^-16 of |x y| per product, below the FP32 rounding of a
// long sum.
//
// A CTA computes one 128 x 128 tile C[m0.., n0..] = epi(sum_k A(m, k) B(k, n))
// over its K range, in chunks of 32: its 256 threads hold a chunk of A and of
// B in registers (loaded from global memory in either orientation,
// "k-contiguous" X[i ld + k] or "i-contiguous" X[k ld + i], coalesced either
// way), split it into BF16 hi / lo tiles in shared memory (K-major, 8 x 16-byte
// core matrices, no swizzle) and load the next chunk, while thread 0 issues six
// MMAs (two K = 16 steps x three terms) and commits them to the chunk's stage
// barrier; two stages.  The epilogue reads the accumulator rows from tensor
// memory (warps w and w + 4 take the lanes of quarter w, half the columns
// each) into shared memory, then each warp takes whole rows:
// bias + tanh, bias, or the tanh derivative of the layer below, and C (or a
// row-slice partial at z x slice_stride) written in coalesced 512-byte rows.
// Every wait is bounded; a wait that runs out sets the error flag and the CTA
// drains its MMAs and leaves.
#include "ws_kernels.cuh"
#include "ws_tc.cuh"

namespace ws {

namespace {

constexpr int kTM = 128, kTN = 128, kBK = 32, kNS = 2, kThreads = 256;
constexpr int kItems = kTM * (kBK / 8) / kThreads;  // (row, 8 k) items per thread per operand
constexpr int kTileBytes = kTM * kBK * 2;      // one BF16 operand tile, 8 KB
constexpr int kStageBytes = 4 * kTileBytes;    // A hi | A lo | B hi | B lo
constexpr int kCP = kTN + 4;                   // row stride (floats) of the output tile
constexpr int kOutBytes = kTM * kCP * 4;       // the output tile, over the stages once done
constexpr int kBarOff = kOutBytes > kNS * kStageBytes ? kOutBytes : kNS * kStageBytes;
constexpr int kSmem = kBarOff + 64 + 1024;
constexpr uint32_t kTmemCols = kTN;

// The 16-byte chunk of tile row `row`, K group kg (8 consecutive k), in the
// K-major core-matrix layout: 8-row groups kBK x 16 bytes apart, K groups 128
// bytes apart.
__device__ __forceinline__ uint32_t chunk_off(int row, int kg) {
  return (uint32_t)((row >> 3) * (kBK * 16) + kg * 128 + (row & 7) * 16);
}

// Eight consecutive k of operand row (or column) i, zero outside i < imax, k < kmax.
// KCONT: X[i ld + k] (contiguous along k); else X[k ld + i].
template <bool KCONT>
__device__ __forceinline__ void load8(const float *__restrict__ X, long ld, int i, int k, int imax,
                                      int kmax, bool vec, float (&v)[8]) {
  if (KCONT) {
    const float *p = X + (long)i * ld + k;
    if (vec && i < imax && k + 7 < kmax) {
      const float4 a = __ldg((const float4 *)p), b = __ldg((const float4 *)(p + 4));
      v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
      v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = (i < imax && k + j < kmax) ? __ldg(p + j) : 0.f;
    }
  } else {
#pragma unroll
    for (int j = 0; j < 8; ++j)
      v[j] = (i < imax && k + j < kmax) ? __ldg(X + (long)(k + j) * ld + i) : 0.f;
  }
}

// Split eight FP32 values into BF16 hi and lo chunks and store both.
__device__ __forceinline__ void store_split(uint32_t hi_addr, uint32_t lo_addr, const float (&v)[8]) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    h[j] = tc::pack_bf16x2(v[2 * j], v[2 * j + 1]);
    l[j] = tc::pack_bf16x2(v[2 * j] - tc::bf16_lo(h[j]), v[2 * j + 1] - tc::bf16_hi(h[j]));
  }
  tc::sts128(hi_addr, h[0], h[1], h[2], h[3]);
  tc::sts128(lo_addr, l[0], l[1], l[2], l[3]);
}

// One operand's chunk (128 rows x 32 k) in kItems items of (row, 8 k) per
// thread: the lanes of a warp cover 8 rows x 4 K groups of a k-contiguous
// operand and 32 consecutive rows of the other orientation, so both load
// whole 128-byte lines.  Loaded into registers one chunk ahead, then split
// into the hi / lo tiles.
template <bool KCONT>
__device__ __forceinline__ void item_pos(int it, int &row, int &kg) {
  const int q = it * kThreads + (int)threadIdx.x;
  row = KCONT ? q >> 2 : q & 127;
  kg = KCONT ? q & 3 : q >> 7;
}
template <bool KCONT>
__device__ __forceinline__ void load_chunk(const float *__restrict__ X, long ld, int i0, int imax,
                                           int k0, int kmax, bool vec, float (&v)[kItems][8]) {
#pragma unroll
  for (int it = 0; it < kItems; ++it) {
    int row, kg;
    item_pos<KCONT>(it, row, kg);
    load8<KCONT>(X, ld, i0 + row, k0 + kg * 8, imax, kmax, vec, v[it]);
  }
}
template <bool KCONT>
__device__ __forceinline__ void store_chunk(const float (&v)[kItems][8], uint32_t hi, uint32_t lo) {
#pragma unroll
  for (int it = 0; it < kItems; ++it) {
    int row, kg;
    item_pos<KCONT>(it, row, kg);
    const uint32_t off = chunk_off(row, kg);
    store_split(hi + off, lo + off, v[it]);
  }
}

// C tile (m0, n0) of epi(A B): A(m, k) = A[m lda + k] (TA: A[k lda + m]),
// B(k, n) = B[k ldb + n] (TB: B[n ldb + k]); k over [k_lo, k_hi), or with
// k_slice > 0 over slice blockIdx.z of it, written at C + z slice_stride.
template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(kThreads)
    k_gemm_tc(const float *__restrict__ A, int lda, const float *__restrict__ B, int ldb,
              float *__restrict__ C, int M, int N, int k_lo, int k_hi, int k_slice,
              size_t slice_stride, const float *__restrict__ aux, int vec_a, int vec_b,
              uint32_t *err) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = tc::smem_u32(smem_raw);
  uint8_t *sm = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
  const uint32_t sb = tc::smem_u32(sm);
  uint64_t *bars = (uint64_t *)(sm + kBarOff);  // [kNS] stage barriers, drain
  uint32_t *tm_holder = (uint32_t *)(sm + kBarOff + 32);
  const int tid = threadIdx.x, warp = tid >> 5;
  // the N tiles of one M tile are consecutive blocks, so that they run together
  // and the second reads A from L2
  const int n0 = blockIdx.x * kTN, m0 = blockIdx.y * kTM;
  int kb = k_lo, ke = k_hi;
  if (k_slice > 0) {
    kb = k_lo + (int)blockIdx.z * k_slice;
    ke = min(k_hi, kb + k_slice);
  }
  const int nk = ke > kb ? (ke - kb + kBK - 1) / kBK : 0;
  if (tid == 0) {
    for (int s = 0; s <= kNS; ++s) tc::mbar_init(bars + s, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tc::tmem_alloc(tm_holder, kTmemCols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tm_holder;
  constexpr uint32_t idesc = tc::idesc_bf16_f32(kTM, kTN);

  bool ok = true;
  float va[kItems][8], vb[kItems][8];
  if (nk > 0) {
    load_chunk<!TA>(A, lda, m0, M, kb, ke, vec_a != 0, va);
    load_chunk<TB>(B, ldb, n0, N, kb, ke, vec_b != 0, vb);
  }
  for (int c = 0; c < nk && ok; ++c) {
    const int s = c % kNS;
    if (c >= kNS && !tc::mbar_wait(bars + s, (uint32_t)((c / kNS - 1) & 1), tc::kDrainNs)) ok = false;
    ok = __syncthreads_and(ok);
    if (!ok) break;
    const uint32_t st = sb + (uint32_t)(s * kStageBytes);
    store_chunk<!TA>(va, st, st + kTileBytes);
    store_chunk<TB>(vb, st + 2 * kTileBytes, st + 3 * kTileBytes);
    if (c + 1 < nk) {  // the next chunk's loads run under this chunk's MMAs
      const int k1 = kb + (c + 1) * kBK;
      load_chunk<!TA>(A, lda, m0, M, k1, ke, vec_a != 0, va);
      load_chunk<TB>(B, ldb, n0, N, k1, ke, vec_b != 0, vb);
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
#pragma unroll
      for (int q = 0; q < kBK / 16; ++q) {
        const uint32_t o = (uint32_t)(q * 256);
        const uint64_t ahi = tc::smem_desc(st + o, 128, kBK * 16, tc::kSwizzleNone);
        const uint64_t alo = tc::smem_desc(st + kTileBytes + o, 128, kBK * 16, tc::kSwizzleNone);
        const uint64_t bhi = tc::smem_desc(st + 2 * kTileBytes + o, 128, kBK * 16, tc::kSwizzleNone);
        const uint64_t blo = tc::smem_desc(st + 3 * kTileBytes + o, 128, kBK * 16, tc::kSwizzleNone);
        tc::mma_bf16(tmem, ahi, bhi, idesc, c > 0 || q > 0);
        tc::mma_bf16(tmem, ahi, blo, idesc, true);
        tc::mma_bf16(tmem, alo, bhi, idesc, true);
      }
      tc::mma_commit(bars + s);
    }
  }
  // the last chunk's commit covers every MMA of the tile
  if (ok && nk > 0 &&
      !tc::mbar_wait(bars + (nk - 1) % kNS, (uint32_t)(((nk - 1) / kNS) & 1), tc::kDrainNs))
    ok = false;
  ok = __syncthreads_and(ok);
  if (!ok) {
    if (tid == 0) {
      tc::mma_commit(bars + kNS);  // drain whatever is still in flight
      tc::mbar_wait(bars + kNS, 0, tc::kDrainNs);
      atomicExch(err, 1u);
      atomicExch(err + 1, 700u);
    }
  } else {
    // the accumulator rows through shared memory (the stages are free now), so
    // that the epilogue reads its operands and writes C in whole rows
    tc::fence_after_sync();
    float *ct = (float *)sm;
    const int r = (warp & 3) * 32 + (tid & 31);        // this thread's accumulator row
    const uint32_t lane = (uint32_t)((warp & 3) * 32) << 16;
    const int jh = (warp >> 2) * (kTN / 64);           // warps 4-7: the upper half of the columns
#pragma unroll 1
    for (int j = jh; j < jh + kTN / 64; ++j) {
      uint32_t z[32];
      if (nk > 0) {
        tc::tmem_ld32(tmem + lane + (uint32_t)(j * 32), z);
        tc::tmem_wait_ld();
      } else {
#pragma unroll
        for (int i = 0; i < 32; ++i) z[i] = 0u;  // an empty K range sums to zero
      }
#pragma unroll
      for (int i = 0; i < 32; i += 4)
        *(float4 *)(ct + r * kCP + j * 32 + i) =
            make_float4(__uint_as_float(z[i]), __uint_as_float(z[i + 1]),
                        __uint_as_float(z[i + 2]), __uint_as_float(z[i + 3]));
    }
    __syncthreads();
    float *Cz = C + (k_slice > 0 ? (size_t)blockIdx.z * slice_stride : 0);
    const int lane_id = tid & 31;
    const int n = n0 + lane_id * 4;
    const bool vec = (N & 3) == 0 && n + 3 < N;
    // the bias of this thread's four columns, the same for every row
    float bv[4] = {0.f, 0.f, 0.f, 0.f};
    if (EPI == kGemmBiasTanh || EPI == kGemmBias) {
#pragma unroll
      for (int i = 0; i < 4; ++i) bv[i] = n + i < N ? aux[n + i] : 0.f;
    }
    const bool avec = vec && ((uintptr_t)aux & 15) == 0;
    // Each warp takes rows warp, warp + 8, ... in batches of kRB, whose operand
    // loads (the layer's activations for tanh') are all issued before the first
    // is used, so that a batch waits on one memory round trip, not kRB.
    constexpr int kRB = 4, kWarps = kThreads / 32;
#pragma unroll 1
    for (int rb = warp; rb < kTM; rb += kRB * kWarps) {
      if (m0 + rb >= M) break;
      float v[kRB][4], hh[kRB][4];
#pragma unroll
      for (int u = 0; u < kRB; ++u) {
        const int rr = rb + u * kWarps, m = m0 + rr;
        const float4 a = *(const float4 *)(ct + rr * kCP + lane_id * 4);
        v[u][0] = a.x; v[u][1] = a.y; v[u][2] = a.z; v[u][3] = a.w;
        if (EPI == kGemmDTanh) {
          const float *hp = aux + (size_t)m * N + n;
          if (m < M && avec) {
            const float4 h4 = __ldg((const float4 *)hp);
            hh[u][0] = h4.x; hh[u][1] = h4.y; hh[u][2] = h4.z; hh[u][3] = h4.w;
          } else {
#pragma unroll
            for (int i = 0; i < 4; ++i) hh[u][i] = (m < M && n + i < N) ? __ldg(hp + i) : 0.f;
          }
        }
      }
#pragma unroll
      for (int u = 0; u < kRB; ++u) {
        const int m = m0 + rb + u * kWarps;
        if (m >= M) break;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          if (EPI == kGemmBiasTanh) v[u][i] = tanhf(v[u][i] + bv[i]);
          if (EPI == kGemmBias) v[u][i] = v[u][i] + bv[i];
          if (EPI == kGemmDTanh) v[u][i] = v[u][i] * (1.f - hh[u][i] * hh[u][i]);
        }
        float *o = Cz + (size_t)m * N + n;
        if (vec) {
          *(float4 *)o = make_float4(v[u][0], v[u][1], v[u][2], v[u][3]);
        } else {
#pragma unroll
          for (int i = 0; i < 4; ++i)
            if (n + i < N) o[i] = v[u][i];
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, kTmemCols);
  }
}

template <bool TA, bool TB, int EPI>
cudaError_t run_gemm(dim3 g, cudaStream_t st, const float *A, int lda, const float *B, int ldb,
                     float *C, int M, int N, int k_lo, int k_hi, int k_slice, size_t slice_stride,
                     const float *aux, uint32_t *err) {
  static bool attr_set[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !attr_set[dev]) {
    const cudaError_t e = cudaFuncSetAttribute(k_gemm_tc<TA, TB, EPI>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) attr_set[dev] = true;
  }
  // 16-byte loads along k where rows start on 16-byte boundaries
  const bool va = !TA && lda % 4 == 0 && ((uintptr_t)A & 15) == 0;
  const bool vb = TB && ldb % 4 == 0 && ((uintptr_t)B & 15) == 0;
  k_gemm_tc<TA, TB, EPI><<<g, kThreads, kSmem, st>>>(A, lda, B, ldb, C, M, N, k_lo, k_hi, k_slice,
                                                     slice_stride, aux, va, vb, err);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gemm_tc(bool ta, bool tb, int epi, const float *A, int lda, const float *B,
                           int ldb, float *C, int M, int N, int k_lo, int k_hi, int k_slice,
                           size_t slice_stride, const float *aux, uint32_t *err, cudaStream_t st) {
  const int nz = k_slice > 0 ? (k_hi - k_lo + k_slice - 1) / k_slice : 1;
  const dim3 g((unsigned)((N + kTN - 1) / kTN), (unsigned)((M + kTM - 1) / kTM), (unsigned)nz);
  if (g.y > 65535u || g.z > 65535u) return cudaErrorInvalidValue;
#define WS_GEMM_ARGS g, st, A, lda, B, ldb, C, M, N, k_lo, k_hi, k_slice, slice_stride, aux, err
  if (!ta && !tb && epi == kGemmBiasTanh) return run_gemm<false, false, kGemmBiasTanh>(WS_GEMM_ARGS);
  if (!ta && !tb && epi == kGemmBias) return run_gemm<false, false, kGemmBias>(WS_GEMM_ARGS);
  if (!ta && tb && epi == kGemmDTanh) return run_gemm<false, true, kGemmDTanh>(WS_GEMM_ARGS);
  if (ta && !tb && epi == kGemmNone) return run_gemm<true, false, kGemmNone>(WS_GEMM_ARGS);
#undef WS_GEMM_ARGS
  return cudaErrorInvalidValue;
}

}  // namespace ws
