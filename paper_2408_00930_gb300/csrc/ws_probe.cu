// ws_probe.cu -- throughput probes of the arithmetic units the roll-out kernels
// lean on (the SFU's tanh / ex2 / rcp / sin and the FMA pipe), in results per
// clock per SM.  The rooflines of the fused kernels divide by these rates; the
// half-warp tanh probe tells whether idle lanes shorten an SFU instruction.
//
// Every thread runs 8 independent chains of the probed operation for `iters`
// rounds; the grid holds 4 blocks of 256 threads per SM (32 warps, so that
// latency is hidden and only throughput is measured).  Each block brackets its
// loop with clock64 reads between block barriers; the rate of an SM is the work
// of its blocks over the longest block span.
#include <vector>

#include "ws_kernels.cuh"

namespace ws {

namespace {

constexpr int kProbeThreads = 256, kProbeBlocksPerSm = 4, kChains = 8;

template <int op>
__device__ __forceinline__ float probe_op(float v) {
  float y = v;
  switch (op) {
    case WS_PROBE_TANH_F32:
      asm volatile("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(v));
      break;
    case WS_PROBE_EX2_F32:  // -2^v keeps the chain in [-1, -1/2]
      asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(v));
      y = -y;
      break;
    case WS_PROBE_RCP_F32:  // 1 / (v + 1): an add on the FMA pipe keeps the chain from folding
      asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(__fadd_rn(v, 1.0f)));
      break;
    case WS_PROBE_LG2_F32:  // -log2(-v) of v in [-1, -1/2] stays in (0, 1]; negated
      asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-v));
      y = -0.5f - 0.25f * y;
      break;
    case WS_PROBE_RSQRT_F32:
      asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(__fadd_rn(v, 2.0f)));
      break;
    case WS_PROBE_SIN_F32:
      asm volatile("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(v));
      break;
    case WS_PROBE_FMA_F32:
      y = __fmaf_rn(v, 0.999f, 1e-3f);
      break;
    default:
      break;
  }
  return y;
}

// Packed forms: two results per lane per instruction.
template <int op>
__device__ __forceinline__ uint32_t probe_op2(uint32_t v) {
  uint32_t y = v;
  switch (op) {
    case WS_PROBE_TANH_BF16X2:
      asm volatile("tanh.approx.bf16x2 %0, %1;" : "=r"(y) : "r"(v));
      break;
    case WS_PROBE_EX2_BF16X2:  // sign flip of both halves keeps the chain bounded
      asm volatile("ex2.approx.ftz.bf16x2 %0, %1;" : "=r"(y) : "r"(v));
      y ^= 0x80008000u;
      break;
    case WS_PROBE_EX2_F16X2:
      asm volatile("ex2.approx.f16x2 %0, %1;" : "=r"(y) : "r"(v));
      y ^= 0x80008000u;
      break;
    default:
      break;
  }
  return y;
}

template <int op>
__global__ void __launch_bounds__(kProbeThreads) k_probe(uint32_t iters, unsigned long long *cycles) {
  constexpr bool packed = op == WS_PROBE_TANH_BF16X2 || op == WS_PROBE_EX2_BF16X2 ||
                      op == WS_PROBE_EX2_F16X2 || op == WS_PROBE_FMA_F32X2;
  float v[kChains];
  uint32_t w[kChains];
  uint64_t q[kChains];
  uint64_t qa, qc;
  asm("mov.b64 %0, {%1, %2};" : "=l"(qa) : "f"(0.999f), "f"(0.999f));
  asm("mov.b64 %0, {%1, %2};" : "=l"(qc) : "f"(1e-3f), "f"(1e-3f));
#pragma unroll
  for (int j = 0; j < kChains; ++j) {
    v[j] = -0.25f - 0.03125f * (float)((threadIdx.x + j) & 7);
    w[j] = 0xBE80BE80u + (uint32_t)j;  // two negative halves
    asm("mov.b64 %0, {%1, %2};" : "=l"(q[j]) : "f"(v[j]), "f"(-v[j]));
  }
  __syncthreads();
  const unsigned long long t0 = clock64();
  if constexpr (op == WS_PROBE_FMA_F32X2) {
    for (uint32_t i = 0; i < iters; ++i)
#pragma unroll
      for (int j = 0; j < kChains; ++j)
        asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(q[j]) : "l"(qa), "l"(qc));
  } else if constexpr (packed) {
    for (uint32_t i = 0; i < iters; ++i)
#pragma unroll
      for (int j = 0; j < kChains; ++j) w[j] = probe_op2<op>(w[j]);
  } else if constexpr (op == WS_PROBE_TANH_F32_HALF) {
    if ((threadIdx.x & 31) < 16)
      for (uint32_t i = 0; i < iters; ++i)
#pragma unroll
        for (int j = 0; j < kChains; ++j) v[j] = probe_op<WS_PROBE_TANH_F32>(v[j]);
    __syncwarp();
  } else {
    for (uint32_t i = 0; i < iters; ++i)
#pragma unroll
      for (int j = 0; j < kChains; ++j) v[j] = probe_op<op>(v[j]);
  }
  __syncthreads();
  const unsigned long long t1 = clock64();
  float acc = 0.f;
  uint32_t accw = 0u;
#pragma unroll
  for (int j = 0; j < kChains; ++j) {
    acc += v[j];
    accw ^= w[j] ^ (uint32_t)q[j] ^ (uint32_t)(q[j] >> 32);
  }
  // keep the chains live: the slot is overwritten with the span below
  if (threadIdx.x == 0) {
    cycles[2 * blockIdx.x + 1] = (unsigned long long)__float_as_uint(acc) ^ accw;
    cycles[2 * blockIdx.x] = t1 - t0;
  }
}

template <int op>
void launch_probe(int grid, uint32_t iters, unsigned long long *cyc, cudaStream_t st) {
  k_probe<op><<<grid, kProbeThreads, 0, st>>>(iters, cyc);
}

}  // namespace

}  // namespace ws

extern "C" ws_status ws_probe_rate(int op, uint32_t iters, void *dev_buf, size_t buf_bytes,
                                   double *per_clk_per_sm, void *cuda_stream) {
  using namespace ws;
  if (!per_clk_per_sm || !dev_buf || iters == 0 || op < 0 || op >= WS_PROBE_COUNT)
    return WS_ERR_INVALID;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
    return WS_ERR_CUDA;
  const int grid = sms * kProbeBlocksPerSm;
  if (buf_bytes < (size_t)grid * 16) return WS_ERR_NOMEM;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  unsigned long long *cyc = (unsigned long long *)dev_buf;
  switch (op) {
    case WS_PROBE_TANH_F32: launch_probe<WS_PROBE_TANH_F32>(grid, iters, cyc, st); break;
    case WS_PROBE_TANH_BF16X2: launch_probe<WS_PROBE_TANH_BF16X2>(grid, iters, cyc, st); break;
    case WS_PROBE_EX2_F32: launch_probe<WS_PROBE_EX2_F32>(grid, iters, cyc, st); break;
    case WS_PROBE_EX2_BF16X2: launch_probe<WS_PROBE_EX2_BF16X2>(grid, iters, cyc, st); break;
    case WS_PROBE_EX2_F16X2: launch_probe<WS_PROBE_EX2_F16X2>(grid, iters, cyc, st); break;
    case WS_PROBE_RCP_F32: launch_probe<WS_PROBE_RCP_F32>(grid, iters, cyc, st); break;
    case WS_PROBE_SIN_F32: launch_probe<WS_PROBE_SIN_F32>(grid, iters, cyc, st); break;
    case WS_PROBE_LG2_F32: launch_probe<WS_PROBE_LG2_F32>(grid, iters, cyc, st); break;
    case WS_PROBE_RSQRT_F32: launch_probe<WS_PROBE_RSQRT_F32>(grid, iters, cyc, st); break;
    case WS_PROBE_FMA_F32: launch_probe<WS_PROBE_FMA_F32>(grid, iters, cyc, st); break;
    case WS_PROBE_TANH_F32_HALF: launch_probe<WS_PROBE_TANH_F32_HALF>(grid, iters, cyc, st); break;
    default: launch_probe<WS_PROBE_FMA_F32X2>(grid, iters, cyc, st); break;
  }
  std::vector<unsigned long long> h((size_t)grid * 2);
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(h.data(), cyc, h.size() * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return WS_ERR_CUDA;
  unsigned long long span = 0;
  for (int b = 0; b < grid; ++b) span = h[2 * (size_t)b] > span ? h[2 * (size_t)b] : span;
  if (span == 0) return WS_ERR_CUDA;
  const bool packed = op == WS_PROBE_TANH_BF16X2 || op == WS_PROBE_EX2_BF16X2 ||
                      op == WS_PROBE_EX2_F16X2 || op == WS_PROBE_FMA_F32X2;
  const double per_sm = (double)kProbeBlocksPerSm * kProbeThreads * kChains * (double)iters *
                        (packed ? 2.0 : 1.0) * (op == WS_PROBE_TANH_F32_HALF ? 0.5 : 1.0);
  *per_clk_per_sm = per_sm / (double)span;
  return WS_OK;
}
