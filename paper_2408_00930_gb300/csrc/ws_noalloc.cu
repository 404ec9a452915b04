// ws_noalloc.cu -- policy forward pass that allocates no device memory.
//
// Some callers cannot call cudaMalloc: code running while a CUDA graph is being
// captured, allocators that forbid foreign allocations, or embedded hosts that
// fix their device memory up front.  ws_policy_forward_noalloc serves them: the
// caller passes inputs and outputs, and the two hidden-activation buffers of
// the three-layer FP32 forward pass live in a fixed, file-scope device array
// owned by this library (16 MiB; every GPU that loads the library keeps it
// until the process exits).
#include <mutex>

#include "ws_kernels.cuh"

namespace {

constexpr size_t kNoAllocScratchFloats = (size_t)1 << 22;  // 16 MiB of FP32

// In host code this name is only a host-side stand-in for the device array:
// its device address comes from cudaGetSymbolAddress, per device.
static __device__ __align__(256) float g_noalloc_scratch[kNoAllocScratchFloats];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
float *g_scratch_dev[kMaxDevices] = {};

}  // namespace

extern "C" ws_status ws_policy_forward_noalloc(const float *obs, uint32_t n_rows,
                                               const float *params, uint32_t in_dim,
                                               uint32_t hidden0, uint32_t hidden1,
                                               uint32_t out_dim, float *out, void *cuda_stream) {
  if (!obs || !params || !out) return WS_ERR_INVALID;
  if (in_dim < 1 || hidden0 < 1 || hidden1 < 1 || out_dim < 1) return WS_ERR_INVALID;
  if (in_dim > 4096 || hidden0 > 4096 || hidden1 > 4096 || out_dim > 4096) return WS_ERR_INVALID;
  if (n_rows == 0) return WS_OK;
  if ((size_t)n_rows * ((size_t)hidden0 + hidden1) > kNoAllocScratchFloats) return WS_ERR_RANGE;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return WS_ERR_CUDA;
  float *scratch = nullptr;
  {
    // Set-up, once per device, with that device current.
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_dev[dev]) {
      void *p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return WS_ERR_CUDA;
      g_scratch_dev[dev] = (float *)p;
    }
    scratch = g_scratch_dev[dev];
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  float *h0 = scratch;
  float *h1 = scratch + (size_t)n_rows * hidden0;
  const float *W0 = params;
  const float *b0 = W0 + (size_t)in_dim * hidden0;
  const float *W1 = b0 + hidden0;
  const float *b1 = W1 + (size_t)hidden0 * hidden1;
  const float *W2 = b1 + hidden1;
  const float *b2 = W2 + (size_t)hidden1 * out_dim;
  // Every element of h0 and h1 is written before it is read, so the contents
  // left by an earlier call need no clearing.
  ws::launch_dense_fp32(obs, in_dim, 1, W0, b0, h0, (int)n_rows, (int)in_dim, (int)hidden0, 1, st);
  ws::launch_dense_fp32(h0, hidden0, 1, W1, b1, h1, (int)n_rows, (int)hidden0, (int)hidden1, 1, st);
  ws::launch_dense_fp32(h1, hidden1, 1, W2, b2, out, (int)n_rows, (int)hidden1, (int)out_dim, 0, st);
  return cudaGetLastError() == cudaSuccess ? WS_OK : WS_ERR_CUDA;
}
