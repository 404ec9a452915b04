// ws_force.cu -- the landscape force F = -grad E(x') of recorded transitions
// (FP32 SIMT path).
//
// Paper grounding: App. C builds the catalytic-reaction environment on a
// first-principles potential energy landscape of the atomic positions; the
// force on the atoms is the negative gradient of that energy.  For the
// Gaussian-sum stand-in E(x) = sum_m a_m exp(-|x - c_m|^2 / (2 w_m^2)),
//   F(x) = -grad E(x) = sum_m a_m e_m (x - c_m) / w_m^2,  e_m = exp(-|x - c_m|^2 / (2 w_m^2)).
// ws_forces evaluates it at the post-step state x' = x + dx of the last n
// steps, both recorded in the ring (obs and action), and writes the FORCE
// field [t][D][slot].  It is a scan over the ring like the returns: the roll-out
// kernels are unchanged and pay nothing when forces are not asked for.
//
// This file holds the FP32 kernel (plain and batched-FP32 paths, and the BF16
// path where the tensor-core kernel of ws_land_tc.cu does not apply, i.e.
// without the fused roll-out kernel's energy image): one thread per (step,
// env) row, the direct difference form in registers, Gaussians staged through
// shared memory 64 at a time; each tile's partial sums are added to the running
// sum once per tile (pairwise-style grouping keeps the FP32 error near 64 + M/64
// roundings rather than M).
#include "ws_kernels.cuh"

namespace ws {

namespace {

constexpr int kFT = 128;     // rows (step, env) per block
constexpr int kFTileM = 64;  // Gaussians staged per tile

template <int DM>
__global__ __launch_bounds__(kFT) void k_force_f32(Dev d, uint32_t n) {
  extern __shared__ float sm[];
  const int D = (int)d.dim;
  float *cs = sm;                          // [kFTileM][D] centres
  float *ps = cs + (size_t)kFTileM * D;    // [kFTileM] a_m / w_m^2
  float *qs = ps + kFTileM;                // [kFTileM] 1 / (2 w_m^2)
  const size_t N = d.n_envs, S = d.n_slots;
  const size_t q = (size_t)blockIdx.x * kFT + threadIdx.x;
  const bool valid = q < (size_t)n * N;
  const uint32_t i = valid ? (uint32_t)(q / N) : 0u;
  const uint32_t e = valid ? (uint32_t)(q % N) : 0u;
  const uint64_t k = d.k[0] - n + i;  // step of this row
  const size_t rowR = (size_t)(k % d.ring_steps);
  const float *obs = d.r_obs + rowR * D * S + e;
  const float *act = (const float *)d.r_act + rowR * D * S + e;
  float y[DM], F[DM];
#pragma unroll
  for (int j = 0; j < DM; ++j) {
    // x' = x + dx in FP32, as the step computed it
    y[j] = (valid && j < D) ? obs[(size_t)j * S] + act[(size_t)j * S] : 0.f;
    F[j] = 0.f;
  }
  const int M = (int)d.n_gauss;
  for (int m0 = 0; m0 < M; m0 += kFTileM) {
    const int nt = min(kFTileM, M - m0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < nt * D; idx += kFT) cs[idx] = d.centres[(size_t)m0 * D + idx];
    for (int idx = threadIdx.x; idx < nt; idx += kFT) {
      const float w = d.widths[m0 + idx];
      const float iw2 = 1.0f / (w * w);
      ps[idx] = d.amps[m0 + idx] * iw2;
      qs[idx] = 0.5f * iw2;
    }
    __syncthreads();
    float T[DM];
#pragma unroll
    for (int j = 0; j < DM; ++j) T[j] = 0.f;
    for (int m = 0; m < nt; ++m) {
      const float *c = cs + m * D;
      float dd[DM];
      float d2[4] = {0.f, 0.f, 0.f, 0.f};  // four chains, summed in a fixed order
#pragma unroll
      for (int j = 0; j < DM; ++j) {
        dd[j] = j < D ? y[j] - c[j] : 0.f;
        d2[j & 3] = fmaf(dd[j], dd[j], d2[j & 3]);
      }
      const float p = ps[m] * expf(-((d2[0] + d2[1]) + (d2[2] + d2[3])) * qs[m]);
#pragma unroll
      for (int j = 0; j < DM; ++j) T[j] = fmaf(p, dd[j], T[j]);
    }
#pragma unroll
    for (int j = 0; j < DM; ++j) F[j] += T[j];
  }
  if (!valid) return;
  float *out = d.r_force + rowR * D * S + e;
#pragma unroll
  for (int j = 0; j < DM; ++j)
    if (j < D) out[(size_t)j * S] = F[j];
}

template <int DM>
void launch_f32(const Dev &d, uint32_t n, cudaStream_t st) {
  const size_t rows = (size_t)n * d.n_envs;
  const size_t smem = sizeof(float) * ((size_t)kFTileM * d.dim + 2 * kFTileM);
  k_force_f32<DM><<<(unsigned)((rows + kFT - 1) / kFT), kFT, smem, st>>>(d, n);
}

}  // namespace

void launch_forces(const Dev &d, uint32_t n_steps, cudaStream_t st) {
  if (n_steps == 0) return;
  if (d.fimg) {  // BF16 path with the fused kernel's energy image: tensor cores
    launch_force_tc(d, d.limg, d.fimg, n_steps, st);
    return;
  }
  if (d.dim <= 8)
    launch_f32<8>(d, n_steps, st);
  else if (d.dim <= 16)
    launch_f32<16>(d, n_steps, st);
  else if (d.dim <= 24)
    launch_f32<24>(d, n_steps, st);
  else if (d.dim <= 32)
    launch_f32<32>(d, n_steps, st);
  else
    launch_f32<64>(d, n_steps, st);
}

}  // namespace ws
