// ws_kernels.cuh -- device view of a roll-out context and the host-side
// launchers of every kernel (defined in ws_plain.cu, ws_control_tc.cu, ...).
#pragma once

#include "ws_common.cuh"

namespace ws {

// Raw device pointers and scalars handed to every kernel by value.
struct Dev {
  int env;
  uint32_t n_envs, n_slots, n_agent_slots, ring_steps, episode_limit, dim, n_gauss;
  uint32_t n_out, n_out_planner;
  float noise_sigma, step_clip, gamma;
  float energy_target;  // landscape: done when E(x') < energy_target (-inf: off)
  uint64_t seed;        // key of the per-step draws (set by ws_reset)
  uint32_t env_base;    // global id of env 0 (the env word of every per-env draw)
  uint64_t *k;          // device step counter
  uint32_t *err;        // [0] error flag, [1] where
  const float *params, *params_planner;
  PolicyShape pol, pol_planner;
  // env state
  float *s;             // control: [4][n]; landscape: x [dim][n]
  int32_t *t;           // [n_envs]
  float *eobs;          // landscape [n]
  int64_t *wealth;      // economy [n_agent_slots]
  float *feat;          // economy [16][n_agent_slots]
  const int32_t *agent_off;  // economy [n_envs + 1]
  const int32_t *slot_env;   // economy [n_agent_slots]
  // landscape parameters and derived tables
  float *centres, *widths, *amps;  // [M][dim], [M], [M]
  float *cnorm, *coef;             // |c|^2, -log2(e) / (2 w^2)
  // plain-path scratch
  float *h0, *h1, *out, *pobs, *ph0, *ph1, *pout;
  int64_t *income;      // economy [n_agent_slots]
  float *epart;         // landscape energy partial sums [kEnergyChunks][2][n]
  uint8_t *needs_energy;  // landscape [n]
  // BF16 tensor-core policy layers (economy / landscape): packed W^T images
  int tc_mlp;
  const uint8_t *pk[2][3];  // [agent, planner][layer]
  const uint8_t *eimg;      // landscape: packed hi/lo centre image + table (BF16 energy)
  const uint8_t *limg;      // landscape, fused kernel: its energy image (blocks of 64 Gaussians)
  const uint8_t *fimg;      // landscape, fused kernel with WS_FLAG_FORCE: the force image
  int mlp3;                 // economy: whole-MLP tensor-core kernel (images in pk[pid][0])
  // economy on the fused persistent kernel: work items {first agent slot, rows,
  // first env, envs} and the work-queue counters {next item, CTAs finished}
  const int32_t *items;
  uint32_t n_items;
  uint32_t *queue;
  int dbg_logits;           // fused kernels also write each step's logits to out / pout
  // launch parameters (ws_launch): per-env kernels' block size, the BF16
  // energy kernel's Gaussian chunks per env tile
  int env_threads;
  int energy_chunks;
  int update_simt;  // the update's hidden-layer GEMMs on FP32 CUDA cores (else tcgen05)
  // limit of the fused kernels' device waits (MMA completions, the SFU token,
  // block loads, the cluster partner), in ns: a wait that runs out sets the
  // error flag (ws_sync reports it) and the kernel leaves after draining
  uint64_t wait_ns;
  // ring
  float *r_obs;
  void *r_act;
  float *r_logp, *r_rew, *r_ret, *r_energy;
  float *r_force;  // landscape FORCE field [t][D][slot] (WS_FLAG_FORCE), else null
  float *r_adv;    // ADVANTAGE field [t][slot] (WS_FLAG_TRAIN), else null
  float *r_sample; // landscape SAMPLE field [t][D][slot] (WS_FLAG_TRAIN), else null
  float *r_pout;   // POLICY_OUT field [t][n_out][slot] (WS_FLAG_DEBUG_LOGITS), else null
  uint8_t *r_done;
  int64_t *r_wealth;
};

constexpr int kEnergyChunks = 8;

// ---- S0: parameter initialisation -------------------------------------
void launch_init_policy(float *params, const PolicyShape &shape, uint64_t seed, uint32_t policy_id,
                        cudaStream_t st);
void launch_init_landscape(const Dev &d, uint64_t param_seed, cudaStream_t st);
void launch_landscape_derive(const Dev &d, cudaStream_t st);

// ---- full reset --------------------------------------------------------
void launch_reset(const Dev &d, cudaStream_t st);

// ---- plain / batched-FP32 step (one launch per sub-step) -----------------
// `aux` (with its fork/join events) lets the economy run the planner's policy
// beside the agents' as a parallel branch (also inside a captured graph).
struct Branch {
  cudaStream_t aux;
  cudaEvent_t fork, join;
};
void launch_plain_step(const Dev &d, uint32_t step_off, cudaStream_t st, const Branch *br);
void launch_advance(const Dev &d, uint32_t n, cudaStream_t st);

// ---- S7: discounted returns ----------------------------------------------
void launch_returns(const Dev &d, uint32_t n_steps, cudaStream_t st);
// ---- actor-critic updates (ws_train.cu) ---------------------------------------
constexpr int kTrainChunk = 65536;  // rows per chunk of the update
struct TrainBufs {                 // per-chunk scratch in the state buffer
  float *x, *ret;
  int32_t *act;
  float *adv, *lpo;                // PPO: held advantage, behaviour log-probability
  float *h1, *h2, *out, *c1, *c2, *vout, *d1, *d2, *part;
  double *stats;                   // policy loss, value loss, entropy, clipped rows (sums)
  float *grad;                     // actor gradient, then the critic's
};
struct TrainGroup {  // one policy and its critic, on slots [slot0, slot0 + n_slots) of every step
  float *params, *critic;
  PolicyShape pol, crit;
  uint32_t slot0, n_slots;
};
// Scratch sized for the widest policy of the context (and its critic).
size_t train_scratch_bytes(const PolicyShape &pol);
TrainBufs train_bufs(uint8_t *base, const PolicyShape &pol);
void launch_a2c_update(const Dev &d, const TrainBufs &tb, const TrainGroup *groups, int n_groups,
                       uint32_t n, float lr, float c_v, float c_e, cudaStream_t st);
// A = G - V(s) of the last n steps into the ADVANTAGE field (returns computed);
// landscape: also the behaviour samples into SAMPLE.
void launch_advantages(const Dev &d, const TrainBufs &tb, const TrainGroup *groups, int n_groups,
                       uint32_t n, cudaStream_t st);
// One PPO epoch over the last n steps.
void launch_ppo_update(const Dev &d, const TrainBufs &tb, const TrainGroup *groups, int n_groups,
                       uint32_t n, float lr, float eps, float c_v, float c_e, cudaStream_t st);

// Landscape force -grad E(x') of the last n_steps ring rows (ws_force.cu).
void launch_forces(const Dev &d, uint32_t n_steps, cudaStream_t st);

// ---- BF16 tensor-core control path -----------------------------------------
size_t control_tc_packed_bytes(const PolicyShape &shape);
bool control_tc_supported(const PolicyShape &shape);
void launch_control_tc_pack(const Dev &d, void *packed, cudaStream_t st);
cudaError_t launch_control_tc(const Dev &d, const void *packed, uint32_t n_steps, int grid,
                              cudaStream_t st);
int control_tc_default_grid(const Dev &d);

// ---- FP32-accurate tensor-core GEMM of the update (ws_gemm_tc.cu) -------------
// C = epi(A B) in 128 x 128 tiles, each FP32 operand split into BF16 hi + lo and
// the three terms hi hi + hi lo + lo hi accumulated in FP32.  A(m, k) =
// A[m lda + k] (ta: A[k lda + m]); B(k, n) = B[k ldb + n] (tb: B[n ldb + k]);
// k over [k_lo, k_hi), or with k_slice > 0 in slices written at C + z
// slice_stride.  Epilogues: bias + tanh, bias (aux = bias), tanh derivative
// of the layer below (aux = its activations [M][N]), none.  Supported:
// (!ta, !tb, bias + tanh | bias), (!ta, tb, tanh derivative), (ta, !tb, none).
enum GemmEpi { kGemmBiasTanh = 0, kGemmBias = 1, kGemmDTanh = 2, kGemmNone = 3 };
cudaError_t launch_gemm_tc(bool ta, bool tb, int epi, const float *A, int lda, const float *B,
                           int ldb, float *C, int M, int N, int k_lo, int k_hi, int k_slice,
                           size_t slice_stride, const float *aux, uint32_t *err, cudaStream_t st);

// ---- CUDA-core control path for small env counts (ws_control_cc.cu) ----------
bool control_cc_supported(const PolicyShape &shape);
bool control_cc_tile_ok(const PolicyShape &shape, int envs_per_cta, int threads_per_env);
cudaError_t launch_control_cc(const Dev &d, uint32_t n_steps, int envs_per_cta, int threads_per_env,
                              cudaStream_t st);

}  // namespace ws

namespace ws {
// ---- BF16 tensor-core dense layer (ws_dense_tc.cu) ----------------------------
size_t dense_tc_packed_bytes(int K, int N);
bool dense_tc_supported(int K, int N);
void launch_dense_tc_pack(const float *W, const float *b, int K, int N, void *packed,
                          cudaStream_t st);
cudaError_t launch_dense_tc(const void *X, long ldr, long ldc, int x_bf16, int K,
                            const void *packed, int N, void *Y, int y_bf16, int act, long M,
                            uint32_t *err, cudaStream_t st);
void dense_tc_init();

// ---- BF16 tensor-core three-layer MLP (ws_mlp3_tc.cu) ------------------------------
bool mlp3_tc_supported(const PolicyShape &p);
size_t mlp3_tc_packed_bytes(const PolicyShape &p);
void launch_mlp3_tc_pack(const float *params, const PolicyShape &p, void *packed, cudaStream_t st);
void launch_mlp3_tc(const float *X, long ldr, long ldc, const void *packed, const PolicyShape &p,
                    float *out, long M, uint32_t *err, cudaStream_t st);
void mlp3_tc_init();

// ---- fused persistent economy kernel (ws_econ_tc.cu) --------------------------------
bool econ_tc_supported(const PolicyShape &p, const PolicyShape &pp);
size_t econ_tc_packed_bytes();
int econ_tc_max_envs_per_item();
void launch_econ_tc_pack(const float *agent_params, const float *planner_params, void *packed,
                         cudaStream_t st);
void econ_tc_init();
cudaError_t launch_econ_tc(const Dev &d, const void *packed, uint32_t n_steps, int tiles, int grid,
                           cudaStream_t st);

// ---- fused persistent landscape kernel (ws_land_tc.cu) ----------------------------
bool land_tc_supported(int D, int M, const PolicyShape &p);
size_t land_tc_policy_bytes();
size_t land_tc_energy_bytes(int M);
void launch_land_tc_pack(const Dev &d, void *policy_img, void *energy_img, cudaStream_t st);
void land_tc_init();
// Force of recorded transitions on the tensor cores over the fused kernel's
// energy image and a force image packed beside it (ws_land_tc.cu).
size_t force_tc_bytes(int M);
void launch_force_tc_pack(const Dev &d, const void *energy_img, void *force_img, cudaStream_t st);
cudaError_t launch_force_tc(const Dev &d, const void *energy_img, const void *force_img,
                            uint32_t n_steps, cudaStream_t st);
cudaError_t launch_land_tc(const Dev &d, const void *policy_img, const void *energy_img,
                           uint32_t n_steps, int tile_ctas, cudaStream_t st);

// ---- BF16 tensor-core landscape energy (ws_energy_tc.cu) -------------------------
size_t energy_tc_bytes(int D, int M);
bool energy_tc_supported(int D, int M);
void launch_energy_tc_pack(const Dev &d, void *buf, cudaStream_t st);
void launch_energy_tc(const Dev &d, const void *buf, uint32_t off, int mode, cudaStream_t st);
void energy_tc_init(int M);
bool energy_tc_chunks_ok(int M, int chunks);

// Y[M][N] = act(X W + b) with the plain path's FP32 dense kernel (X row-major
// when ldc == 1, or addressed X[r * ldr + c * ldc]).
void launch_dense_fp32(const float *X, long ldr, long ldc, const float *W, const float *b, float *Y,
                       int M, int K, int N, int act, cudaStream_t st);
}  // namespace ws
