/*
 * warpsci.h -- C ABI of the GB300-native in-place RL roll-out engine.
 *
 * The engine runs the whole roll-out loop of the paper on one GPU with no
 * host round-trip (paper Sec. 2: "the entire RL workflow on a single or
 * multiple GPUs, utilizing a unified and in-place data store within GPUs for
 * simulation roll-outs"; App. B: roll-outs, action inference and reset share
 * one GPU-resident store, policy models live in global memory and are
 * referenced, not copied).  Each step observes the env state, runs the policy
 * MLP, samples an action, steps the environment (state update, reward, done,
 * auto-reset) and writes the transition into a time-major trajectory ring.
 *
 * Conventions for every entry point:
 *   - Nothing is thrown across the ABI; every call returns a ws_status.  The
 *     first error is sticky in the context (later calls return it again) and
 *     ws_last_error() gives a one-line message.
 *   - Device memory and the CUDA stream belong to the caller; the context
 *     borrows them from ws_create until ws_destroy.  Host arrays passed in are
 *     copied before the call returns.
 *   - Every call is asynchronous on the context's stream, except
 *     ws_query_bytes, ws_sync, ws_last_error and ws_destroy.
 *   - Step counter k: the number of steps run since the last ws_reset.  It is
 *     the first Philox counter word of every per-step random draw and selects
 *     the ring row (k mod ring_steps).
 *
 * Random streams (all Philox4x32-10, Salmon et al. SC'11): key = seed,
 * counter = (k, env, agent, tag << 24 | sub); tags ACTION 0, RESET 1,
 * PARTNER 2, NOISE 3, POLICY_INIT 4, LANDSCAPE_INIT 5, ECON_INIT 6.
 */
#ifndef WARPSCI_H
#define WARPSCI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define WS_ABI_VERSION 1u

typedef struct ws_ctx ws_ctx;

typedef enum {
  WS_OK = 0,
  WS_ERR_INVALID = 1,     /* bad argument or configuration                  */
  WS_ERR_NOMEM = 2,       /* a buffer is smaller than ws_query_bytes asks   */
  WS_ERR_CUDA = 3,        /* a CUDA call or a kernel failed, or a bounds-
                             check canary was overwritten (ws_sync)         */
  WS_ERR_TIMEOUT = 4,     /* ws_sync gave up, or a device wait ran out      */
  WS_ERR_STATE = 5,       /* call not valid in the context's current state  */
  WS_ERR_RANGE = 6,       /* requested steps are not (or no longer) in ring */
  WS_ERR_UNSUPPORTED = 7  /* env/path/size combination not built            */
} ws_status;

/* Environment families (paper App. C: classic control, multi-agent
 * economics, catalytic reaction paths on an energy landscape).  ACROBOT is the
 * second classic-control benchmark: the two-link acrobot of Sutton & Barto
 * (book dynamics, one RK4 step of 0.2 s per env step, torque a - 1 for action
 * a in {0, 1, 2}, done when the tip rises more than one link above the pivot
 * or at the episode limit, reward -1 per step and 0 on the terminal step). */
typedef enum {
  WS_ENV_CONTROL = 0,
  WS_ENV_ECONOMY = 1,
  WS_ENV_LANDSCAPE = 2,
  WS_ENV_ACROBOT = 3
} ws_env;

/* Execution paths.  PLAIN_FP32: one kernel launch per sub-step (observe,
 * each policy layer, sample, env step) per step, FP32 SIMT, launched from the
 * host every step.  BATCHED_FP32: the same kernels, captured as a CUDA graph
 * per chunk of steps.  BATCHED_BF16: policy GEMMs (and the landscape
 * cross-term) on the tcgen05 tensor cores in BF16 with FP32 accumulation;
 * for the control env, the economy with 16-128-128-20 / -10 policies and at
 * most 384 agents per env, and the landscape with D in {8, 16, 24} and
 * D-256-256-2D policies, one persistent fused kernel runs a whole chunk (the
 * economy's over a device work queue of env groups). */
typedef enum { WS_PATH_PLAIN_FP32 = 0, WS_PATH_BATCHED_FP32 = 1, WS_PATH_BATCHED_BF16 = 2 } ws_path;

/* Fields of ws_fetch / ws_load.  Ring fields are time-major per step t:
 *   OBS     f32 [t][obs_dim][n_slots]   pre-step observation (acrobot:
 *                                       cos th1, sin th1, cos th2, sin th2,
 *                                       w1, w2)
 *   ACTION  i32 [t][n_slots]            (landscape: f32 [t][dim][n_slots] step dx)
 *   LOGP    f32 [t][n_slots]            log-probability of the sampled action
 *   REWARD  f32 [t][n_slots]
 *   DONE    u8  [t][n_slots]            1 if the step ended the episode
 *   RETURN  f32 [t][n_slots]            discounted return (after ws_returns)
 *   WEALTH  i64 [t][n_slots]            economy: pre-step agent wealth;
 *                                       planner slot: total wealth of its env
 *   ENERGY  f32 [t][n_slots]            landscape: E of the post-step state
 *   FORCE   f32 [t][dim][n_slots]       landscape with WS_FLAG_FORCE: -grad E
 *                                       of the post-step state (ws_forces)
 *   ADVANTAGE f32 [t][n_slots]          WS_FLAG_TRAIN: G - V(s) (ws_advantages)
 *   SAMPLE  f32 [t][dim][n_slots]       landscape with WS_FLAG_TRAIN: the
 *                                       unclipped Gaussian sample mean + sigma z
 *                                       of each step (ws_advantages)
 *   POLICY_OUT f32 [t][n_out][n_slots]  WS_FLAG_DEBUG_LOGITS: the policy outputs
 *                                       each step's sampler used, in FP32 (the
 *                                       logits; landscape: mean, then the raw
 *                                       log sigma before its clamp), written by
 *                                       every path; n_out is the agents' width
 *                                       (economy 20) and a planner slot holds
 *                                       its 10 logits in rows 0..9, zeros after
 * State fields (no step range; t0 and n_steps must be 0):
 *   STATE   control:   f32 s[4][n_envs] (x, v, th, w), i32 t[n_envs]
 *           acrobot:   f32 s[4][n_envs] (th1, th2, w1, w2), i32 t[n_envs]
 *           economy:   i64 wealth[n_agents], f32 feat[16][n_agents], i32 t[n_envs]
 *           landscape: f32 x[dim][n_envs], f32 eobs[n_envs], i32 t[n_envs]
 *   PARAMS  f32 policy parameters, per layer W[n_in][n_out] row-major then b;
 *           economy: agent policy then planner policy
 *   ENV_PARAMS  landscape: f32 centres[M][dim], f32 widths[M], f32 amps[M];
 *               economy:   i32 agents_per_env[n_envs]
 *   CRITIC  f32 critic parameters (WS_FLAG_TRAIN), laid out as PARAMS
 *           (economy: the agents' critic then the planner's)
 *   LOGITS  f32 [n_slots][n_out] policy outputs of the last step (plain and
 *           batched-FP32 paths, the economy's per-layer BF16 path, and its
 *           fused kernel with WS_FLAG_DEBUG_LOGITS)                         */
typedef enum {
  WS_F_OBS = 0,
  WS_F_ACTION = 1,
  WS_F_LOGP = 2,
  WS_F_REWARD = 3,
  WS_F_DONE = 4,
  WS_F_RETURN = 5,
  WS_F_WEALTH = 6,
  WS_F_ENERGY = 7,
  WS_F_STATE = 8,
  WS_F_PARAMS = 9,
  WS_F_ENV_PARAMS = 10,
  WS_F_LOGITS = 11,
  WS_F_FORCE = 12,
  WS_F_CRITIC = 13,
  WS_F_ADVANTAGE = 14,
  WS_F_SAMPLE = 15,
  WS_F_POLICY_OUT = 16
} ws_field;

/* ws_config.flags: every path also records each step's policy outputs in the
 * ring's POLICY_OUT field, and the fused economy and landscape kernels also
 * keep the last step's in the LOGITS field (costs HBM bandwidth; for tests and
 * debugging: the sampled actions can then be checked against the very logits
 * the sampler read).  The per-step paths always keep LOGITS. */
#define WS_FLAG_DEBUG_LOGITS 1u
/* ws_config.flags: landscape episodes also end when the pure energy E(x') of
 * the post-step state falls below ws_config.energy_target (the low-energy
 * product basin is the reaction's terminal state, paper App. C); the env then
 * resets like at the step limit.  On the BF16 paths E is the tensor-core
 * estimate, so a decision within its error of the target can go either way. */
#define WS_FLAG_ENERGY_TARGET 2u
/* ws_config.flags: the ring also holds the landscape FORCE field (D floats
 * per slot-step), written by ws_forces.  Landscape only. */
#define WS_FLAG_FORCE 4u
/* ws_config.flags: the context also holds a critic per policy (an MLP obs ->
 * hidden0 -> hidden1 -> 1, drawn from param_seed like the policies; the
 * economy's agents and planners have one each), the scratch of
 * ws_a2c_update and ws_ppo_update, and the ring's ADVANTAGE (and, for the
 * landscape, SAMPLE) field. */
#define WS_FLAG_TRAIN 8u
/* ws_config.flags: bounds check for debugging.  The state and the ring buffer
 * each end in a 256-byte canary (counted by ws_query_bytes) that ws_create
 * fills with 0xA5; ws_sync checks both after its wait and fails with
 * WS_ERR_CUDA ("canary overwritten", sticky) if a kernel wrote past the end of
 * either buffer's used part. */
#define WS_FLAG_BOUNDS_CHECK 16u

/* Roll-out configuration.  Slots: control and landscape have one agent per
 * env (n_slots = n_envs); the economy has agents_per_env[e] agents in env e,
 * laid out env by env, followed by one planner slot per env. */
typedef struct {
  uint32_t struct_size;   /* = sizeof(ws_config); guards ABI drift            */
  int32_t env;            /* ws_env                                           */
  int32_t path;           /* ws_path                                          */
  uint32_t n_envs;        /* >= 1                                             */
  uint32_t ring_steps;    /* steps the trajectory ring holds (>= 1)           */
  uint32_t episode_limit; /* episode step count that forces done (>= 1)      */
  uint32_t chunk_steps;   /* steps per graph / persistent launch; 0 = auto    */
  uint32_t hidden0;       /* policy hidden widths                             */
  uint32_t hidden1;
  uint32_t dim;           /* landscape: coordinates D (1..64)                 */
  uint32_t n_gauss;       /* landscape: Gaussians M (>= 1)                    */
  float noise_sigma;      /* landscape: observation-noise sigma               */
  float step_clip;        /* landscape: |dx_j| clip                           */
  float gamma;            /* discount of ws_returns                           */
  uint32_t flags;         /* WS_FLAG_* bits, others must be 0                 */
  uint64_t param_seed;    /* Philox key of policy / landscape / agent counts  */
  const int32_t *agents_per_env; /* economy, host, n_envs entries in 2..1024;
                                    NULL = draw U{8..256} from param_seed      */
  float energy_target;    /* landscape, with WS_FLAG_ENERGY_TARGET: done when
                             E(x') < energy_target (finite); else ignored    */
  uint32_t env_base;      /* global id of this context's env 0 (env_base +
                             n_envs <= 2^32 - 1).  Every per-env Philox
                             counter (action, reset, partner, noise draws,
                             the economy's drawn agent counts) carries the
                             global id env_base + e, while parameters depend
                             on param_seed alone: contexts over disjoint
                             ranges [b, b + n) of one workload (one per GPU)
                             record exactly what one context over the union
                             records for those envs (paper Sec. 2: one
                             workflow on one or several GPUs).            */
} ws_config;

/* Bytes of the two caller-owned device buffers a configuration needs:
 * state_bytes (parameters, env state, scratch, step counter) and ring_bytes
 * (the trajectory store).  Also reports the slot count.  Host-only, sync. */
ws_status ws_query_bytes(const ws_config *cfg, size_t *state_bytes, size_t *ring_bytes,
                         uint32_t *n_slots);

/* Create a context over caller-owned device buffers (at least the sizes of
 * ws_query_bytes, 256-byte aligned) on `cuda_stream` (a cudaStream_t; NULL =
 * legacy default stream).  Draws the policy parameters (and the landscape or
 * the agent counts) from param_seed (S0, paper App. B: policy models and the
 * environment reference live in global memory) and performs ws_reset with
 * seed = param_seed.  On failure *out is NULL. */
ws_status ws_create(const ws_config *cfg, void *state_buf, size_t state_bytes, void *ring_buf,
                    size_t ring_bytes, void *cuda_stream, ws_ctx **out);

/* Full reset (paper App. B, "reset" is part of the on-device workflow):
 * every env redraws its state from Philox(seed; k = 0xFFFFFFFF, env, agent,
 * RESET), episode counters and the step counter k become 0, and `seed`
 * becomes the key of all later per-step draws. */
ws_status ws_reset(ws_ctx *ctx, uint64_t seed);

/* One step of every env (observe, policy, sample, env step with auto-reset,
 * store), asynchronous.  k advances by 1. */
ws_status ws_step(ws_ctx *ctx);

/* n_steps steps, asynchronous.  The batched paths launch cached CUDA graphs
 * (and the persistent fused kernel); the plain path launches every kernel of
 * every step from the host.  k advances by n_steps. */
ws_status ws_rollout(ws_ctx *ctx, uint32_t n_steps);

/* Discounted returns over the last n_steps ring rows (steps k-n..k-1):
 * G_t = r_t + gamma (1 - done_t) G_{t+1}, with G = 0 after the window, in
 * compensated (float-float) FP32.  n_steps <= min(k, ring_steps). */
ws_status ws_returns(ws_ctx *ctx, uint32_t n_steps);

/* Actor-critic update on the last n_steps ring rows (steps k-n..k-1), in place
 * (paper Sec. 2 / App. B: the roll-out store feeds training on the GPU).
 * Advantage actor-critic with Monte-Carlo returns (on policy: the ring's steps
 * were sampled by the current parameters): the returns scan runs first
 * (into RETURN), then over the R = n_steps x n_slots rows (obs s, action a,
 * return G), with A = G - V(s) held constant in the policy's loss,
 *   L = (1/R) sum [ -A log pi(a|s) - c_e H(pi(.|s)) + c_v (G - V(s))^2 ],
 * and one SGD step of rate lr on the policy and the critic (FP32; the BF16
 * operand images are repacked).  The economy's agents (slots of agents) and
 * planner (planner slots) are two such updates, each the mean over its own
 * rows.  stats (host, may be NULL; the call then waits for the stream): the
 * means over all rows of -A log pi, (G - V)^2 and H.  Needs
 * WS_FLAG_TRAIN (WS_ERR_STATE); n_steps <= min(k, ring_steps) (WS_ERR_RANGE). */
ws_status ws_a2c_update(ws_ctx *ctx, uint32_t n_steps, float lr, float c_v, float c_e,
                        double *stats);

/* Advantages for a PPO update over the last n_steps ring rows (steps
 * k-n..k-1): the returns scan (into RETURN), then A = G - V(s) under the
 * critic as it is now, written to the ADVANTAGE field, where it stays fixed
 * for the epochs of ws_ppo_update that follow.  Landscape: also each row's
 * behaviour sample u = mean + sigma z (before the step clip) under the policy
 * as it is now, with the row's Philox normals z as the sampler drew them, into
 * the SAMPLE field (the ring keeps only the clipped step).  Asynchronous.  Needs
 * WS_FLAG_TRAIN (WS_ERR_STATE); n_steps <= min(k, ring_steps) (WS_ERR_RANGE). */
ws_status ws_advantages(ws_ctx *ctx, uint32_t n_steps);

/* One epoch of proximal policy optimisation (clipped surrogate) on the last
 * n_steps ring rows, in place (paper Sec. 2: the roll-out store feeds the
 * actor-critic trainer on the GPU; Sec. 3: actor-critic for discrete and
 * continuous actions).  Per row (obs s, action a, recorded log-probability
 * logp_old of the behaviour policy, return G, advantage A from
 * ws_advantages): rho = exp(log pi(a|s) - logp_old) and
 *   L = (1/R) sum [ -min(rho A, clip(rho, 1 - clip_eps, 1 + clip_eps) A)
 *                   - c_e H(pi(.|s)) + c_v (G - V(s))^2 ],
 * then one SGD step of rate lr on the policy and the critic (FP32; the BF16
 * operand images are repacked).  The landscape's diagonal Gaussian head scores
 * the SAMPLE field's u as its action.  The economy's agents and planners are
 * two such updates, each over its own rows.  Call it once per epoch: A stays
 * fixed, rho moves with the policy.  stats (host, may be NULL; the call then
 * waits for the stream): the means over all rows of -min(..), (G - V)^2, H,
 * and the fraction of rows with |rho - 1| > clip_eps.
 * Errors: WS_ERR_STATE without WS_FLAG_TRAIN, or unless ws_advantages covered
 * these n_steps rows since the last step, roll-out, reset or step-counter load;
 * WS_ERR_INVALID for clip_eps not > 0 or a non-finite argument. */
ws_status ws_ppo_update(ws_ctx *ctx, uint32_t n_steps, float lr, float clip_eps, float c_v,
                        float c_e, double *stats);

/* Landscape force over the last n_steps ring rows (steps k-n..k-1), written to
 * the FORCE field: F = -grad E(x') = sum_m a_m e_m (x' - c_m) / w_m^2 at the
 * post-step state x' = x + dx recorded in OBS and ACTION (paper App. C: the
 * landscape is the potential energy of the atomic positions, the force its
 * negative gradient).  Asynchronous.  WS_ERR_STATE without WS_FLAG_FORCE;
 * n_steps <= min(k, ring_steps) (WS_ERR_RANGE).  A step that ended an episode
 * still has its pre-reset x' recorded, so its force is that of x'. */
ws_status ws_forces(ws_ctx *ctx, uint32_t n_steps);

/* Copy a field (see ws_field) for absolute steps [t0, t0 + n_steps) into
 * dst (device memory if dst_on_device, else host memory; a host copy is
 * synchronous to the context stream).  dst_bytes must cover the block.
 * Steps not yet run or already overwritten in the ring -> WS_ERR_RANGE. */
ws_status ws_fetch(ws_ctx *ctx, ws_field field, uint64_t t0, uint32_t n_steps, void *dst,
                   size_t dst_bytes, int dst_on_device);

/* Overwrite STATE or PARAMS (same layouts as ws_fetch) from src, e.g. a
 * trainer's new policy weights or a checkpoint; then set the step counter to
 * k.  PARAMS keep the current k when k == UINT64_MAX. */
ws_status ws_load(ws_ctx *ctx, ws_field field, const void *src, size_t src_bytes,
                  int src_on_device, uint64_t k);

/* Current step counter k (host mirror; exact, since only the host enqueues). */
ws_status ws_get_step(const ws_ctx *ctx, uint64_t *k);

/* Block the host until the context's stream is idle, or return
 * WS_ERR_TIMEOUT after timeout_ms milliseconds (0 = wait forever; this one is
 * not sticky).  Then reads the device error flag of the tensor-core kernels: a
 * set flag (a bounded device wait ran out) is a sticky WS_ERR_TIMEOUT, and
 * ws_last_error names the wait's site.  With WS_FLAG_BOUNDS_CHECK it also
 * checks the canaries: an overwritten one is a sticky WS_ERR_CUDA, and
 * ws_last_error names the buffer, the field the canary guards and the byte. */
ws_status ws_sync(ws_ctx *ctx, uint32_t timeout_ms);

/* One-line description of the sticky error, or "" if none.  Never NULL. */
const char *ws_last_error(const ws_ctx *ctx);

/* Release the context (graphs, events); the caller's buffers are untouched.
 * Waits for the context's outstanding work first. */
void ws_destroy(ws_ctx *ctx);

/* ------------------------------------------------------------------------
 * Launch configuration and autotuning.  Every batched path has launch
 * parameters that change speed, not results (the one exception is the
 * landscape energy's Gaussian chunk count, which regroups an FP32 sum and so
 * moves its last bits): the chunk of steps per
 * persistent launch or captured graph, the persistent grid of the fused
 * control kernel, the rows per work item ("envs per CTA") of the fused economy
 * kernel and the order of its work queue, the Gaussian chunks per env tile of
 * the BF16 landscape energy kernel, the CTAs per env tile of the fused
 * landscape kernel, and the block size of the per-step kernels (envs per
 * block).  A context starts with defaults; ws_tune times the
 * candidates of its path on the device and keeps the fastest.
 * ------------------------------------------------------------------------ */
typedef struct {
  uint32_t struct_size;    /* = sizeof(ws_launch)                                   */
  uint32_t chunk_steps;    /* steps per persistent launch / captured graph (>= 1);
                              a nonzero ws_config.chunk_steps fixes it              */
  uint32_t grid;           /* fused control kernel: persistent CTAs, 0 = one per SM
                              (at most one per tile)                                */
  uint32_t econ_tiles;     /* fused economy kernel: 128-row agent tiles per work
                              item (1..3; at least the largest env's agents / 128)  */
  uint32_t econ_lpt;       /* fused economy kernel: 1 = queue the largest work items
                              first, 0 = in env order                               */
  uint32_t energy_chunks;  /* BF16 landscape: Gaussian chunks per env tile (1, 2, 4)*/
  uint32_t env_threads;    /* per-step kernels: threads per block, 64..1024, a
                              multiple of 32                                        */
  uint32_t tile_ctas;      /* fused landscape kernel: CTAs per 128-env tile, 1 or 2 (a
                              cluster whose CTAs split the Gaussians)               */
  uint32_t wait_ns;        /* limit of every device wait of the fused control,
                              acrobot, economy and landscape kernels (an MMA's
                              completion, the SFU token, a block load, the cluster
                              partner), in ns; 0 = 2 s.  A wait that runs out makes
                              the kernel drain its own MMAs and copies, free its
                              tensor memory and leave, and ws_sync reports a
                              sticky WS_ERR_TIMEOUT naming the wait's site.  For
                              tests of that path; results do not depend on it    */
  uint32_t ctrl_envs_per_cta; /* BF16 control / acrobot with hidden widths 64-64 or
                              128-128: 0 = the tensor-core kernel (128-env tiles,
                              two threads per env); else the CUDA-core kernels,
                              for env counts that leave SMs idle under 128-env
                              tiles, with this many envs per CTA (see
                              ctrl_threads_per_env).  They round the same
                              operands to BF16 (W2, h1) and accumulate in FP32;
                              their records do not depend on the two ctrl_
                              fields                                            */
  uint32_t ctrl_threads_per_env; /* CUDA-core kernels: 4, 8 or 16 = GEMM register
                              tiles of 16 / this envs x H / 16 units per thread,
                              W2 in shared memory (ctrl_envs_per_cta 4, 8, 16 or
                              32; 64..512 threads per CTA); 64 = one thread per
                              hidden unit with its W2 column in registers (hidden
                              width 64; ctrl_envs_per_cta 1, 2, 4 or 8)          */
  uint32_t update_gemm;    /* ws_a2c_update / ws_advantages / ws_ppo_update: the
                              hidden-by-hidden GEMMs on the tensor cores with
                              FP32 operands split into BF16 hi + lo (0, the
                              default), or on the FP32 CUDA cores (1)           */
} ws_launch;

/* The context's current launch configuration. */
ws_status ws_get_launch(const ws_ctx *ctx, ws_launch *out);

/* Replace the launch configuration (fields the context's path does not use
 * are ignored but must be in range).  Cached graphs are rebuilt on the next
 * roll-out; results are unchanged.  WS_ERR_INVALID for an out-of-range field. */
ws_status ws_set_launch(ws_ctx *ctx, const ws_launch *l);

/* Autotune: run each candidate launch configuration of the context's path for
 * trial_steps steps (after one untimed run of the same length), three times,
 * timed with CUDA events on the context's stream, and keep the candidate with
 * the fastest of its three runs.  The choice is
 * cached per process for the configuration's shape (env, path, sizes, agent
 * counts, device), so a later context of the same shape reuses it without
 * timing.  The trials advance the envs, so the call ends with ws_reset under
 * the context's current seed (step counter 0, ring contents overwritten).
 * Synchronous.  chosen and ms_per_step (the winner's time per step; NULL
 * allowed) report the result. */
ws_status ws_tune(ws_ctx *ctx, uint32_t trial_steps, ws_launch *chosen, float *ms_per_step);

/* ------------------------------------------------------------------------
 * Serving: a request loop with continuous batching over roll-out contexts.
 * Clients (trainers) submit roll-out requests of any env type and size.  A
 * request is admitted as soon as its device bytes (env state, parameters,
 * scratch and a trajectory ring of two chunks) fit in the server's budget;
 * it then keeps its env state resident on the device and advances one chunk
 * of chunk_steps steps at a time on a stream of its own, concurrently with the
 * other admitted requests.  A finished or released request frees its bytes.
 * All functions are thread-safe; ws_server_wait_chunk and ws_server_fetch
 * (host destination) block the calling thread only.
 * ------------------------------------------------------------------------ */
typedef struct ws_server ws_server;

#define WS_REQ_CONSUME_ON_READY 1u /* chunks need no ack; ring rows are reused at once
                                      and the request is released when done      */

typedef struct {
  uint32_t struct_size;   /* = sizeof(ws_request)                           */
  int32_t env, path;      /* ws_env, ws_path                                */
  uint32_t n_envs;
  uint32_t horizon;       /* total steps of the request                     */
  uint32_t chunk_steps;   /* steps per delivered chunk (>= 1)               */
  uint32_t episode_limit;
  uint32_t hidden0, hidden1, dim, n_gauss;
  uint32_t flags;         /* WS_REQ_* bits                                  */
  uint64_t seed;          /* parameter and roll-out key                     */
  const int32_t *agents_per_env; /* economy, host, copied; NULL = drawn     */
} ws_request;

typedef struct {
  uint32_t struct_size;   /* = sizeof(ws_server_stats), set by the caller   */
  uint64_t submitted, admitted, completed, rejected, failed, chunks;
  double agent_steps;     /* agent-steps of all delivered chunks            */
  double elapsed_s;       /* first submission to last delivered chunk       */
  double p50_ms, p99_ms;  /* chunk latency: chunk k ready - chunk k-1 ready
                             (chunk 0: from submission)                     */
  size_t used_bytes, peak_bytes, budget_bytes;
  uint32_t active, pending;
} ws_server_stats;

/* Create a server owning one device arena of budget_bytes (cudaMalloc on the
 * current device) and its scheduler thread.  WS_ERR_NOMEM if the arena cannot
 * be allocated. */
ws_status ws_server_create(size_t budget_bytes, ws_server **out);

/* Queue a request; *id names it.  WS_ERR_NOMEM if it can never fit the
 * budget, WS_ERR_INVALID / WS_ERR_UNSUPPORTED for a bad configuration. */
ws_status ws_server_submit(ws_server *s, const ws_request *req, uint64_t *id);

/* Block until chunk `chunk` of request id is ready, or WS_ERR_TIMEOUT after
 * timeout_ms (0 = no limit).  A failed request returns its error. */
ws_status ws_server_wait_chunk(ws_server *s, uint64_t id, uint32_t chunk, uint32_t timeout_ms);

/* Copy a ring field (ws_fetch layouts) of a ready, not yet acknowledged chunk
 * into dst (device or host memory); returns when the copy is complete. */
ws_status ws_server_fetch(ws_server *s, uint64_t id, ws_field field, uint32_t chunk, void *dst,
                          size_t dst_bytes, int dst_on_device);

/* Acknowledge chunks up to and including `chunk`: their ring rows may be
 * reused.  Without WS_REQ_CONSUME_ON_READY at most two chunks run ahead of
 * the last acknowledgement. */
ws_status ws_server_ack(ws_server *s, uint64_t id, uint32_t chunk);

/* Cancel (if running) and forget a request, freeing its bytes. */
ws_status ws_server_release(ws_server *s, uint64_t id);

ws_status ws_server_get_stats(ws_server *s, ws_server_stats *out);

/* Serve clients in other processes (trainer processes on the same machine)
 * over a Unix-domain stream socket created at `path` (a file already there is
 * replaced); one thread per connection.  Messages are [u32 op][u32 payload
 * bytes][payload] in host byte order, every reply begins with an i32 ws_status:
 *   1 SUBMIT  ws_request [+ i32 agents_per_env[n_envs]]  -> status, u64 id
 *   2 WAIT    u64 id, u32 chunk, u32 timeout_ms (0: none)  -> status
 *   3 FETCH   u64 id, i32 field, u32 chunk                 -> status, u64 n, n bytes
 *             (the ws_fetch layout of the chunk's steps)
 *   4 ACK     u64 id, u32 chunk                            -> status
 *   5 RELEASE u64 id (one this connection submitted)       -> status
 *   6 STATS                                                -> status, ws_server_stats
 * When a connection closes (the client exited or was killed) the requests it
 * submitted and did not release are released, freeing their bytes.  The
 * socket is removed by ws_server_destroy.  WS_ERR_STATE if the socket cannot be
 * created, WS_ERR_INVALID if the server already listens. */
ws_status ws_server_listen(ws_server *s, const char *path);

/* Stop the scheduler (and the socket of ws_server_listen), release every
 * request and free the arena. */
void ws_server_destroy(ws_server *s);

/* Policy forward pass that allocates no device memory (the paper has no
 * counterpart; it is a service for callers that cannot call cudaMalloc, such
 * as code running during CUDA-graph capture, hosts whose allocator forbids
 * foreign allocations, or embedded runtimes with fixed device memory).
 *   out[n_rows][out_dim] = tanh(tanh(obs W0 + b0) W1 + b1) W2 + b2, in FP32,
 * obs [n_rows][in_dim] row-major and params in the PARAMS layout (per layer
 * W[n_in][n_out] row-major, then b), all device pointers owned by the caller.
 * The hidden activations use a 16 MiB library-owned static device array
 * (every GPU that loads the library holds it until the process exits), so
 * n_rows * (hidden0 + hidden1) may not exceed 4,194,304 floats: larger
 * requests return WS_ERR_RANGE before anything is launched.  No cudaMalloc,
 * cudaFree or allocating library call is made.  The first call on a device
 * looks up that array's device address (with that device current); make that
 * first call before any stream capture.  All calls on a device share the
 * array: calls that overlap on the GPU (other streams, other threads) race and
 * must be serialised by the caller.  Asynchronous on cuda_stream. */
ws_status ws_policy_forward_noalloc(const float *obs, uint32_t n_rows, const float *params,
                                    uint32_t in_dim, uint32_t hidden0, uint32_t hidden1,
                                    uint32_t out_dim, float *out, void *cuda_stream);

/* ------------------------------------------------------------------------
 * Throughput probes (the paper has no counterpart: these measure the peak
 * rates the roofline fractions of the fused kernels divide by).  One launch of
 * a probe kernel on the current device: 4 blocks of 256 threads per SM, each
 * thread running 8 independent chains of the operation for `iters` rounds;
 * *per_clk_per_sm = results per SM clock (packed forms count two results per
 * lane), from clock64 spans.  dev_buf: caller-owned device memory of at least
 * 16 bytes per block (4 x SMs blocks).  Synchronous on cuda_stream.
 * WS_ERR_INVALID for an unknown op or iters == 0, WS_ERR_NOMEM for a small
 * buffer.
 * ------------------------------------------------------------------------ */
typedef enum {
  WS_PROBE_TANH_F32 = 0,     /* tanh.approx.f32                               */
  WS_PROBE_TANH_BF16X2 = 1,  /* tanh.approx.bf16x2 (two results)              */
  WS_PROBE_EX2_F32 = 2,      /* ex2.approx.ftz.f32                            */
  WS_PROBE_EX2_BF16X2 = 3,   /* ex2.approx.ftz.bf16x2 (two results)           */
  WS_PROBE_EX2_F16X2 = 4,    /* ex2.approx.f16x2 (two results)                */
  WS_PROBE_RCP_F32 = 5,      /* rcp.approx.ftz.f32 (with one FP32 add)        */
  WS_PROBE_SIN_F32 = 6,      /* sin.approx.ftz.f32                            */
  WS_PROBE_FMA_F32 = 7,      /* fma.rn.f32                                    */
  WS_PROBE_FMA_F32X2 = 8,    /* fma.rn.f32x2 (two results)                    */
  WS_PROBE_LG2_F32 = 9,      /* lg2.approx.ftz.f32 (with one FP32 FMA)        */
  WS_PROBE_RSQRT_F32 = 10,   /* rsqrt.approx.ftz.f32 (with one FP32 add)      */
  WS_PROBE_TANH_F32_HALF = 11, /* tanh.approx.f32 on lanes 0-15 of every warp
                                  only; counts the results of those lanes, so
                                  half the full rate means a warp instruction
                                  costs the same with half its lanes idle      */
  WS_PROBE_COUNT = 12
} ws_probe_op;

ws_status ws_probe_rate(int op, uint32_t iters, void *dev_buf, size_t buf_bytes,
                        double *per_clk_per_sm, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* WARPSCI_H */
