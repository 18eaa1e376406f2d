/*
 * mppi_jump.h -- C ABI of libmppi_jump.so: GB300 (sm_103a) MPPI on jump
 * diffusion processes, after Wang, Williams & Theodorou, "Information
 * Theoretic Model Predictive Control on Jump Diffusion Processes".
 *
 * One optimisation iteration (Algorithm 1) is
 *   rollout_cost : sample delta ~ N(0, c diag(sigma^2)) per rollout and step,
 *                  jump counts (compound Poisson, E[dP] = nu dt, Eq. 2, or the
 *                  zero-one jump timer of Algorithm 1) and marks, roll the
 *                  plant out with Euler steps and accumulate the augmented
 *                  cost S~ of Eq. 34-35;
 *   update       : weights w_k = exp(-S~_k/lambda) / sum exp(-S~/lambda)
 *                  (Eq. 36-37) and U_j += alpha sum_k w_k delta_eff_{k,j}
 *                  (Eq. 37 with alpha of Eq. 49);
 *   step         : `iters` iterations from the same x0, then execute u_0,
 *                  shift and append u_init (Algorithm 1, MPC loop of Sec. V).
 *
 * Conventions for every call below.
 *   - Pointers are DEVICE pointers unless the argument name ends in `_host`.
 *   - Device work is enqueued on the context's stream (given at init); calls
 *     return once the work is enqueued, except those with host outputs, which
 *     synchronise that stream before returning.
 *   - Errors are returned as mppi_status codes; nothing aborts, traps or
 *     throws.  mppi_jump_last_error() gives a message for the last failure on
 *     a context.  Device-side conditions (all costs non-finite: MPPI_ENONFINITE;
 *     a bounded device wait that expired: MPPI_ETIMEOUT) are recorded in a
 *     status word that the next synchronising call returns.
 *   - A context is not thread-safe; distinct contexts are independent.
 *   - All arrays are dense, row-major, float32 unless stated:
 *       x0 [n], U [T][m], costs [K], weights [K],
 *       noise delta_eff [T][K][m] (step-major: all rollouts of step 0 first),
 *       counts [T][K] uint8, jumps J [T][K][q].
 *     n = 4, m = 1 for the cart-pole; n = 12, m = 4 for the quadrotor.
 */
#ifndef MPPI_JUMP_H
#define MPPI_JUMP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MPPI_JUMP_ABI_VERSION 1
#define MPPI_MAX_JUMPS 16 /* largest jump count per step the sampler draws */

typedef enum {
  MPPI_OK = 0,
  MPPI_EINVAL = 1,     /* invalid argument or configuration */
  MPPI_ENOMEM = 2,     /* device or host allocation failed, or over budget */
  MPPI_ECUDA = 3,      /* a CUDA runtime call failed */
  MPPI_ETIMEOUT = 4,   /* a bounded device wait gave up */
  MPPI_ENONFINITE = 5, /* every rollout cost was non-finite: U left unchanged */
  MPPI_EBUSY = 6,      /* resource in use (e.g. session already has a request) */
  MPPI_EBOUNDS = 7     /* a kernel's launch check failed (MPPI_CHECK_BOUNDS builds only) */
} mppi_status;

typedef enum { MPPI_CARTPOLE = 0, MPPI_QUADROTOR = 1 } mppi_system;
typedef enum { MPPI_COUNT_POISSON = 0, MPPI_COUNT_BERNOULLI = 1 } mppi_count_law;
typedef enum { MPPI_MARK_NORMAL = 0, MPPI_MARK_LAPLACE = 1 } mppi_mark_law;
typedef enum { MPPI_JUMP_STATE = 0, MPPI_JUMP_CONTROL = 1 } mppi_jump_channel;
typedef enum { MPPI_NOISE_F32 = 0, MPPI_NOISE_BF16 = 1 } mppi_noise_dtype;

/* Plant constants.  Cart-pole: point-mass pole, theta = 0 hanging down,
 * q(x) = (x-goal)^T diag(Q) (x-goal), phi(x) = (x-goal)^T diag(Qf) (x-goal).
 * Quadrotor: state (p, v, eta = ZYX Euler angles, omega = body rates), rotor
 * thrusts in a "+" layout (1,2,3,4 on +x,+y,-x,-y), torque
 * (arm (f2-f4), arm (f3-f1), kappa (f1-f2+f3-f4));
 * q(x) = wp|p-goal|^2 + wv|v|^2 + weta|eta|^2 + wom|omega|^2
 *        + obs_cost [|p-obs|^2 < obs_r^2],  phi(x) = q(x) without the indicator. */
typedef struct {
  float mc, mp, l, g;
  float goal[4], Q[4], Qf[4];
} mppi_cartpole_params;

typedef struct {
  float mass, J[3], arm, kappa, g;
  float goal[3], wp, wv, weta, wom;
  float obs[3], obs_r, obs_cost;
} mppi_quadrotor_params;

/* Problem configuration: the "Given" list of Algorithm 1 (M = K samples,
 * N = T steps, dt, plant f/G/B/H, cost phi/q/lambda/R, noise c/Sigma_D/
 * Sigma_J/nu, u_init).  R is implied by Eq. 14 (R = lambda G^T Sigma^-1 G) and
 * B = G (Sec. IV), so the control cost follows from sigma and lambda. */
typedef struct {
  int32_t system;        /* mppi_system */
  int32_t K;             /* rollouts, 1 .. 2^24 */
  int32_t T;             /* horizon steps, 1 .. 4096 */
  float dt;              /* step, > 0 */
  float lambda;          /* temperature, > 0 */
  float c;               /* exploration variance scale of Eq. 33, > 0 */
  float alpha;           /* step size of Eq. 49 (1 gives Eq. 36) */
  float sigma[4];        /* std of the control perturbation delta = eps/sqrt(dt) */
  float jump_rate;       /* nu, jumps per second, >= 0 */
  int32_t count_law;     /* mppi_count_law */
  int32_t mark_law;      /* mppi_mark_law */
  float mark_scale[4];   /* Normal std / Laplace scale per mark component */
  int32_t jump_channel;  /* mppi_jump_channel */
  int32_t q;             /* mark dimension (must equal m for MPPI_JUMP_CONTROL) */
  int32_t jump_rows[4];  /* state rows hit by the marks (MPPI_JUMP_STATE) */
  int32_t jump_sqrt_dt;  /* state mode: 1 scales the jump by sqrt(dt) */
  int32_t noise_dtype;   /* mppi_noise_dtype for the stored delta_eff */
  float u_init[4];       /* appended after each MPC shift */
  uint64_t seed;         /* Philox key: (seed mod 2^32, seed >> 32) */
  mppi_cartpole_params cartpole;
  mppi_quadrotor_params quadrotor;
  float alpha_decay;     /* step size alpha^r = alpha * alpha_decay^r at iteration r
                            of an MPC step (Eq. 48-49); in [0, 1], 0 reads as 1 */
} mppi_jump_config;

typedef struct mppi_jump_ctx mppi_jump_ctx;

/* Fills *out with the defaults for `system` (the cart-pole swing-up or the
 * quadrotor waypoint flight, K = 1000 / 4096 rollouts).  Host only. */
mppi_status mppi_jump_default_config(int32_t system, mppi_jump_config* out);

/* Checks a configuration without touching the GPU. */
mppi_status mppi_jump_validate(const mppi_jump_config* cfg);

/* sizeof(mppi_jump_config) as compiled into the library, so that bindings
 * can verify their struct layout. */
size_t mppi_jump_config_bytes(void);

/* Jump-count threshold table for rate nu and step dt (host only).  Poisson:
 * thr[n-1] = ceil(2^32 F(n-1; nu dt)), F the Poisson CDF summed term by term
 * (term_0 = e^-mu, term_n = term_{n-1} mu / n), a word w giving the count
 * #{n : w >= thr[n-1]}; entries that would equal 2^32 end the table (*nmax).
 * Bernoulli: thr[0] = round(2^32 nu dt), count = [w < thr[0]].  Returns
 * MPPI_EINVAL when nu dt is negative or non-finite, when the Poisson tail
 * beyond MPPI_MAX_JUMPS is not negligible (> 2^-32), or Bernoulli nu dt >= 1. */
mppi_status mppi_jump_count_table(float jump_rate, float dt, int32_t count_law,
                                  uint32_t thr_host[MPPI_MAX_JUMPS], int32_t* nmax_host);

/* Device bytes a context with this configuration allocates. */
mppi_status mppi_jump_workspace_bytes(const mppi_jump_config* cfg, size_t* bytes_host);

/* Creates a context on the current device: allocates the perturbation,
 * cost, weight and control buffers (cudaMalloc), sets U = u_init for every
 * step and the iteration counter to 0.  `stream` is the cudaStream_t on which
 * every later call enqueues its work; NULL makes the context create and own a
 * non-blocking stream (the caller then orders its own work with
 * mppi_jump_sync).  Fails with MPPI_ENOMEM when the device allocation fails.
 * The context owns its device memory until mppi_jump_destroy. */
mppi_status mppi_jump_init(const mppi_jump_config* cfg, void* stream, mppi_jump_ctx** out);

/* Frees everything the context owns (synchronises its stream).  NULL is a no-op. */
mppi_status mppi_jump_destroy(mppi_jump_ctx* ctx);

/* Message describing the last failure on ctx (static string when ctx is NULL). */
const char* mppi_jump_last_error(const mppi_jump_ctx* ctx);
const char* mppi_jump_status_string(mppi_status st);

/* Replaces / reads the control sequence U [T][m] (device pointers). */
mppi_status mppi_jump_set_controls(mppi_jump_ctx* ctx, const float* U);
mppi_status mppi_jump_get_controls(mppi_jump_ctx* ctx, float* U);

/* Sets / reads the iteration counter that selects the Philox stream. */
mppi_status mppi_jump_set_iteration(mppi_jump_ctx* ctx, uint32_t it);
mppi_status mppi_jump_get_iteration(mppi_jump_ctx* ctx, uint32_t* it_host);

/* A1+A2 (Algorithm 1 sampling and rollout loop; Eq. 2, 4, 34-35): for the
 * current iteration counter, samples the noise, rolls out all K rollouts
 * from x0 [n] under the context's U and stores delta_eff and the costs in
 * the context.  If `costs` is not NULL it receives S~ [K]. */
mppi_status mppi_jump_rollout_cost(mppi_jump_ctx* ctx, const float* x0, float* costs);

/* A3+A4 (Eq. 36-37, 49): softmin weights of the last rollout_cost and the
 * in-place update of the context's U with step size alpha (the schedule's
 * first step), then counter += 1.  If every cost was non-finite, U is left
 * unchanged and the next synchronising call returns MPPI_ENONFINITE. */
mppi_status mppi_jump_update(mppi_jump_ctx* ctx);

/* Rollout sharding: one problem's rollouts split over several contexts
 * (typically one per GPU).  Eq. 37 is a ratio of two sums over the rollouts,
 * which are independent (Sec. V runs them in parallel), so a shard reduces its
 * rollouts to a partial record and the records combine exactly, up to
 * rounding.  A shard is a context whose configuration has K = the shard's
 * rollout count and whose rollout offset is the index k0 of its first rollout
 * in the unsharded problem: its rollouts draw the random numbers of rollouts
 * k0 .. k0+K-1.
 * mppi_jump_set_rollout_offset: sets k0 (default 0; k0 + K must stay below
 *   2^32; drops the cached step graphs).
 * mppi_jump_rollout_partial: rollout_cost from x0 [n] (device) for the current
 *   counter, then writes the shard's partial record partial [2 + T*m]
 *   (device): rho_g = min_k S~_k, Z_g = sum_k e_k and N_g[j][i] =
 *   sum_k e_k delta_eff[j][k][i] with e_k = exp(-(S~_k - rho_g)/lambda)
 *   (S~ without the rollout-independent control cost).  U and the counter are
 *   unchanged.  A shard whose costs are all non-finite writes (+inf, 0, 0 ...).
 * mppi_jump_apply_partials: combines n_parts records [n_parts][2 + T*m]
 *   (device, 1 .. 4096 of them) with rho = min_g rho_g,
 *   Z = sum_g Z_g exp(-(rho_g - rho)/lambda) and N likewise, applies
 *   U += alpha_r N / Z (alpha_r = alpha * alpha_decay^r, iteration r of an MPC
 *   step); shift != 0 also executes u0 [m] (device, may be NULL), shifts and
 *   appends u_init; the counter advances by one.  Shards that apply the same
 *   records in the same order keep bit-identical controls.  If every record
 *   has rho = +inf, U is unchanged and the next synchronising call returns
 *   MPPI_ENONFINITE. */
mppi_status mppi_jump_set_rollout_offset(mppi_jump_ctx* ctx, uint32_t k_offset);
mppi_status mppi_jump_rollout_partial(mppi_jump_ctx* ctx, const float* x0, float* partial);
mppi_status mppi_jump_apply_partials(mppi_jump_ctx* ctx, const float* partials, int32_t n_parts,
                                     int32_t r, int32_t shift, float* u0);

/* A5 (Algorithm 1 MPC loop): `iters` x (rollout_cost + update) from the same
 * x0, iteration r with step size alpha * alpha_decay^r, then u0 = U_0,
 * U_i <- U_{i+1}, U_{T-1} <- u_init.  The work is replayed from a CUDA graph
 * captured on first use for each `iters`.
 * mppi_jump_step takes HOST x0 [n] and writes HOST u0 [m] (synchronous);
 * mppi_jump_step_async takes device pointers and does not synchronise. */
mppi_status mppi_jump_step(mppi_jump_ctx* ctx, const float* x0_host, int32_t iters,
                           float* u0_host);
mppi_status mppi_jump_step_async(mppi_jump_ctx* ctx, const float* x0, int32_t iters,
                                 float* u0);

/* Rollout launch shape ("tile").  rollout_variant 1 = fused: one kernel,
 * one thread per rollout, draws the noise and rolls out; 2 = split: a noise
 * pass over K x T/4 threads stores delta_eff and the state-jump records
 * (every step's while the rollout blocks of 128 fit on the SMs at once;
 * beyond that jump masks, and a marks pass writes the records of the jumping
 * steps), then one thread per rollout runs the sequential dynamics (more
 * parallelism when K alone does not fill the GPU); 3 = staged: the split
 * form with the step data of each block's rollouts moved into shared memory
 * by bulk copies;
 * 4 = staged, and each rollout block also reduces its own rollouts to the
 * partial record of mppi_jump_rollout_partial (re-reading its perturbation
 * rows through shared memory), so that the update only combines the blocks'
 * records.
 * rollout_block: threads per block of the rollout kernel (32, 64, 96 or
 * 128).  rollout_chunk: for the split form, how many steps ahead its loads
 * run (2, 4 or 8); for the staged forms, steps per shared-memory stage (4, 8
 * or 16); for the fused form, steps per unrolled chunk (4, 8 or 16).  The
 * staged forms launch one extra (producer) warp per block.  The default is
 * staged with 16-step stages, block 96 while blocks of 96 fit on the SMs at
 * once, else block 128, with 8-step stages from two waves of blocks of 128
 * on.  Every tile
 * computes identical costs; tiles 1-3 give identical updates, tile 4 the
 * same update up to the summation order.  Setting a tile drops the cached
 * graphs. */
typedef struct {
  int32_t rollout_variant;
  int32_t rollout_block;
  int32_t rollout_chunk;
} mppi_jump_tuning;
mppi_status mppi_jump_set_tuning(mppi_jump_ctx* ctx, const mppi_jump_tuning* tuning_host);
mppi_status mppi_jump_get_tuning(mppi_jump_ctx* ctx, mppi_jump_tuning* tuning_host);

/* Autotuner: times the MPC step (graph replay, `iters` iterations from the
 * device state x0 [n]) for every rollout tile (fused x block 32, 64, 128;
 * split x block 32, 64, 128 x chunk 2, 4, 8; staged and staged with block
 * records x blocks and stages), `reps` timed steps each after
 * one warm-up, with CUDA events on the
 * context's stream, and keeps the fastest.  U and the iteration counter are
 * restored afterwards, so tuning does not change later results (every tile
 * computes the same values).  best_host (may be NULL) receives the choice and
 * best_ms_host (may be NULL) its mean step time. */
mppi_status mppi_jump_autotune(mppi_jump_ctx* ctx, const float* x0, int32_t iters, int32_t reps,
                               mppi_jump_tuning* best_host, float* best_ms_host);

/* Phase timing.  With timing enabled, each MPC step records CUDA events
 * around every rollout launch and every weights+update launch (event record
 * nodes inside the replayed graph); mppi_jump_phase_times synchronises and
 * returns the summed durations of the last step in milliseconds
 * (out_host[0] = rollout, out_host[1] = softmin + update) and the number
 * of iterations they cover in *iters_host.  Enabling or disabling timing
 * drops the cached graphs. */
mppi_status mppi_jump_enable_timing(mppi_jump_ctx* ctx, int32_t on);
mppi_status mppi_jump_phase_times(mppi_jump_ctx* ctx, float out_host[2], int32_t* iters_host);

/* Synchronises the context's stream and returns (then clears) the device
 * status word: MPPI_OK, MPPI_ENONFINITE, MPPI_ETIMEOUT or (debug builds with
 * MPPI_CHECK_BOUNDS, libmppi_jump_checked.so) MPPI_EBOUNDS: a kernel found
 * its launch geometry or shared memory inconsistent with its problem and
 * returned before touching memory; the context should then be destroyed. */
mppi_status mppi_jump_sync(mppi_jump_ctx* ctx);

/* Debug outputs of the following rollout_cost calls (NULL disables):
 * counts [T][K] uint8 jump counts, jumps [T][K][q] summed marks J. */
mppi_status mppi_jump_set_debug(mppi_jump_ctx* ctx, uint8_t* counts, float* jumps);

/* Copies of the last iteration's intermediates:
 * noise: delta_eff [T][K][m] in the context's noise dtype (float32 or
 * bfloat16 bits); weights: w [K]; free energy (host, 3 floats):
 * rho = min S~, Z = sum exp(-(S~-rho)/lambda), F = rho/lambda - ln(Z/K)
 * (the Monte Carlo form of Eq. 5).  The free-energy call synchronises. */
mppi_status mppi_jump_get_noise(mppi_jump_ctx* ctx, void* noise);
mppi_status mppi_jump_get_weights(mppi_jump_ctx* ctx, float* weights);
mppi_status mppi_jump_get_free_energy(mppi_jump_ctx* ctx, float out_host[3]);

/* Checkpoint: serialises (configuration, U, counter) into buf_host.  With
 * buf_host NULL, *size_host receives the size needed.  Restoring into a
 * context created from the same configuration continues the random stream
 * exactly, so restore-then-solve equals solve-without-interruption. */
mppi_status mppi_jump_get_state(mppi_jump_ctx* ctx, void* buf_host, size_t* size_host);
mppi_status mppi_jump_set_state(mppi_jump_ctx* ctx, const void* buf_host, size_t size);

/* Allocation-free weights + weighted update.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory
 * while they run -- a fixed-rate control loop (a cudaMalloc or cudaFree may
 * synchronise the device and take unbounded time) or a program whose device
 * memory belongs to another allocator or a fixed memory plan.  It computes
 * what mppi_jump_update computes (the softmin weights of the rollout costs
 * and U += alpha * the weighted mean of the perturbations, without the MPC
 * shift) from caller-supplied arrays, all DEVICE pointers:
 *   costs [K] rollout costs S~ (non-finite entries get weight 0),
 *   noise [T][K][m] float32 perturbations delta_eff, step-major,
 *   U [T][m] controls, updated in place.
 * m is 1 or 4.  The work is enqueued on `stream` (a cudaStream_t); the call
 * does not synchronise.  It allocates nothing: its scratch (the split-K
 * partial sums, chunk normalisers, running minimum and completion ticket) is
 * a file-scope device array of 4 MiB (2^20 floats) that every GPU loading
 * this library holds until the process exits.  The first call on a device
 * looks up that array's device address (cudaGetSymbolAddress), so make the
 * first call on each device outside any stream capture.  Every call shares
 * the array and clears its control words first: calls whose work overlaps on
 * the GPU race and must be serialised by the caller.  Limits: T <= 524280
 * (8 steps per block along the grid's y dimension) and
 * 64 + ceil(K/1024) * (T*m + 1) floats within the scratch.  Returns
 * MPPI_EINVAL for bad arguments or T beyond its limit and MPPI_ENOMEM when
 * the scratch is too small, in both cases before any work is enqueued; if
 * every cost is non-finite, U is left unchanged. */
mppi_status mppi_jump_update_noalloc(const float* costs, const float* noise, int32_t K, int32_t T,
                                     int32_t m, float lambda, float alpha, float* U, void* stream);

/* ------------------------------------------------------------------------ */
/* Batched form: n independent MPC instances (any mix of plants, K, T, noise */
/* laws and iteration counts; one noise dtype for all) advanced together by  */
/* ONE persistent kernel per batched step, replayed from a CUDA graph.  Each */
/* instance computes exactly what mppi_jump_step computes for it (Algorithm  */
/* 1: iters[i] x (rollout_cost + update), then execute u_0 and shift); only  */
/* the summation order of the weighted update differs.  The kernel claims    */
/* work items (rollout tiles, weighted-sum chunks, combines) in a fixed      */
/* dependency order; a dependency wait that exceeds 2 s ends the step with   */
/* MPPI_ETIMEOUT instead of hanging.                                         */
/* ------------------------------------------------------------------------ */
typedef struct mppi_batch mppi_batch;

/* cfgs [n] configurations, iters_host [n] iterations per MPC step (>= 1).
 * Allocates all device state (cudaMalloc) and sets every U to u_init.
 * stream: cudaStream_t for all work (NULL: the batch creates its own). */
mppi_status mppi_batch_create(const mppi_jump_config* cfgs_host, const int32_t* iters_host,
                              int32_t n, void* stream, mppi_batch** out);
mppi_status mppi_batch_destroy(mppi_batch* b);
const char* mppi_batch_last_error(const mppi_batch* b);

/* One batched MPC step.  x0s [n][12] (row i holds instance i's state in its
 * first n_i entries), u0s [n][4] (first m_i entries).  _async takes device
 * pointers (u0s may be NULL) and does not synchronise; mppi_batch_step takes
 * HOST arrays, synchronises and returns the batch status. */
mppi_status mppi_batch_step_async(mppi_batch* b, const float* x0s, float* u0s);
mppi_status mppi_batch_step(mppi_batch* b, const float* x0s_host, float* u0s_host);
/* Synchronises and returns the status word of the last step(s):
 * MPPI_OK, MPPI_ENONFINITE (an instance had only non-finite costs; its U is
 * unchanged) or MPPI_ETIMEOUT (a dependency wait expired). */
mppi_status mppi_batch_sync(mppi_batch* b);

/* Instance i's control sequence [T_i][m_i] (device or host pointer; both
 * calls synchronise) and iteration counter. */
mppi_status mppi_batch_get_controls(mppi_batch* b, int32_t i, float* U);
mppi_status mppi_batch_set_controls(mppi_batch* b, int32_t i, const float* U);
mppi_status mppi_batch_get_iteration(mppi_batch* b, int32_t i, uint32_t* it_host);

/* Tile of the persistent kernel: block = rollouts per rollout item and
 * threads per block (64, 128 or 256); chunk = steps per unrolled chunk of a
 * rollout item (4 or 8: the chunk's random numbers are drawn together, so
 * later steps' sampling overlaps earlier steps' dynamics).  Every tile
 * computes the same costs.  set_tuning changes the block only. */
mppi_status mppi_batch_set_tuning(mppi_batch* b, int32_t block);
mppi_status mppi_batch_get_tuning(mppi_batch* b, int32_t* block_host);
mppi_status mppi_batch_set_tile(mppi_batch* b, int32_t block, int32_t chunk);
mppi_status mppi_batch_get_tile(mppi_batch* b, int32_t* block_host, int32_t* chunk_host);
/* Failure-path test hook: with on != 0 the following steps start with a work
 * item whose dependency is never satisfied, so the step ends with
 * MPPI_ETIMEOUT after the bounded wait (about 2 s) instead of running; the
 * instances' controls may then be partially advanced.  on = 0 restores the
 * normal work list. */
mppi_status mppi_batch_inject_stall(mppi_batch* b, int32_t on);
/* Autotuner: times `reps` batched steps for each tile (block 64, 128, 256 x
 * chunk 4, 8) from device x0s and keeps the fastest (read it back with
 * mppi_batch_get_tile); controls and counters are restored afterwards. */
mppi_status mppi_batch_autotune(mppi_batch* b, const float* x0s, int32_t reps,
                                int32_t* best_block_host, float* best_ms_host);
/* Trajectory-steps of one batched step (sum of K_i T_i iters_i), the number of
 * work items and the persistent grid size (any may be NULL). */
mppi_status mppi_batch_info(mppi_batch* b, int64_t* steps_per_solve_host, int32_t* n_items_host,
                            int32_t* grid_host);

/* ------------------------------------------------------------------------ */
/* Served form: a native request loop over n sessions (any mix of plants, K, */
/* T).  Each request is one MPC step (Algorithm 1 with the session's         */
/* iteration count) warm-started from the session's device-resident controls */
/* and counter (Sec. V).  A worker thread admits requests as soon as the     */
/* session is idle (per-session order = submission order), one of            */
/* max_inflight slots is free, and the session's device memory fits the      */
/* budget -- idle sessions are checkpointed to the host and released, least  */
/* recently used first, to make room.  Admitted requests run concurrently on */
/* their sessions' own streams (continuous batching at the stream level).    */
/* A session's results do not depend on what else is in flight.  All         */
/* pointers are HOST pointers.                                               */
/* ------------------------------------------------------------------------ */
typedef struct mppi_server mppi_server;

typedef struct {
  int64_t submitted, completed, inflight, evictions;
  double mean_ms, max_ms, p50_ms, p99_ms; /* submit-to-completion latency */
  double span_s;                          /* first submission to last completion */
  size_t resident_bytes;                  /* device bytes of resident sessions */
} mppi_serve_stats;

/* cfgs [n], iters [n] (>= 1); budget_bytes bounds the device memory of the
 * resident sessions (a session larger than the budget is MPPI_EINVAL). */
mppi_status mppi_serve_create(const mppi_jump_config* cfgs_host, const int32_t* iters_host,
                              int32_t n_sessions, size_t budget_bytes, int32_t max_inflight,
                              mppi_server** out);
/* Waits for all queued and running requests, then frees everything. */
mppi_status mppi_serve_destroy(mppi_server* s);
const char* mppi_serve_last_error(const mppi_server* s);
/* Queues one MPC step of `session` from state x0 [n]; returns at once. */
mppi_status mppi_serve_submit(mppi_server* s, int32_t session, const float* x0_host,
                              uint64_t* ticket_host);
/* done_host = 1 once the request finished; then u0 [m] is written and the
 * request's status returned. */
mppi_status mppi_serve_poll(mppi_server* s, uint64_t ticket, float* u0_host, int32_t* done_host);
/* Blocks until the request finished (MPPI_ETIMEOUT after timeout_s). */
mppi_status mppi_serve_wait(mppi_server* s, uint64_t ticket, float* u0_host, double timeout_s);
/* Blocks until every submitted request finished (MPPI_ETIMEOUT after timeout_s). */
mppi_status mppi_serve_drain(mppi_server* s, double timeout_s);
mppi_status mppi_serve_get_stats(mppi_server* s, mppi_serve_stats* out_host);
/* Forgets finished requests and latencies (MPPI_EBUSY while any is pending). */
mppi_status mppi_serve_reset_stats(mppi_server* s);
/* The session's control sequence [T][m] (MPPI_EBUSY while it has requests). */
mppi_status mppi_serve_get_controls(mppi_server* s, int32_t session, float* U_host);

#ifdef __cplusplus
}
#endif

#endif /* MPPI_JUMP_H */
