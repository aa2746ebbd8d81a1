/*
 * mppi.h -- C ABI of the B300 (sm_103a) MPPI library.
 *
 * One MPPI iteration with covariance-variable importance sampling (Williams,
 * Aldrich, Theodorou, "Model Predictive Path Integral Control using Covariance
 * Variable Importance Sampling"):
 *
 *   noise     du_{i,k} = sqrt(nu) chol(Sigma) eps_{i,k}          Theorem 1 with A = sqrt(nu) I (Sec. III-C)
 *   rollout   x_{i+1} = F(x_i, u_i + du_{i,k}),  i = 0..T-1       Algorithm 1 (Sec. IV); Euler step of Sec. II-A
 *   cost      S~_k = phi(x_T) + sum_i q~_i,
 *             q~_i = q(x_{i+1}) + (1-1/nu)/2 du^T R du + u^T R du + 1/2 u^T R u   reduced q~ of Sec. III-C
 *   weights   rho = min_k S~_k,  eta = sum_k exp(-(S~_k - rho)/lambda)
 *   update    u_i <- u_i + sum_k exp(-(S~_k - rho)/lambda) du_{i,k} / eta          Eq. App_PI (Sec. III-C)
 *   send/shift  u_0 out; u_i <- u_{i+1}, u_{T-1} <- u_init                         Algorithm 1
 *
 * Conventions shared by every call:
 *   - Return value: MPPI_OK (0) or a negative MPPI_E* code.  Nothing throws across
 *     the ABI.  mppi_last_error() gives the text of the last failure of a ctx.
 *   - Ownership: every input array is copied before the call returns; outputs go
 *     to caller-owned buffers.  The ctx owns all device memory it allocates and
 *     frees it in mppi_destroy().
 *   - Pointers named h_* (or documented "host") are host memory; d_* are device
 *     memory on the ctx's device.  Arrays are dense, row-major, float32 unless
 *     stated.  U is [T][m] (time-major), du and noise are [T][m][K] (K fastest).
 *   - A ctx is not thread-safe: one host thread at a time.  All device work of a
 *     ctx goes to its stream (mppi_set_stream); by default a non-blocking stream
 *     the ctx creates on the device that is current at mppi_create.
 *   - Floating point: rollouts and path costs in FP32 (Kahan-compensated sum);
 *     the normaliser eta and the cross-block sums of the weighted perturbation in
 *     FP64; controls stored in FP32.
 */
#ifndef MPPI_B300_H
#define MPPI_B300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define MPPI_OK 0
#define MPPI_EINVAL (-1)   /* bad argument: null pointer, size out of range, not SPD, ...  */
#define MPPI_ENOMEM (-2)   /* device or pinned host allocation failed                      */
#define MPPI_ECUDA (-3)    /* a CUDA runtime call failed (text in mppi_last_error)          */
#define MPPI_ETIMEOUT (-4) /* a bounded device-side wait ran out (serving)                  */
#define MPPI_ESTATE (-5)   /* call not valid in the ctx's current state (e.g. no env set)   */
#define MPPI_ENOSYS (-6)   /* feature not built into this library                           */
#define MPPI_EBUSY (-7)    /* admission refused: no free slot or not enough arena memory     */
#define MPPI_EAGAIN (-8)   /* a submitted step request has not finished yet (serving poll)   */

/* systems (plants and their state costs; see the design notes for the models) */
typedef enum {
  MPPI_CARTPOLE = 0, /* n=4 (x, xdot, theta, thetadot), m=1 cart force; Euler          */
  MPPI_CAR = 1,      /* n=7 (X, Y, psi, vx, vy, r, delta), m=2 (steer, throttle); Euler;
                        cost map lookup + (vx-7)^2 (speed term of Sec. V-B)              */
  MPPI_QUAD = 2,     /* n=12 (p, v, roll/pitch/yaw, body rates), m=4 rotor thrusts; RK4;
                        cost of Sec. V-C with crash weight 1e4                          */
  MPPI_CAR_MLP = 3,  /* MPPI_CAR's cost with learned dynamics x' = x + MLP([x; u])       */
  MPPI_CARTPOLE_VEL = 4 /* the cart-pole of Sec. V-A: n=4 (p, pdot, theta, thetadot), theta = 0
                           hanging down; m=1 desired cart velocity, pddot = 10 (u - pdot); Euler;
                           q = p^2 + 500 (1 + cos theta)^2 + thetadot^2 + pdot^2            */
} mppi_system;

/* implementation of mppi_step */
typedef enum {
  MPPI_IMPL_FUSED = 0, /* default: one fused rollout+cost+block-reduction kernel, one merge
                          kernel, both in a CUDA graph                                     */
  MPPI_IMPL_PLAIN = 1  /* baseline "plain loop": noise kernel writes du to HBM, separate
                          rollout, min, normaliser and weighted-sum kernels, a stream sync
                          after each step, no graph                                        */
} mppi_impl;

/* weighting of the update (Eq. App_PI) */
typedef enum {
  MPPI_WEIGHT_PATH = 0,  /* default: one total path cost S~_k weights every u_i (Algorithm 1) */
  MPPI_WEIGHT_TO_GO = 1  /* u_i weighted by each rollout's cost-to-go from t_i onward,
                            S~(tau_{i,k}) = sum_{j >= i} q~_{j,k} + phi(x_T), with its own
                            minimum and normaliser per i (Eq. App_PI read literally)        */
} mppi_weighting;

typedef struct mppi_ctx mppi_ctx;

/* Create a controller (Algorithm 1's "Given" block: K, N=T, dt, nu, Sigma, R, lambda).
 *   sys      plant and cost
 *   K        samples, 1 <= K <= 1048576
 *   T        horizon steps, 1 <= T <= 1024
 *   dt       integration step [s], > 0
 *   nu       exploration variance factor (A = sqrt(nu) I), > 0.  nu = 1 is plain MPPI.
 *   lambda   temperature, > 0
 *   Sigma    host [m][m] natural control-noise covariance, symmetric positive
 *            semi-definite (copied).  The perturbation covariance is nu * Sigma.
 *   R        host [m][m] control-cost matrix, symmetric positive definite (copied), or
 *            NULL for R = lambda * Sigma^-1 (the noise/cost relation of Sec. II), which
 *            then needs Sigma positive definite.
 *   out      receives the ctx.
 * Initial state: U = 0, u_init = 0, seed 0, controller id 0, iteration counter 0.
 * Errors: EINVAL (ranges, non-SPD), ENOMEM, ECUDA.  *out is NULL on failure. */
int mppi_create(mppi_system sys, int K, int T, float dt, float nu, float lambda,
                const float *Sigma, const float *R, mppi_ctx **out);

/* Free every device and host resource of the ctx.  NULL is accepted. */
int mppi_destroy(mppi_ctx *ctx);

/* One MPPI iteration from state h_state (host [n], copied): noise, rollout, cost,
 * weights and update of U (not the shift).  Writes the updated u_0 to h_u0_out
 * (host [m]).  Blocks until u_0 is on the host: on the fused path with the path-cost
 * weighting the update kernel raises a flag in mapped host memory as soon as u_0 is
 * there, and the call returns while the rest of the iteration (the write of U, a shift)
 * may still run on the ctx's stream; every later call on the ctx is ordered after it,
 * and an error of that remainder is returned by the next call that synchronises.
 * ESTATE if the system needs an environment (car: cost map; quadrotor: forest;
 * car_mlp: map + weights) that was not set. */
int mppi_step(mppi_ctx *ctx, const float *h_state, float *h_u0_out);

/* One pass of Algorithm 1's loop body from host buffers: the iteration of mppi_step,
 * u_0 to h_u0_out (host [m]), then the shift of mppi_shift (u_i <- u_{i+1},
 * u_{T-1} <- u_init, iteration counter += 1).  Blocks until u_0 is on the host, as
 * mppi_step does (the shift is ordered before every later call on the ctx).  Same errors
 * as mppi_step.  On the fused path this is one CUDA graph in which the shift runs inside
 * the update's launch when T*m <= 256. */
int mppi_step_shift(mppi_ctx *ctx, const float *h_state, float *h_u0_out);

/* Same iteration, asynchronous on the ctx stream, device pointers: d_state [n] is
 * read, d_u0_out [m] written (may be NULL), when the stream reaches the work.  No
 * host sync.  Equivalent to mppi_rollout_async followed by mppi_update_async. */
int mppi_step_async(mppi_ctx *ctx, const float *d_state, float *d_u0_out);

/* The two phases of mppi_step_async, for callers that interleave their own work
 * (events, other streams) between them:
 *   mppi_rollout_async  copy d_state [n] into the ctx, then noise + rollout + cost
 *                       (fused: one kernel that also forms the block partials of the
 *                       weights; plain: noise kernel + rollout kernel).
 *   mppi_update_async   min / normaliser / weighted sum and U update (fused: the FP64
 *                       merge kernel; plain: min, normaliser and weighted-sum kernels),
 *                       then copy u_0 to d_u0_out [m] if it is not NULL.
 * update must follow rollout on the same stream. */
int mppi_rollout_async(mppi_ctx *ctx, const float *d_state);
int mppi_update_async(mppi_ctx *ctx, float *d_u0_out);

/* One receding-horizon iteration on device buffers: mppi_step_async followed by
 * mppi_shift, launched as one CUDA graph (captured on the first call, and again when
 * d_state / d_u0_out or the ctx configuration change).  d_u0_out may be NULL.
 * Asynchronous on the ctx stream (the legacy stream runs the three launches directly). */
int mppi_iterate_async(mppi_ctx *ctx, const float *d_state, float *d_u0_out);

/* Shift (Algorithm 1): u_i <- u_{i+1}, u_{T-1} <- u_init, iteration counter += 1.
 * Asynchronous on the ctx stream. */
int mppi_shift(mppi_ctx *ctx);

/* Noise seed (Philox key = (seed & 0xffffffff, seed >> 32)) and controller id g (the
 * fourth Philox counter word).  The normal of sample k, time i, control j at
 * iteration counter c is lane (r & 3) of Philox4x32-10 block (r >> 2, k, c, g),
 * r = i*m + j; words w become u = ((w >> 9) + 1/2) 2^-23; Box-Muller on lanes
 * (0,1) and (2,3). */
int mppi_set_seed(mppi_ctx *ctx, uint64_t seed);
int mppi_set_controller_id(mppi_ctx *ctx, uint32_t gid);
int mppi_set_iteration(mppi_ctx *ctx, uint32_t counter);
int mppi_get_iteration(mppi_ctx *ctx, uint32_t *counter);

/* Stream for all device work of the ctx (a cudaStream_t on the ctx's device). */
int mppi_set_stream(mppi_ctx *ctx, void *cuda_stream);

/* Select the fused path (default) or the plain-loop baseline.  EINVAL for the plain loop
 * while the cost-to-go weighting or per-step sampling covariances are selected. */
int mppi_set_impl(mppi_ctx *ctx, mppi_impl impl);

/* Per-step sampling covariances Sigma_E [T][m][m] (host, row-major, each symmetric positive
 * definite; copied) in place of nu * Sigma: Theorem 1 with a general A_t in control space.
 * The noise of step i is chol(Sigma_E,i) eps and the likelihood-ratio running term becomes
 * 1/2 du^T (R - lambda Sigma_E,i^-1) du + u_i^T R du + 1/2 u_i^T R u_i (with Sigma_E,i = nu Sigma
 * the (1 - 1/nu)/2 form).  The covariances stay indexed by horizon step across shifts.  NULL
 * restores nu * Sigma.  Fused path only, one thread per sample with du and the per-step
 * matrices in shared memory.  Errors: EINVAL (not symmetric / not positive definite; learned
 * dynamics; plain loop selected; horizon too long for the shared memory), ENOMEM. */
int mppi_set_sampling_covariance(mppi_ctx *ctx, const float *h_Sigma_E);

/* Select the weighting of the update (mppi_weighting).  MPPI_WEIGHT_TO_GO runs on the fused
 * path only, with one thread per sample and du and the per-step costs kept in shared memory
 * (4*T*(m+1) bytes per sample); the update and the shift are then two launches.
 * Errors: EINVAL (unknown mode; learned dynamics; plain loop selected; horizon too long for
 * the shared memory), ENOMEM. */
int mppi_set_weighting(mppi_ctx *ctx, int mode);

/* Nominal control sequence, host [T][m] (copied in / out; get synchronises). */
int mppi_set_controls(mppi_ctx *ctx, const float *h_U);
int mppi_get_controls(mppi_ctx *ctx, float *h_U);

/* u_init: value new controls are initialised to by the shift, host [m]. */
int mppi_set_u_init(mppi_ctx *ctx, const float *h_u);

/* Environment of the system, host blob (copied):
 *   MPPI_CAR / MPPI_CAR_MLP cost map: mppi_env_map header followed by
 *     width*height float32 values, row-major [iy][ix]; node (ix, iy) is at world
 *     (origin_x + ix*cell, origin_y + iy*cell); lookups are bilinear, clamped to the grid.
 *   MPPI_QUAD forest: mppi_env_forest header followed by n_obstacles rows of
 *     float32 (cx, cy, radius) (vertical cylinders), at most 256 rows.
 * The blob kind must match the system; EINVAL otherwise. */
#define MPPI_ENV_MAP 0x3150414du    /* "MAP1" */
#define MPPI_ENV_FOREST 0x31524f46u /* "FOR1" */
#define MPPI_ENV_MLP 0x31504c4du    /* "MLP1" */
typedef struct {
  uint32_t kind; /* MPPI_ENV_MAP */
  int32_t width, height;
  float origin_x, origin_y, cell;
} mppi_env_map;
typedef struct {
  uint32_t kind; /* MPPI_ENV_FOREST */
  int32_t n_obstacles;
  float goal[3];
  float pad;
} mppi_env_forest;
/*   MPPI_CAR_MLP also needs the learned dynamics: mppi_env_mlp header followed by
 *     MPPI_MLP_NUM_PARAMS float32 parameters (layout of the mppi_mlp_* functions);
 *     converted to tensor-core tiles on the device.  precision 0 = BF16 weights and
 *     activations; 1 = E4M3 (FP8) weights with per-tensor scales (largest |w| -> 448)
 *     and E4M3 activations; FP32 accumulation either way. */
typedef struct {
  uint32_t kind; /* MPPI_ENV_MLP */
  int32_t precision;
  float out_scale[7];
  float pad;
} mppi_env_mlp;
int mppi_set_env(mppi_ctx *ctx, const void *blob, size_t bytes);

/* Results of the last mppi_step, host outputs (any may be NULL); synchronises.
 *   S      [K]   path costs S~ (non-finite costs reported as +inf)
 *   argmin       lowest k with S~_k = rho
 *   eta          sum_k exp(-(S~_k - rho)/lambda) (FP64)
 *   dU     [T][m] the weighted perturbation sum_k w_k du_{i,k} that was added to U */
int mppi_get_debug(mppi_ctx *ctx, float *S, int *argmin, double *eta, float *dU);

/* The perturbations du of iteration counter `counter`, recomputed on the device by
 * the same noise code as the rollout, host [T][m][K] out. */
int mppi_get_noise(mppi_ctx *ctx, uint32_t counter, float *h_du);

/* Raw Philox4x32-10 words on the device, for checking the generator:
 * out[b][4][k] for blocks b < n_blocks, samples k < K, counter (b, k, counter, gid),
 * key (seed lo, seed hi).  h_out is host uint32 [n_blocks][4][K]. */
int mppi_philox_words(uint64_t seed, int K, int n_blocks, uint32_t counter, uint32_t gid,
                      uint32_t *h_out);

/* ---- K-sharding: one controller's K samples over R ranks (data parallel) --------------
 * The samples of one iteration are independent (the sampling loop of Algorithm 1), so rank r
 * rolls out a contiguous range of them and the ranks exchange one small partial each:
 *   1. every rank: mppi_set_shard(ctx, k_begin_r, k_count_r) once (global sample indices, so
 *      the noise is the unsharded controller's; boundaries multiples of 128 except at K);
 *   2. every rank: mppi_shard_partial_async(ctx, d_state, d_partial_r) -- rollout of the
 *      rank's samples and its partial, TM + 3 doubles (TM = T*m):
 *        [0] rho_r = min over the rank's S~ (+inf if none is finite), [1] k*_r (lowest global
 *        index attaining it), [2] eta_r = sum_k exp(-(S~_k - rho_r)/lambda),
 *        [3 + o] N_r[o] = sum_k exp(-(S~_k - rho_r)/lambda) du_{o,k}   (o = i*m + j);
 *   3. the caller gathers the R partials in rank order into d_partials [R][TM + 3] on every
 *      rank (one all-gather of (TM + 3) * R doubles);
 *   4. every rank: mppi_shard_update_async(ctx, d_partials, R, d_u0_out) merges them in rank
 *      order (FP64: rho = min rho_r, s_r = exp(-(rho_r - rho)/lambda), eta = sum_r s_r eta_r,
 *      du = sum_r s_r N_r / eta -- Eq. App_PI with the min shift), updates U and writes u_0;
 *      every rank holds the same U; then mppi_shift as usual.
 * The result equals the unsharded iteration's up to the order of the FP64 sums.  With a
 * shard set, mppi_step and the other iteration calls run the shard's samples alone.  Fused
 * path, path weighting, analytic dynamics only (EINVAL otherwise).  All calls are
 * asynchronous on the ctx stream; pointers named d_* are device memory. */
int mppi_set_shard(mppi_ctx *ctx, int k_begin, int k_count);
int mppi_shard_partial_async(mppi_ctx *ctx, const float *d_state, double *d_partial);
int mppi_shard_update_async(mppi_ctx *ctx, const double *d_partials, int n_ranks, float *d_u0_out);

/* One MPPI iteration that allocates nothing (no ctx, no cudaMalloc, no pinned memory)./* One MPPI iteration that allocates nothing (no ctx, no cudaMalloc, no pinned memory).
 * The paper has no counterpart: this is a service for callers that may not allocate
 * device memory while they run -- a real-time control loop that must not call
 * cudaMalloc after start-up (it can synchronise the device and its latency has no
 * bound), or a host whose own memory pool owns all device memory.
 *
 * It does what mppi_step_async does (noise, rollout, cost, weights, update of U, u_0
 * out; not the shift) on buffers the caller owns:
 *   sys                the cart-pole (either form), the car or the quadrotor; MPPI_CAR_MLP
 *                      (learned dynamics) is refused with MPPI_EINVAL
 *   K, T, dt, nu, lambda, h_Sigma, h_R   as in mppi_create, with the same checks (host
 *                      arrays, copied; h_R NULL gives R = lambda Sigma^-1)
 *   seed, gid, counter Philox key, controller id, iteration counter
 *   h_env_header       host mppi_env_map (car) or mppi_env_forest (quadrotor); NULL for
 *                      the cart-pole
 *   d_env_payload      device: the map values [height][width] or the cylinder rows [n][3]
 *                      (float32), read by the kernels
 *   env_payload_bytes  size of the caller's d_env_payload buffer; a header that needs more
 *                      (4*width*height or 12*n bytes) is refused with MPPI_EINVAL
 *   d_state            device [n] state, read
 *   d_U                device [T][m] nominal controls, updated in place
 *   d_u0_out           device [m] updated u_0
 *   cuda_stream        stream for all work (cudaStream_t, may be NULL = legacy stream)
 *   h_err, err_len     optional host buffer that receives the error text (may be NULL)
 * The work is enqueued on cuda_stream and not waited for.  For the same inputs the
 * cart-pole and the car give the bits mppi_step gives; the quadrotor searches every
 * cylinder where a ctx uses its nearest-cylinder grid (the same distances, to rounding).
 *
 * Scratch: a static device array of MPPI_STATIC_SCRATCH_BYTES (4 MiB) inside the
 * library, which every GPU that loads the library holds until the process exits.
 * A configuration needs about 4*K + 4*ceil(K/B)*T*m bytes (B = 128, or 64 when
 * T*m*128 floats would not fit in shared memory) plus a few KB; larger ones return
 * MPPI_EINVAL with the sizes in the error text.  Every call on a device shares the
 * array and leaves the last call's contents in it, so calls whose work overlaps on
 * the GPU (two streams, two host threads) race.  The first call on each device looks
 * up the array's device address and sets kernel attributes (once per device, retried
 * if it failed); make that first call before any stream capture. */
#define MPPI_STATIC_SCRATCH_BYTES (4u << 20)
int mppi_step_static(mppi_system sys, int K, int T, float dt, float nu, float lambda, const float *h_Sigma,
                     const float *h_R, uint64_t seed, uint32_t gid, uint32_t counter, const void *h_env_header,
                     const float *d_env_payload, size_t env_payload_bytes, const float *d_state, float *d_U,
                     float *d_u0_out, void *cuda_stream, char *h_err, size_t err_len);

/* ---------------------------------------------------------------------------------
 * Serving: many controllers of different systems, K and T stepped together.
 * (An extension beyond the paper, which runs one controller.)
 *
 * A server owns a device arena (allocated once at create) and a device slot table.
 * mppi_server_admit places a controller in a free slot if its buffers fit in the arena
 * (first-fit, coalescing free list): admission is by memory, and a refusal returns
 * MPPI_EBUSY, which is not an error.  A controller's U, u_init, Philox key / id and
 * iteration counter stay on the device from admission to release.
 *
 * mppi_server_tick runs, for the listed slots, one MPPI iteration followed by the
 * shift of Algorithm 1 (receding horizon), all slots in the same two persistent
 * kernels (rollout work items = (slot, block of samples), heaviest first, taken from
 * an atomic queue; then one merge + update + shift per slot), replayed as one CUDA
 * graph.  Every slot's result equals what a lone mppi_ctx with the same
 * configuration, seed, controller id and iteration counter computes.
 * --------------------------------------------------------------------------------- */
typedef struct mppi_server mppi_server;

/* Configuration of one controller (host struct, copied by admit).  Sigma and R are
 * row-major m x m in their first m*m entries; has_R = 0 selects R = lambda Sigma^-1.
 * env_id names an environment set with mppi_server_set_env (-1: none, cart-pole). */
typedef struct {
  int32_t system, K, T;
  float dt, nu, lambda;
  float Sigma[16];
  float R[16];
  int32_t has_R;
  int32_t env_id;
  uint64_t seed;
  uint32_t gid;
  uint32_t counter; /* initial iteration counter */
  float u_init[4];
} mppi_slot_config;

typedef struct {
  int32_t max_slots, active_slots;
  uint64_t arena_bytes, arena_used;
  int32_t rollout_block, rollout_ctas_per_sm; /* shapes in use (from the autotuner)   */
  int32_t ticks;
  double last_tick_ms;
} mppi_server_info;

/* max_slots in [1, 4096]; arena_bytes of device memory for the controllers' buffers. */
int mppi_server_create(int max_slots, size_t arena_bytes, mppi_server **out);
int mppi_server_destroy(mppi_server *srv);
/* Environment env_id in [0, 16): same blob formats as mppi_set_env (copied). */
int mppi_server_set_env(mppi_server *srv, int env_id, const void *blob, size_t bytes);
/* Admit a controller: *slot_out receives its slot.  U starts at u_init repeated.
 * MPPI_EBUSY when no slot is free or its buffers do not fit in the arena. */
int mppi_server_admit(mppi_server *srv, const mppi_slot_config *cfg, int *slot_out);
int mppi_server_release(mppi_server *srv, int slot);
int mppi_server_set_controls(mppi_server *srv, int slot, const float *h_U);
int mppi_server_get_controls(mppi_server *srv, int slot, float *h_U);
/* Results of the slot's last tick, host outputs (any may be NULL); synchronises the server:
 *   S [K] path costs S~ (non-finite as +inf), argmin the lowest k attaining rho, eta the
 *   FP64 normaliser sum_k exp(-(S~_k - rho)/lambda) -- as mppi_get_debug for a ctx. */
int mppi_server_get_debug(mppi_server *srv, int slot, float *h_S, int *argmin, double *eta);
/* One receding-horizon step of the n listed slots: h_states [n][16] (state in the first
 * n_x entries of each row), h_u0_out [n][4] receives each slot's u_0 (first m entries).
 * Blocks until the results are on the host. */
int mppi_server_tick(mppi_server *srv, int n, const int *slots, const float *h_states, float *h_u0_out);
/* Pick the rollout block shape and persistent grid by timing the current mix
 * (tick on the listed slots, restoring their controls and counters afterwards). */
int mppi_server_autotune(mppi_server *srv, int n, const int *slots, const float *h_states);
int mppi_server_get_info(mppi_server *srv, mppi_server_info *out);
/* Text of the server's last error (or of the last failed mppi_server_create when srv is NULL). */
const char *mppi_server_last_error(mppi_server *srv);

/* ---- Asynchronous serving: submit / poll / cancel (continuous batching) ----------------
 * mppi_server_start launches the server's scheduler thread.  From then on a step request
 * (one receding-horizon iteration + shift of one admitted controller from a given state) is
 * submitted with mppi_server_submit and returns at once with a request id.  The scheduler
 * batches queued requests into ticks -- at most one per controller and tick, at most
 * max_batch per tick (0: no limit) -- and keeps two ticks in the GPU's queue: while one runs,
 * the requests that arrived meanwhile are filled into the other tick's buffers and enqueued
 * behind it, so requests that arrive while others are on the GPU join the next tick without
 * waiting for a host round trip.  Requests of one controller run in submission order.  A
 * request's result is the u_0 the synchronous mppi_server_tick (and a lone mppi_ctx with the
 * same configuration, seed, controller id and iteration counter) gives for the same state.
 *
 * While the scheduler runs, mppi_server_admit, _release, _set_env, _get_controls,
 * _set_controls and _get_debug may be called from any thread (one lock guards the host
 * state; admission uploads go on a separate copy stream and do not wait for ticks in flight;
 * control and debug copies are ordered after every tick already enqueued).  A slot released
 * while a tick in flight uses it has its queued requests cancelled and its memory returned to
 * the arena when that tick retires.  mppi_server_tick and mppi_server_autotune return
 * MPPI_ESTATE while the scheduler runs (tune first, then start). */
typedef struct {
  int32_t running, pad;
  int64_t queued;     /* submitted, not yet on the GPU                       */
  int64_t in_flight;  /* in a tick on the GPU                                */
  int64_t ticks;      /* ticks the scheduler has retired                      */
  int64_t completed;  /* requests those ticks finished                        */
} mppi_server_stats;

/* Start the scheduler thread.  ESTATE if it already runs. */
int mppi_server_start(mppi_server *srv, int max_batch);
/* Batching of the scheduler: whenever the GPU has no tick, the queued requests are launched
 * at once; while a tick runs, the next tick is formed when the running tick is predicted to
 * end within 0.25 ms (its work, sum of K*T per controller weighted by system, times the
 * GPU time per unit of work of the recent ticks), or once min_batch (>= 1) requests wait, or
 * once the oldest has waited max_wait_ms (>= 0) -- so that it gathers what arrives while the
 * GPU is busy and is enqueued just before the GPU would go idle.  Defaults 1024 and 4.0 ms.
 * May be called at any time. */
int mppi_server_set_batching(mppi_server *srv, int min_batch, double max_wait_ms);
/* Finish every submitted request, then stop the thread.  Safe when it is not running. */
int mppi_server_stop(mppi_server *srv);
/* Queue one step of the controller in `slot` from h_state (host [16], state in the first n
 * entries, copied).  *id_out receives the request id (ids are never reused).  ESTATE if the
 * scheduler is not running; EINVAL for a slot that is not admitted; EBUSY past 2^20
 * outstanding requests. */
int mppi_server_submit(mppi_server *srv, int slot, const float *h_state, uint64_t *id_out);
/* mppi_server_submit for n requests at once (one lock, one wake-up): slot_ids [n],
 * h_states [n][16], ids_out [n].  All or none are queued (EINVAL / EBUSY / ESTATE as above). */
int mppi_server_submit_batch(mppi_server *srv, int n, const int *slot_ids, const float *h_states, uint64_t *ids_out);
/* MPPI_OK and u_0 into h_u0 (host [4], first m entries) if the request has finished (the id
 * is then forgotten), MPPI_EAGAIN if not yet, the tick's error status if it failed, EINVAL
 * for an unknown (never issued, already taken or cancelled) id. */
int mppi_server_poll(mppi_server *srv, uint64_t id, float *h_u0);
/* As poll, but waits up to timeout_ms for the request to finish (ETIMEOUT after that). */
int mppi_server_wait(mppi_server *srv, uint64_t id, double timeout_ms, float *h_u0);
/* Take up to max_n finished requests in completion order, waiting up to timeout_ms for the
 * first: ids [max_n], h_u0 [max_n][4], status [max_n] (may be NULL: MPPI_OK or the tick's
 * error per request), latency_ms [max_n] (may be NULL: from the submission to the moment the
 * scheduler saw its tick finish); *n_out receives how many (0 after the timeout). */
int mppi_server_reap(mppi_server *srv, int max_n, uint64_t *ids, float *h_u0, int *status, double *latency_ms,
                     double timeout_ms, int *n_out);
/* Forget a request.  Queued: it never runs (the controller's controls and iteration counter
 * are untouched).  In flight: its tick completes (the controller's controls and counter
 * advance, every other request of the tick is unaffected) and the result is dropped.
 * Finished: the result is dropped.  EINVAL for an unknown id. */
int mppi_server_cancel(mppi_server *srv, uint64_t id);
int mppi_server_get_stats(mppi_server *srv, mppi_server_stats *out);

/* ---------------------------------------------------------------------------------
 * Learned car dynamics (an extension beyond the paper).
 *   features  z (16) = (X/20, Y/20, wrap(psi)/pi, (vx-5)/5, vy/2, r/3, delta/0.5,
 *             u_steer/1.6, u_throttle/1.8, 0 ...), psi wrapped to (-pi, pi]
 *   network   h1 = tanh(W1 z + b1), h2 = tanh(W2 h1 + b2), y = W3 h2 + b3
 *   step      x' = x + y[0:7] * out_scale
 * Parameters: one flat float array of MPPI_MLP_NUM_PARAMS values, W1 [256][16], b1 [256],
 * W2 [256][256], b2 [256], W3 [16][256], b3 [16] (row = output unit).
 * Training and prediction run on the tensor cores (tcgen05, BF16 operands, FP32
 * accumulation); the FP32 master weights are updated by Adam.
 * --------------------------------------------------------------------------------- */
#define MPPI_MLP_NUM_PARAMS 74256
typedef struct mppi_mlp mppi_mlp;
/* Random initial weights (uniform +-1/sqrt(fan_in), zero biases) from `seed`. */
int mppi_mlp_create(uint64_t seed, mppi_mlp **out);
int mppi_mlp_destroy(mppi_mlp *mlp);
/* Host parameters in (copied; resets the Adam state) / out; out_scale [7] may be NULL. */
int mppi_mlp_set_params(mppi_mlp *mlp, const float *h_params, const float *h_out_scale);
int mppi_mlp_get_params(mppi_mlp *mlp, float *h_params, float *h_out_scale);
/* Training set from device (state [n][7], control [n][2]) pairs: the analytic car step
 * (dt) gives each next state on the GPU; out_scale becomes the per-state standard
 * deviation of the increments.  The pairs are only read during the call. */
int mppi_mlp_set_data(mppi_mlp *mlp, const float *d_states, const float *d_controls, int n, float dt);
/* `steps` Adam steps (learning rate lr) on random batches of `batch` rows (multiple of
 * 128) drawn with Philox under `seed`; h_loss_trace [steps] receives each batch loss
 * (may be NULL; recording it synchronises every step). */
int mppi_mlp_train(mppi_mlp *mlp, int steps, int batch, float lr, uint64_t seed, float *h_loss_trace);
/* Loss and gradients of one batch: d_X [B][16] BF16 features, d_T [B][16] FP32 targets
 * (normalised increments; entries 7..15 ignored), both 16-byte aligned (MPPI_EINVAL
 * otherwise).  h_grads [MPPI_MLP_NUM_PARAMS]. */
int mppi_mlp_grad(mppi_mlp *mlp, const void *d_X, const float *d_T, int B, float *h_grads, double *h_loss);
/* One learned step for n device (state [n][7], control [n][2]) pairs into d_next [n][7]. */
int mppi_mlp_predict(mppi_mlp *mlp, const float *d_states, const float *d_controls, int n, float *d_next);
const char *mppi_mlp_last_error(mppi_mlp *mlp);
/* The analytic car step (the learned model's fallback and yardstick): d_next [n][7] from
 * device (state [n][7], control [n][2]) pairs, enqueued on `stream` (NULL = legacy). */
int mppi_car_step(const float *d_states, const float *d_controls, int n, float dt, float *d_next, void *stream);

/* Check hook for the tensor-core GEMM used by the learned-dynamics training step:
 * C[m*ldc + n] = sum_k A[m*sam + k*sak] * B[k*sbk + n*sbn] on device buffers (A, B BF16,
 * C FP32), BN the output tile width (multiple of 16, <= 256).  Synchronises.
 * Returns 0, MPPI_EINVAL, MPPI_ENOMEM, MPPI_ECUDA or MPPI_ETIMEOUT (a bounded wait ran out). */
int mppi_debug_gemm_bf16(int M, int N, int K, const void *dA, int64_t sam, int64_t sak, const void *dB, int64_t sbk,
                         int64_t sbn, float *dC, int64_t ldc, int BN);

/* Check hook of the bounded-wait exit path of the tensor-core kernels: one GEMM CTA whose MMA
 * issuer issues nothing, so its mbarrier wait gives up after `polls` polls (1 .. 2^20); the
 * kernel raises its error flag, waits once more (bounded), frees its TMEM and returns, with no
 * MMA or bulk copy outstanding.  Returns MPPI_ETIMEOUT (the expected outcome), MPPI_OK if the
 * wait did not run out, MPPI_EINVAL, MPPI_ENOMEM or MPPI_ECUDA.  Synchronises the device. */
int mppi_debug_gemm_wait_timeout(uint32_t polls);

/* Host-side fault injection for tests of the out-of-memory paths: with after_n >= 0 the
 * device or pinned allocation of mppi_create / mppi_server_create that follows after_n
 * successful ones fails (once) with MPPI_ENOMEM as if CUDA had refused it; after_n < 0
 * disarms it.  Process-wide; always returns MPPI_OK. */
int mppi_debug_fail_allocations(int after_n);

/* Check hook for the quadrotor's nearest-cylinder grid (host only, no GPU needed).  Builds
 * the grid that mppi_set_env builds for the forest obs [n_obs][3] (x, y, radius; n_obs in
 * [1, 256]) and, for each of the n_points host points (px[i], py[i]), writes the distance
 * to the nearest cylinder surface, sqrt((x - cx)^2 + (y - cy)^2) - r in FP32, minimised over
 * the candidate list of the point's cell (d_grid[i]) and over every cylinder (d_all[i]), and
 * in_grid[i] = 1 when the point lies inside the grid (else 0 and d_grid[i] = d_all[i]).
 * Caller-owned host buffers.  Returns 0, or MPPI_EINVAL for bad arguments or when no grid
 * fits its caps. */
int mppi_debug_forest_nearest(const float *obs, int n_obs, int n_points, const float *px, const float *py,
                              float *d_grid, float *d_all, int *in_grid);

/* Text of the last error on this ctx (or of the last failed create when ctx is NULL).
 * Valid until the next call on the ctx. */
const char *mppi_last_error(mppi_ctx *ctx);

/* Library version string. */
const char *mppi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MPPI_B300_H */
