// Host-side launchers of the MPPI kernels (implemented in kernels.cu).
#pragma once
#include <cuda_runtime.h>
#include "merge_common.cuh"
#include "mppi_device.cuh"

namespace mppi {

// Block sizes the fused rollout is built for.
constexpr int kFusedBlockLarge = 128;
constexpr int kFusedBlockSmall = 64;
constexpr int kFusedBlockRegen = 129;   // code for "128 samples, du regenerated (no shared-memory copy)"
constexpr int kFusedBlockCarWs = 257;   // code for "car, 128 samples, three threads per sample"
constexpr int kFusedBlockCarWs32 = 258;  // code for "car, 32 samples, three threads per sample" (small K)
constexpr int kWsSmallSamples = 32;
constexpr int kWsSmallMaxK = 148 * kWsSmallSamples;  // up to one 32-sample CTA per SM of a B300
constexpr int kFusedBlockQuadLanes = 513;  // code for "quadrotor, 32 samples, a group of lanes per sample"
constexpr int kFusedBlockQuadWs = 1025;    // code for "quadrotor, 64 samples, three warp roles"
constexpr int kQuadLanesBlock = 64, kQuadLanes = 2;
constexpr int kMinBlockSamples = kQuadLanesBlock / kQuadLanes;  // fewest samples per block of any shape
constexpr int kMergeThreads = 256;
constexpr int kMergeUpdateThreads = kMergeThreads + 32;  // k_merge_update: + the normaliser's warp
constexpr int kMergeOutputs = 32;       // outputs (i, j) per merge block
constexpr size_t kFusedSmemLimit = 200 * 1024;
// the warp-role kernels whose per-step tables (the car's step costs, the quadrotor's
// per-step covariances) take them past kFusedSmemLimit
constexpr size_t kBigWsSmemLimit = 220 * 1024;

// Raise the dynamic shared-memory limit of the kernels that need it (once per
// device, before any launch or capture).
cudaError_t prepare_kernels();

// Fused path ---------------------------------------------------------------
// Shared memory of the fused rollout for block size blk (bytes).
size_t fused_smem_bytes(const CtrlParams &p, int blk);
// Block shape for a controller of system sys: for the car kFusedBlockCarWs and for the
// quadrotor kFusedBlockQuadWs (else kFusedBlockQuadLanes) when their shared memory fits; else
// 128 or 64 samples with
// du kept in shared memory, else kFusedBlockRegen (128 samples, du regenerated); 0 if
// nothing fits.
int fused_block_size(int sys, const CtrlParams &p);
// Samples per block of a block shape.
int fused_block_samples(int blk);
// Rollout + cost + IS term + block-local weights and weighted perturbation sums.
// x0: device state [n] read at launch time (the ctx's own copy or the caller's buffer);
// st: iteration counter.
cudaError_t launch_rollout_fused(int sys, int blk, const CtrlParams &p, const float *x0, const CtrlState *st,
                                 const float *U, float *S, float *part_sums, BlockPartial *part, cudaStream_t s);
// Cross-block merge (FP64 normaliser, double-FP32 sums in a fixed order): rho, kstar, eta,
// du; U += du; u0 out.  u0_ready (optional, mapped host memory): set to 1 once u0_out holds
// u0 (visible to the host before the flag), ahead of the kernel's remaining work.
cudaError_t launch_merge_update(int nblk, const CtrlParams &p, const float *part_sums, const BlockPartial *part,
                                float *U, float *u0_out, float *dU_dbg, StepDebug *dbg, cudaStream_t s,
                                unsigned int *u0_ready = nullptr);
// The merge and the shift of Algorithm 1 in one launch.  The controls live in two buffers
// that the shifts alternate: U (read) and U_next (written with the shifted update, u_init in
// the last step); U_next must not alias U.
cudaError_t launch_merge_update_shift(int nblk, const CtrlParams &p, const float *part_sums, const BlockPartial *part,
                                      float *U, float *U_next, float *u0_out, float *dU_dbg, StepDebug *dbg,
                                      const float *u_init, CtrlState *st, cudaStream_t s,
                                      unsigned int *u0_ready = nullptr);
// Cost-to-go weighting (Eq. App_PI per time step): block shape (the car's warp roles,
// kFusedBlockCarWs, when their shared memory fits kBigWsSmemLimit; else 128 or 64 samples,
// du and the step costs in shared memory; 0 if they do not fit), the rollout with per-step
// block partials
// (part_rho / part_eta [nblk][T]) and their FP64 merge + update.
int fused_block_size_to_go(int sys, const CtrlParams &p);
cudaError_t launch_rollout_to_go(int sys, int blk, const CtrlParams &p, const float *x0, const CtrlState *st,
                                 const float *U, float *S, float *part_sums, BlockPartial *part, float *part_rho,
                                 DF *part_eta, cudaStream_t s);
// The merge of the per-step partials and the update; with `shift` also Algorithm 1's shift in
// the same launch, from U into U_next as for launch_merge_update_shift.  u0_ready as for
// launch_merge_update.
cudaError_t launch_merge_to_go(int nblk, const CtrlParams &p, const float *part_sums, const float *part_rho,
                               const DF *part_eta, const BlockPartial *part, float *U, float *u0_out,
                               float *dU_dbg, StepDebug *dbg, cudaStream_t s, bool shift = false,
                               const float *u_init = nullptr, CtrlState *st = nullptr, float *U_next = nullptr,
                               unsigned int *u0_ready = nullptr);
// Shift of Algorithm 1 from U into the other control buffer U_next, and the iteration counter
// increment.
cudaError_t launch_shift(const CtrlParams &p, const float *U, float *U_next, const float *u_init, CtrlState *st,
                         cudaStream_t s);

// Learned car dynamics (mlp_rollout.cu) -----------------------------------------
constexpr size_t kMlpSmemLimit = 225 * 1024;
constexpr int kMlpMaxT = 500;
size_t mlp_rollout_smem_bytes(int T, int precision);
cudaError_t prepare_mlp_kernel();
// precision 0: BF16 weights and activations; 1: E4M3 (FP8) with per-tensor weight scales
cudaError_t launch_rollout_mlp(const CtrlParams &p, const float *x0, const CtrlState *st, const float *U, float *S,
                               float *part_sums, BlockPartial *part, int precision, cudaStream_t s);

// Plain-loop baseline ---------------------------------------------------------
cudaError_t launch_plain_noise(const CtrlParams &p, const uint32_t *counter, float *du, cudaStream_t s);
cudaError_t launch_plain_rollout(int sys, const CtrlParams &p, const CtrlState *st, const float *U,
                                 const float *du, float *S, cudaStream_t s);
// K-sharding (kernels.cu): the rank's partial [TM + 3] doubles, and the merge of R of them.
constexpr int kShardAlign = 128;  // shard boundaries: multiples of every rollout block's sample count
cudaError_t launch_shard_partial(int nblk, const CtrlParams &p, const float *part_sums, const BlockPartial *part,
                                 double *out, cudaStream_t s);
cudaError_t launch_shard_update(const CtrlParams &p, const double *all, int n_ranks, float *U, float *u0_out,
                                float *dU_dbg, StepDebug *dbg, cudaStream_t s);
// Scratch (doubles) of the plain loop's reduction for this configuration.
size_t plain_scratch_doubles(const CtrlParams &p);
cudaError_t launch_plain_reduce_update(const CtrlParams &p, const float *S, const float *du, float *U,
                                       float *u0_out, float *dU_dbg, StepDebug *dbg, double *scratch, cudaStream_t s);

// Debug ------------------------------------------------------------------------
cudaError_t launch_philox_words(uint32_t key_lo, uint32_t key_hi, int K, int n_blocks, uint32_t counter,
                                uint32_t gid, uint32_t *out, cudaStream_t s);

}  // namespace mppi
