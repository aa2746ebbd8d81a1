// MPPI iteration kernels for sm_103a.
//
// Fused path (two launches per iteration):
//   k_rollout_fused  one thread per sample k.  Philox noise -> du (kept in shared
//                    memory) -> T dynamics steps with the state in registers ->
//                    q + importance-sampling running cost (Kahan FP32) -> phi.
//                    Then, per block: rho_b = min S~, w_k = exp(-(S~_k - rho_b)/lambda),
//                    eta_b = sum w_k (FP64) and the FP32 block sums sum_k w_k du_{i,k}.
//   k_merge_update   merge of the block partials (flash-softmax style):
//                    rho = min rho_b, eta = sum_b eta_b e^{-(rho_b - rho)/lambda} (FP64),
//                    du_i = sum_b e^{-(rho_b-rho)/lambda} part_b[i] / eta (double-FP32
//                    sums in a fixed order, FP64 division; merge_common.cuh); U += du.
// The min shift is exact algebra: it cancels between numerator and denominator of
// Eq. App_PI and only keeps the exponentials in range.
//
// Plain loop (the single-controller baseline): noise -> HBM, rollout reading du
// from HBM, single-block min, single-block normaliser, one block per output for
// the weighted sum (FP64 throughout).
#include <cfloat>
#include <climits>

#include "kernels.cuh"
#include "merge_common.cuh"
#include "rollout_body.cuh"
#include "rollout_lanes.cuh"
#include "rollout_quad_ws.cuh"
#include "rollout_ws.cuh"

namespace mppi {

// ---------------------------------------------------------------------------
// fused rollout: one block of BLK samples per CTA (body in rollout_body.cuh)
// ---------------------------------------------------------------------------
template <class Sys, int BLK, bool REGEN, bool GEN = false>
__global__ void __launch_bounds__(BLK) k_rollout_fused(const CtrlParams p, const float *__restrict__ x0,
                                                       const CtrlState *__restrict__ st, const float *__restrict__ U,
                                                       float *__restrict__ S_out, float *__restrict__ part_sums,
                                                       BlockPartial *__restrict__ part) {
  extern __shared__ __align__(16) float smem[];
  rollout_block<Sys, BLK, REGEN, false, GEN>(p, x0, st->counter, U, p.k_begin + blockIdx.x * BLK, S_out,
                                 part_sums + static_cast<size_t>(blockIdx.x) * p.T * Sys::M, part + blockIdx.x,
                                 smem);
}

// cost-to-go weighting: one thread per sample, du in shared memory, per-step block partials
template <class Sys, int BLK, bool GEN = false>
__global__ void __launch_bounds__(BLK) k_rollout_to_go(const CtrlParams p, const float *__restrict__ x0,
                                                       const CtrlState *__restrict__ st, const float *__restrict__ U,
                                                       float *__restrict__ S_out, float *__restrict__ part_sums,
                                                       BlockPartial *__restrict__ part, float *__restrict__ part_rho,
                                                       DF *__restrict__ part_eta) {
  extern __shared__ __align__(16) float smem[];
  rollout_block<Sys, BLK, false, true, GEN>(p, x0, st->counter, U, p.k_begin + blockIdx.x * BLK, S_out,
                                       part_sums + static_cast<size_t>(blockIdx.x) * p.T * Sys::M, part + blockIdx.x,
                                       smem, nullptr, part_rho + static_cast<size_t>(blockIdx.x) * p.T,
                                       part_eta + static_cast<size_t>(blockIdx.x) * p.T);
}

// car: three threads per sample (velocity recurrence / noise / pose and cost), see rollout_ws.cuh
// (GEN: a general sampling covariance per step)
template <int NS, bool GEN = false>
__global__ void __launch_bounds__(kWsRoles * NS, 1) k_rollout_car_ws(const CtrlParams p, const float *__restrict__ x0,
                                                              const CtrlState *__restrict__ st,
                                                              const float *__restrict__ U, float *__restrict__ S_out,
                                                              float *__restrict__ part_sums,
                                                              BlockPartial *__restrict__ part) {
  extern __shared__ __align__(16) float smem[];
  rollout_block_car_ws<NS, false, GEN>(p, x0, st->counter, U, p.k_begin + blockIdx.x * NS, S_out,
                                       part_sums + static_cast<size_t>(blockIdx.x) * p.T * Car::M, part + blockIdx.x,
                                       smem);
}

// car, cost-to-go weighting: the three warp roles with per-step partials
template <int NS, bool GEN = false>
__global__ void __launch_bounds__(kWsRoles * NS, 1) k_rollout_car_ws_to_go(
    const CtrlParams p, const float *__restrict__ x0, const CtrlState *__restrict__ st, const float *__restrict__ U,
    float *__restrict__ S_out, float *__restrict__ part_sums, BlockPartial *__restrict__ part,
    float *__restrict__ part_rho, DF *__restrict__ part_eta) {
  extern __shared__ __align__(16) float smem[];
  rollout_block_car_ws<NS, true, GEN>(p, x0, st->counter, U, p.k_begin + blockIdx.x * NS, S_out,
                                 part_sums + static_cast<size_t>(blockIdx.x) * p.T * Car::M, part + blockIdx.x, smem,
                                 part_rho + static_cast<size_t>(blockIdx.x) * p.T,
                                 part_eta + static_cast<size_t>(blockIdx.x) * p.T);
}

// quadrotor: noise / RK4 dynamics / crash decisions and cost in three warp roles, see rollout_quad_ws.cuh
template <int NS, bool GEN = false>
__global__ void __launch_bounds__(3 * NS, 1) k_rollout_quad_ws(const CtrlParams p, const float *__restrict__ x0,
                                                               const CtrlState *__restrict__ st,
                                                               const float *__restrict__ U, float *__restrict__ S_out,
                                                               float *__restrict__ part_sums,
                                                               BlockPartial *__restrict__ part) {
  extern __shared__ __align__(16) float smem[];
  rollout_block_quad_ws<NS, GEN>(p, x0, st->counter, U, p.k_begin + blockIdx.x * NS, S_out,
                            part_sums + static_cast<size_t>(blockIdx.x) * p.T * Quad::M, part + blockIdx.x, smem);
}

// quadrotor, cost-to-go weighting: the three warp roles with per-step partials
template <int NS>
__global__ void __launch_bounds__(3 * NS, 1) k_rollout_quad_ws_to_go(
    const CtrlParams p, const float *__restrict__ x0, const CtrlState *__restrict__ st, const float *__restrict__ U,
    float *__restrict__ S_out, float *__restrict__ part_sums, BlockPartial *__restrict__ part,
    float *__restrict__ part_rho, DF *__restrict__ part_eta) {
  extern __shared__ __align__(16) float smem[];
  rollout_block_quad_ws<NS, false, true>(p, x0, st->counter, U, p.k_begin + blockIdx.x * NS, S_out,
                                         part_sums + static_cast<size_t>(blockIdx.x) * p.T * Quad::M, part + blockIdx.x,
                                         smem, part_rho + static_cast<size_t>(blockIdx.x) * p.T,
                                         part_eta + static_cast<size_t>(blockIdx.x) * p.T);
}

// quadrotor: four lanes per sample (shared RK4 step, split cylinder search), see rollout_lanes.cuh
template <int BLK, int LANES>
__global__ void __launch_bounds__(BLK) k_rollout_quad_lanes(const CtrlParams p, const float *__restrict__ x0,
                                                            const CtrlState *__restrict__ st,
                                                            const float *__restrict__ U, float *__restrict__ S_out,
                                                            float *__restrict__ part_sums,
                                                            BlockPartial *__restrict__ part) {
  extern __shared__ __align__(16) float smem[];
  constexpr int NS = BLK / LANES;
  rollout_block_quad_lanes<BLK, LANES>(p, x0, st->counter, U, p.k_begin + blockIdx.x * NS, S_out,
                                       part_sums + static_cast<size_t>(blockIdx.x) * p.T * Quad::M,
                                       part + blockIdx.x, smem);
}

// ---------------------------------------------------------------------------
// FP64 merge of block partials + update of U (+ the shift, into the other control buffer)
// ---------------------------------------------------------------------------
namespace {
constexpr int kMergePrefetch = 16;  // block partials per thread loaded before the reductions
}  // namespace

// One CTA per 32 outputs (i, j), warp r = range r of the block partials (merge_common.cuh:
// the fixed arithmetic order every path shares).  The CTA's loads (block partials, the first
// kMergePrefetch block sums of each lane's range, the controls it updates) are issued first,
// so their latency is paid once; then rho/k* (argmin), the block scales, and beside each other
// eta (a ninth warp, FP64) and the double-FP32 range sums, combined in range order by warp 0.
// SHIFT: Algorithm 1's shift in the same launch.  The controls live in two buffers that the
// shifts alternate: the update reads U and writes the shifted result, u_{i+1} + du_{i+1} into
// slot i and u_init into the last step, to U_next, so no CTA reads what another writes;
// CTA 0 advances the iteration counter.
template <bool SHIFT>
__global__ void __launch_bounds__(kMergeUpdateThreads) k_merge_update(int nblk, int TM, int m, float inv_lambda,
                                                                const float *__restrict__ part_sums,
                                                                const BlockPartial *__restrict__ part,
                                                                float *__restrict__ U, float *__restrict__ U_next,
                                                                float *__restrict__ u0_out,
                                                                float *__restrict__ dU_dbg,
                                                                StepDebug *__restrict__ dbg,
                                                                const float *__restrict__ u_init,
                                                                CtrlState *__restrict__ st,
                                                                unsigned int *__restrict__ u0_ready) {
  constexpr int NW = kMergeRanges;             // warps 0..NW-1: one range of block partials each
  constexpr int NT = kMergeUpdateThreads;      // warp NW: the normaliser
  static_assert(NT == 32 * (NW + 1), "range warps + the normaliser's warp");
  extern __shared__ double s_eb[];  // [nblk] eta_b, then [nblk] floats: rho_b, then s_b
  float *s_sc = reinterpret_cast<float *>(s_eb + nblk);
  __shared__ float s_rho[NW + 1];
  __shared__ int s_k[NW + 1];
  __shared__ DF s_part[NW][kMergeOutputs];
  __shared__ double s_inv_eta;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int o = blockIdx.x * kMergeOutputs + lane;
  const int L = merge_range_len(nblk), b0 = min(nblk, warp * L), b1 = warp < NW ? min(nblk, b0 + L) : b0;
  // launched as a programmatic dependent of the rollout: its partials are complete and
  // visible after this wait (a no-op for an ordinary launch)
  asm volatile("griddepcontrol.wait;" ::: "memory");

  // loads first: the first kMergePrefetch block sums of this lane's output in the warp's range
  float pre[kMergePrefetch];
#pragma unroll
  for (int j = 0; j < kMergePrefetch; ++j) {
    const int b = b0 + j;
    pre[j] = (o < TM && b < b1) ? part_sums[static_cast<size_t>(b) * TM + o] : 0.0f;
  }
  const bool own = warp == 0 && o < TM;  // warp 0 writes the CTA's outputs
  const float u_old = own ? U[o] : 0.0f;
  const float u_last = (SHIFT && warp == 0 && o < m) ? u_init[o] : 0.0f;
  float v = INFINITY;
  int idx = INT_MAX;
  for (int b = tid; b < nblk; b += NT) {
    const BlockPartial bp = part[b];
    s_eb[b] = bp.eta;
    s_sc[b] = bp.rho;
    if (bp.rho < v || (bp.rho == v && bp.kstar < idx)) {
      v = bp.rho;
      idx = bp.kstar;
    }
  }
  warp_argmin(v, idx);
  if (lane == 0) {
    s_rho[warp] = v;
    s_k[warp] = idx;
  }
  __syncthreads();
  if (warp == 0) {
    float vv = lane <= NW ? s_rho[lane] : INFINITY;
    int ii = lane <= NW ? s_k[lane] : INT_MAX;
    warp_argmin(vv, ii);
    if (lane == 0) {
      s_rho[0] = vv;
      s_k[0] = ii;
    }
  }
  __syncthreads();
  const float rho = s_rho[0];
  for (int b = tid; b < nblk; b += NT) s_sc[b] = merge_scale(s_sc[b], rho, inv_lambda);
  __syncthreads();
  // the normaliser (FP64, on B300's slow FP64 pipe) on its own warp, beside the range sums
  if (warp == NW) {
    const double eta = merge_eta_warp(s_sc, s_eb, nblk, lane);
    if (lane == 0) {
      s_inv_eta = eta > 0.0 ? 1.0 / eta : 0.0;
      if (blockIdx.x == 0) {
        dbg->rho = rho;
        dbg->kstar = s_k[0];
        dbg->eta = eta;
      }
    }
  }

  DF acc{0.0f, 0.0f};
#pragma unroll
  for (int j = 0; j < kMergePrefetch; ++j)
    if (b0 + j < b1) df_add_prod(acc, s_sc[b0 + j], pre[j]);
  if (o < TM)
    for (int b = b0 + kMergePrefetch; b < b1; ++b)
      df_add_prod(acc, s_sc[b], part_sums[static_cast<size_t>(b) * TM + o]);
  if (warp < NW) s_part[warp][lane] = acc;
  __syncthreads();
  if (own) {
    DF tot = s_part[0][lane];
#pragma unroll
    for (int r = 1; r < kMergeRanges; ++r) df_add(tot, s_part[r][lane]);
    const double du = merge_du(tot, s_inv_eta);
    const float un = u_old + static_cast<float>(du);
    dU_dbg[o] = static_cast<float>(du);
    if (o < m) u0_out[o] = un;
    if (!SHIFT) {
      U[o] = un;
    } else if (o >= m) {
      U_next[o - m] = un;
    } else {
      U_next[TM - m + o] = u_last;
    }
  }
  // u0 is final: raise the host's flag (u0 in host memory before it) ahead of the rest
  if (u0_ready != nullptr && blockIdx.x == 0 && warp == 0) {
    __syncwarp();
    if (lane == 0) {
      __threadfence_system();
      *reinterpret_cast<volatile unsigned int *>(u0_ready) = 1u;
    }
  }
  if (SHIFT && blockIdx.x == 0 && tid == 0) st->counter += 1u;
}

// ---------------------------------------------------------------------------
// K-sharding: the rank-local reduction and the merge of every rank's partial
// ---------------------------------------------------------------------------
// k_shard_partial reduces this rank's block partials in the merge's fixed order (merge_common.cuh)
// relative to the rank's own minimum, and writes the rank's partial as TM + 3 doubles:
//   [0] rho_r (+inf if no finite cost), [1] k*_r (lowest global sample index attaining it),
//   [2] eta_r = sum_{k in rank} exp(-(S~_k - rho_r)/lambda),
//   [3 + o] N_r[o] = sum_{k in rank} exp(-(S~_k - rho_r)/lambda) du_{o,k}.
// One CTA per 32 outputs, warp r = range r of the block partials.
__global__ void __launch_bounds__(kMergeThreads) k_shard_partial(int nblk, int TM, float inv_lambda,
                                                                 const float *__restrict__ part_sums,
                                                                 const BlockPartial *__restrict__ part,
                                                                 double *__restrict__ out) {
  constexpr int NW = kMergeThreads / 32;
  extern __shared__ double s_eb[];  // [nblk] eta_b, then [nblk] floats: rho_b, then s_b
  float *s_sc = reinterpret_cast<float *>(s_eb + nblk);
  __shared__ float s_rho[NW];
  __shared__ int s_k[NW];
  __shared__ DF s_part[NW][kMergeOutputs];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int o = blockIdx.x * kMergeOutputs + lane;
  const int L = merge_range_len(nblk), b0 = min(nblk, warp * L), b1 = min(nblk, b0 + L);
  float v = INFINITY;
  int idx = INT_MAX;
  for (int b = tid; b < nblk; b += kMergeThreads) {
    const BlockPartial bp = part[b];
    s_eb[b] = bp.eta;
    s_sc[b] = bp.rho;
    if (bp.rho < v || (bp.rho == v && bp.kstar < idx)) {
      v = bp.rho;
      idx = bp.kstar;
    }
  }
  warp_argmin(v, idx);
  if (lane == 0) {
    s_rho[warp] = v;
    s_k[warp] = idx;
  }
  __syncthreads();
  if (warp == 0) {
    float vv = lane < NW ? s_rho[lane] : INFINITY;
    int ii = lane < NW ? s_k[lane] : INT_MAX;
    warp_argmin(vv, ii);
    if (lane == 0) {
      s_rho[0] = vv;
      s_k[0] = ii;
    }
  }
  __syncthreads();
  const float rho = s_rho[0];
  for (int b = tid; b < nblk; b += kMergeThreads) s_sc[b] = merge_scale(s_sc[b], rho, inv_lambda);
  __syncthreads();
  if (warp == 0) {
    const double eta = merge_eta_warp(s_sc, s_eb, nblk, lane);
    if (lane == 0 && blockIdx.x == 0) {
      out[0] = static_cast<double>(rho);
      out[1] = static_cast<double>(s_k[0]);
      out[2] = eta;
    }
  }
  DF acc{0.0f, 0.0f};
  if (o < TM)
    for (int b = b0; b < b1; ++b) df_add_prod(acc, s_sc[b], part_sums[static_cast<size_t>(b) * TM + o]);
  s_part[warp][lane] = acc;
  __syncthreads();
  if (warp == 0 && o < TM) {
    DF tot = s_part[0][lane];
#pragma unroll
    for (int r = 1; r < kMergeRanges; ++r) df_add(tot, s_part[r][lane]);
    out[3 + o] = static_cast<double>(tot.hi) + static_cast<double>(tot.lo);
  }
}

// k_shard_update merges the R rank partials [R][TM + 3] in rank order (FP64):
//   rho = min_r rho_r (lowest k* on ties), s_r = exp(-(rho_r - rho)/lambda),
//   eta = sum_r s_r eta_r, du[o] = sum_r s_r N_r[o] / eta;  U += du, u0 out.
// Every rank runs it on the same gathered partials and gets the same U.
__global__ void __launch_bounds__(256) k_shard_update(const double *__restrict__ all, int R, int TM, int m,
                                                      double inv_lambda, float *__restrict__ U,
                                                      float *__restrict__ u0_out, float *__restrict__ dU_dbg,
                                                      StepDebug *__restrict__ dbg) {
  const int W = TM + 3;
  double rho = INFINITY;
  int ks = INT_MAX;
  for (int r = 0; r < R; ++r) {
    const double rr = all[static_cast<size_t>(r) * W];
    const int kk = static_cast<int>(all[static_cast<size_t>(r) * W + 1]);
    if (rr < rho || (rr == rho && kk < ks)) {
      rho = rr;
      ks = kk;
    }
  }
  double eta = 0.0;
  for (int r = 0; r < R; ++r) {
    const double rr = all[static_cast<size_t>(r) * W];
    const double sr = (isfinite(rho) && isfinite(rr)) ? exp(-(rr - rho) * inv_lambda) : 0.0;
    eta = fma(sr, all[static_cast<size_t>(r) * W + 2], eta);
  }
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o < TM) {
    double n = 0.0;
    for (int r = 0; r < R; ++r) {
      const double rr = all[static_cast<size_t>(r) * W];
      const double sr = (isfinite(rho) && isfinite(rr)) ? exp(-(rr - rho) * inv_lambda) : 0.0;
      n = fma(sr, all[static_cast<size_t>(r) * W + 3 + o], n);
    }
    const double du = eta > 0.0 ? n / eta : 0.0;
    const float un = U[o] + static_cast<float>(du);
    U[o] = un;
    dU_dbg[o] = static_cast<float>(du);
    if (o < m) u0_out[o] = un;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    dbg->rho = static_cast<float>(rho);
    dbg->kstar = ks == INT_MAX ? 0 : ks;
    dbg->eta = eta;
  }
}

// ---------------------------------------------------------------------------
// merge of the per-step block partials of the cost-to-go weighting + update of U (+ the shift)
// ---------------------------------------------------------------------------
// One CTA per 32 outputs o = (i, j); lane = output, warp w takes blocks w, w + 8, ... .  Per
// output:
//   rho_i = min_b rho_{b,i},  s_b = exp(-(rho_{b,i} - rho_i)/lambda) (FP32),
//   eta_i = sum_b s_b eta_{b,i},  N_o = sum_b s_b part_b[o]   (double-FP32, warps combined in
//   order), du_o = N_o / eta_i (FP64), U[o] += du_o.
// CTA 0 also reports step 0's (rho, k*, eta) from the BlockPartials.  SHIFT: Algorithm 1's
// shift as in k_merge_update (the shifted update written to the other control buffer).
template <bool SHIFT>
__global__ void __launch_bounds__(kMergeThreads) k_merge_to_go(int nblk, int T, int m, float inv_lambda,
                                                               const float *__restrict__ part_sums,
                                                               const float *__restrict__ part_rho,
                                                               const DF *__restrict__ part_eta,
                                                               const BlockPartial *__restrict__ part,
                                                               float *__restrict__ U, float *__restrict__ U_next,
                                                               float *__restrict__ u0_out,
                                                               float *__restrict__ dU_dbg,
                                                               StepDebug *__restrict__ dbg,
                                                               const float *__restrict__ u_init,
                                                               CtrlState *__restrict__ st,
                                                               unsigned int *__restrict__ u0_ready) {
  constexpr int NW = kMergeThreads / 32;
  __shared__ float s_r[NW][32];
  __shared__ DF s_e[NW][32], s_a[NW][32];
  __shared__ float s_rho0[NW];
  __shared__ int s_k0[NW];
  __shared__ double s_e0[NW];
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int TM = T * m;
  const int o = blockIdx.x * kMergeOutputs + lane;
  const bool live = o < TM;
  const int i = live ? o / m : 0;
  // loads first: this lane's first kMergePrefetch blocks (b = warp, warp + NW, ...)
  float pr[kMergePrefetch], ps[kMergePrefetch];
  DF pe[kMergePrefetch];
#pragma unroll
  for (int j = 0; j < kMergePrefetch; ++j) {
    const int b = warp + j * NW;
    const bool in = live && b < nblk;
    pr[j] = in ? part_rho[static_cast<size_t>(b) * T + i] : INFINITY;
    ps[j] = in ? part_sums[static_cast<size_t>(b) * TM + o] : 0.0f;
    pe[j] = in ? part_eta[static_cast<size_t>(b) * T + i] : DF{0.0f, 0.0f};
  }
  const float u_old = (warp == 0 && live) ? U[o] : 0.0f;
  const float u_last = (SHIFT && warp == 0 && o < m) ? u_init[o] : 0.0f;
  float r = INFINITY;
#pragma unroll
  for (int j = 0; j < kMergePrefetch; ++j) r = fminf(r, pr[j]);
  for (int b = warp + kMergePrefetch * NW; b < nblk; b += NW) r = fminf(r, part_rho[static_cast<size_t>(b) * T + i]);
  s_r[warp][lane] = r;
  __syncthreads();
  float rho = INFINITY;
#pragma unroll
  for (int q = 0; q < NW; ++q) rho = fminf(rho, s_r[q][lane]);
  DF e{0.0f, 0.0f}, a{0.0f, 0.0f};
  if (live && isfinite(rho)) {
#pragma unroll
    for (int j = 0; j < kMergePrefetch; ++j) {
      if (warp + j * NW >= nblk) break;
      const float sc = isfinite(pr[j]) ? expf(-(pr[j] - rho) * inv_lambda) : 0.0f;
      df_add_prod(e, sc, pe[j].hi);
      e.lo = __fmaf_rn(sc, pe[j].lo, e.lo);
      df_add_prod(a, sc, ps[j]);
    }
    for (int b = warp + kMergePrefetch * NW; b < nblk; b += NW) {
      const float rb = part_rho[static_cast<size_t>(b) * T + i];
      const float sc = isfinite(rb) ? expf(-(rb - rho) * inv_lambda) : 0.0f;
      const DF pq = part_eta[static_cast<size_t>(b) * T + i];
      df_add_prod(e, sc, pq.hi);
      e.lo = __fmaf_rn(sc, pq.lo, e.lo);
      df_add_prod(a, sc, part_sums[static_cast<size_t>(b) * TM + o]);
    }
  }
  s_e[warp][lane] = e;
  s_a[warp][lane] = a;
  __syncthreads();
  if (warp == 0 && live) {
    DF et = s_e[0][lane], at = s_a[0][lane];
#pragma unroll
    for (int q = 1; q < NW; ++q) {
      df_add(et, s_e[q][lane]);
      df_add(at, s_a[q][lane]);
    }
    const double eta = static_cast<double>(et.hi) + static_cast<double>(et.lo);
    const double du = eta > 0.0 ? (static_cast<double>(at.hi) + static_cast<double>(at.lo)) / eta : 0.0;
    const float un = u_old + static_cast<float>(du);
    dU_dbg[o] = static_cast<float>(du);
    if (o < m) u0_out[o] = un;
    if (!SHIFT) {
      U[o] = un;
    } else if (o >= m) {
      U_next[o - m] = un;
    } else {
      U_next[TM - m + o] = u_last;
    }
  }
  // u0 is final: raise the host's flag (u0 in host memory before it) ahead of the rest
  if (u0_ready != nullptr && blockIdx.x == 0 && warp == 0) {
    __syncwarp();
    if (lane == 0) {
      __threadfence_system();
      *reinterpret_cast<volatile unsigned int *>(u0_ready) = 1u;
    }
  }
  if (blockIdx.x == 0) {  // step 0's scalars for the debug surface
    float v = INFINITY;
    int idx = INT_MAX;
    for (int b = tid; b < nblk; b += kMergeThreads) {
      const float rb = part[b].rho;
      const int kk = part[b].kstar;
      if (rb < v || (rb == v && kk < idx)) {
        v = rb;
        idx = kk;
      }
    }
    warp_argmin(v, idx);
    if (lane == 0) {
      s_rho0[warp] = v;
      s_k0[warp] = idx;
    }
    __syncthreads();
    float vv = INFINITY;
    int ii = INT_MAX;
#pragma unroll
    for (int q = 0; q < NW; ++q)
      if (s_rho0[q] < vv || (s_rho0[q] == vv && s_k0[q] < ii)) {
        vv = s_rho0[q];
        ii = s_k0[q];
      }
    double e0 = 0.0;
    if (isfinite(vv))
      for (int b = tid; b < nblk; b += kMergeThreads)
        e0 += (isfinite(part[b].rho) ? static_cast<double>(expf(-(part[b].rho - vv) * inv_lambda)) : 0.0) *
              part[b].eta;
    e0 = warp_sum_d(e0);
    if (lane == 0) s_e0[warp] = e0;
    __syncthreads();
    if (tid == 0) {
      double eta = 0.0;
#pragma unroll
      for (int q = 0; q < NW; ++q) eta += s_e0[q];
      dbg->rho = vv;
      dbg->kstar = (ii == INT_MAX) ? 0 : ii;  // every cost +inf: all tie at rho, the lowest k is 0
      dbg->eta = eta;
    }
  }
  if (SHIFT && blockIdx.x == 0 && tid == 0) st->counter += 1u;
}

// ---------------------------------------------------------------------------
// shift (Algorithm 1): u_i <- u_{i+1}, u_{T-1} <- u_init; counter += 1.  From U into the
// other control buffer U_next.
// ---------------------------------------------------------------------------
__global__ void k_shift(const float *__restrict__ U, float *__restrict__ U_next, const float *__restrict__ u_init,
                        int TM, int m, CtrlState *__restrict__ st) {
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < TM; o += gridDim.x * blockDim.x)
    U_next[o] = (o + m < TM) ? U[o + m] : u_init[o - (TM - m)];
  if (blockIdx.x == 0 && threadIdx.x == 0) st->counter += 1u;
}

// ---------------------------------------------------------------------------
// plain-loop baseline kernels
// ---------------------------------------------------------------------------
template <int M>
__global__ void k_plain_noise(const CtrlParams p, const uint32_t *__restrict__ counter, float *__restrict__ du) {
  constexpr int SPB = 4 / M;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int b = blockIdx.y;
  if (k >= p.K) return;
  float eps[4];
  normals4(static_cast<uint32_t>(b), static_cast<uint32_t>(k), *counter, p.gid, p.key_lo, p.key_hi, eps);
  float Lnu[M * M];
#pragma unroll
  for (int a = 0; a < M * M; ++a) Lnu[a] = p.Lnu[a];
#pragma unroll
  for (int s = 0; s < SPB; ++s) {
    const int i = b * SPB + s;
    if (i < p.T) {
      float d[M];
      scale_noise<M>(Lnu, eps + s * M, d);
#pragma unroll
      for (int j = 0; j < M; ++j) du[static_cast<size_t>(i * M + j) * p.K + k] = d[j];
    }
  }
}

template <class Sys>
__global__ void __launch_bounds__(128) k_plain_rollout(const CtrlParams p, const CtrlState *__restrict__ st,
                                                       const float *__restrict__ U, const float *__restrict__ du,
                                                       float *__restrict__ S_out) {
  constexpr int M = Sys::M, N = Sys::N;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= p.K) return;
  const Env env = make_env(p, p.obs);
  float x[N];
#pragma unroll
  for (int a = 0; a < N; ++a) x[a] = st->x0[a];
  typename Sys::Aux aux;
  Sys::init(x, aux, env);
  KahanSum S;
  for (int i = 0; i < p.T; ++i) {
    float d[M], v[M], u[M];
#pragma unroll
    for (int j = 0; j < M; ++j) {
      u[j] = U[i * M + j];
      d[j] = du[static_cast<size_t>(i * M + j) * p.K + k];
      v[j] = u[j] + d[j];
    }
    float duRdu = 0.0f, uRdu = 0.0f, uRu = 0.0f;
#pragma unroll
    for (int j = 0; j < M; ++j) {
      float rd = 0.0f, ru = 0.0f;
#pragma unroll
      for (int l = 0; l < M; ++l) {
        rd = fmaf(p.R[j * M + l], d[l], rd);
        ru = fmaf(p.R[j * M + l], u[l], ru);
      }
      duRdu = fmaf(d[j], rd, duRdu);
      uRdu = fmaf(ru, d[j], uRdu);
      uRu = fmaf(u[j], ru, uRu);
    }
    Sys::step(x, v, aux, env, p.dt);
    S.add(Sys::cost(x, aux, env) + (p.is_du * duRdu + uRdu + 0.5f * uRu));
  }
  S.add(Sys::cost(x, aux, env));
  const float Sk = S.s;
  S_out[k] = isfinite(Sk) ? Sk : INFINITY;
}

__global__ void __launch_bounds__(1024) k_plain_min(const float *__restrict__ S, int K, StepDebug *__restrict__ dbg) {
  __shared__ float s_v[32];
  __shared__ int s_i[32];
  float v = INFINITY;
  int idx = INT_MAX;
  constexpr int J = 8;  // loads of a pass issued before its comparisons
  for (int k0 = threadIdx.x; k0 < K; k0 += J * blockDim.x) {
    float s[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const int k = k0 + j * blockDim.x;
      s[j] = k < K ? S[k] : INFINITY;
    }
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const int k = k0 + j * blockDim.x;
      if (s[j] < v || (s[j] == v && k < idx)) {
        v = s[j];
        idx = k;
      }
    }
  }
  warp_argmin(v, idx);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    s_v[warp] = v;
    s_i[warp] = idx;
  }
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    v = lane < nw ? s_v[lane] : INFINITY;
    idx = lane < nw ? s_i[lane] : INT_MAX;
    warp_argmin(v, idx);
    if (lane == 0) {
      dbg->rho = v;
      dbg->kstar = (idx == INT_MAX) ? 0 : idx;
    }
  }
}

// The plain loop's reduction (Eq. App_PI with the min shift), unfused and coalesced:
// k_plain_weights forms every w_k = exp(-(S~_k - rho)/lambda) once (FP64 exponential, stored
// rounded to FP32) with per-block FP64 partial sums of eta; k_plain_wsum reads each row of du
// [T*m][K] once, kPlainRows rows by kPlainSplitK samples per block: each thread sums its
// kPlainSplitK / kPlainBlock products per row in FP32, each warp adds its lanes' sums in FP32
// (a fixed tree), the block adds the warp sums in FP64 into per-split partials; k_plain_finalize adds the partials in a fixed order (FP64), divides
// by eta and updates U.  Scratch: w [K] floats (in a K-double slot) | eta partials
// [ceil(K/256)] | wsum partials [splits][T*m] (doubles).
constexpr int kPlainBlock = 256;
constexpr int kPlainRows = 4;
constexpr int kPlainSplitK = 2048;

__global__ void __launch_bounds__(kPlainBlock) k_plain_weights(const float *__restrict__ S, int K, float lambda,
                                                               const StepDebug *__restrict__ dbg,
                                                               float *__restrict__ w, double *__restrict__ eta_part) {
  __shared__ double s_e[kPlainBlock / 32];
  const int k = blockIdx.x * kPlainBlock + threadIdx.x;
  const float rho = dbg->rho;
  double e = 0.0;
  if (k < K) {
    const float Sk = S[k];
    if (isfinite(rho) && isfinite(Sk))
      e = exp(-(static_cast<double>(Sk) - static_cast<double>(rho)) / static_cast<double>(lambda));
    w[k] = static_cast<float>(e);
  }
  e = warp_sum_d(e);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) s_e[warp] = e;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < kPlainBlock / 32; ++q) t += s_e[q];
    eta_part[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(kPlainBlock) k_plain_wsum(const float *__restrict__ du, const float *__restrict__ w,
                                                            int K, int TM, double *__restrict__ part) {
  __shared__ double s_a[kPlainRows][kPlainBlock / 32];
  constexpr int J = kPlainSplitK / kPlainBlock;  // samples per thread
  const int k0 = blockIdx.x * kPlainSplitK, r0 = blockIdx.y * kPlainRows;
  const int k1 = min(K, k0 + kPlainSplitK);
  // every load of the thread issued before the first product (latency paid once)
  float wk[J];
  float dv[kPlainRows][J];
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const int k = k0 + threadIdx.x + j * kPlainBlock;
    wk[j] = k < k1 ? w[k] : 0.0f;
#pragma unroll
    for (int r = 0; r < kPlainRows; ++r)
      dv[r][j] = (k < k1 && r0 + r < TM) ? du[static_cast<size_t>(r0 + r) * K + k] : 0.0f;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int r = 0; r < kPlainRows; ++r) {
    float acc = 0.0f;
#pragma unroll
    for (int j = 0; j < J; ++j) acc = fmaf(wk[j], dv[r][j], acc);
    acc = warp_sum_f(acc);
    if (lane == 0) s_a[r][warp] = static_cast<double>(acc);
  }
  __syncthreads();
  if (threadIdx.x < kPlainRows && r0 + threadIdx.x < TM) {
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < kPlainBlock / 32; ++q) t += s_a[threadIdx.x][q];
    part[static_cast<size_t>(blockIdx.x) * TM + r0 + threadIdx.x] = t;
  }
}

__global__ void __launch_bounds__(kPlainBlock) k_plain_finalize(const double *__restrict__ eta_part, int n_eta,
                                                                const double *__restrict__ part, int n_split, int TM,
                                                                int m, StepDebug *__restrict__ dbg,
                                                                float *__restrict__ U, float *__restrict__ u0_out,
                                                                float *__restrict__ dU_dbg) {
  __shared__ double s_eta;
  if (threadIdx.x == 0) {
    double e = 0.0;
    for (int b = 0; b < n_eta; ++b) e += eta_part[b];
    s_eta = e;
    if (blockIdx.x == 0) dbg->eta = e;
  }
  __syncthreads();
  const double eta = s_eta;
  const int o = blockIdx.x * kPlainBlock + threadIdx.x;
  if (o >= TM) return;
  double t = 0.0;
  for (int b = 0; b < n_split; ++b) t += part[static_cast<size_t>(b) * TM + o];
  const double d = eta > 0.0 ? t / eta : 0.0;
  const float un = U[o] + static_cast<float>(d);
  U[o] = un;
  dU_dbg[o] = static_cast<float>(d);
  if (o < m) u0_out[o] = un;
}

// ---------------------------------------------------------------------------
// debug
// ---------------------------------------------------------------------------
__global__ void k_philox_words(uint32_t key_lo, uint32_t key_hi, int K, int n_blocks, uint32_t counter, uint32_t gid,
                               uint32_t *__restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int b = blockIdx.y;
  if (k >= K || b >= n_blocks) return;
  const Words4 w = philox4x32_10(static_cast<uint32_t>(b), static_cast<uint32_t>(k), counter, gid, key_lo, key_hi);
  uint32_t *o = out + static_cast<size_t>(b) * 4 * K + k;
  o[0] = w.x;
  o[static_cast<size_t>(K)] = w.y;
  o[2 * static_cast<size_t>(K)] = w.z;
  o[3 * static_cast<size_t>(K)] = w.w;
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
size_t fused_smem_bytes(const CtrlParams &p, int blk) {
  if (blk == kFusedBlockCarWs) return car_ws_smem_bytes(p.T, kWsSamples, false, p.gen != nullptr);
  if (blk == kFusedBlockCarWs32) return car_ws_smem_bytes(p.T, kWsSmallSamples, false, p.gen != nullptr);
  if (blk == kFusedBlockQuadLanes) return quad_lanes_smem_bytes(p.T, p.n_obs, kQuadLanesBlock / kQuadLanes);
  if (blk == kFusedBlockQuadWs)
    return quad_ws_smem_bytes(p.T, p.n_obs, kQwsSamples, quad_grid_bytes(p), p.gen != nullptr);
  const bool regen = blk == kFusedBlockRegen;
  return rollout_smem_bytes(p.T, p.m, p.n_obs, regen ? kFusedBlockLarge : blk, regen, false, p.gen != nullptr,
                            quad_grid_bytes(p));
}

int fused_block_size(int sys, const CtrlParams &p) {
  // a small controller: 32 samples per CTA, so that its CTAs spread over the SMs and each
  // role's warp has a scheduler to itself instead of sharing one with the other two roles
  if (sys == 1 && p.T <= kWsChunk * kWsMaxChunks && shard_samples(p) <= kWsSmallMaxK &&
      fused_smem_bytes(p, kFusedBlockCarWs32) <= kFusedSmemLimit)
    return kFusedBlockCarWs32;
  if (sys == 1 && p.T <= kWsChunk * kWsMaxChunks && fused_smem_bytes(p, kFusedBlockCarWs) <= kFusedSmemLimit)
    return kFusedBlockCarWs;
  if (sys == 2 && p.gen && p.T <= kQwsChunk * kQwsMaxChunks && fused_smem_bytes(p, kFusedBlockQuadWs) <= kBigWsSmemLimit)
    return kFusedBlockQuadWs;
  if (p.gen) {  // else the general sampling covariance runs on the one-thread kernels, du in shared memory
    if (fused_smem_bytes(p, kFusedBlockLarge) <= kFusedSmemLimit) return kFusedBlockLarge;
    if (fused_smem_bytes(p, kFusedBlockSmall) <= kFusedSmemLimit) return kFusedBlockSmall;
    return 0;
  }
  if (sys == 2 && p.T <= kQwsChunk * kQwsMaxChunks && fused_smem_bytes(p, kFusedBlockQuadWs) <= kBigWsSmemLimit)
    return kFusedBlockQuadWs;
  if (sys == 2 && fused_smem_bytes(p, kFusedBlockQuadLanes) <= kFusedSmemLimit) return kFusedBlockQuadLanes;
  if (fused_smem_bytes(p, kFusedBlockLarge) <= kFusedSmemLimit) return kFusedBlockLarge;
  if (fused_smem_bytes(p, kFusedBlockSmall) <= kFusedSmemLimit) return kFusedBlockSmall;
  if (fused_smem_bytes(p, kFusedBlockRegen) <= kFusedSmemLimit) return kFusedBlockRegen;
  return 0;
}

int fused_block_samples(int blk) {
  if (blk == kFusedBlockCarWs) return kWsSamples;
  if (blk == kFusedBlockCarWs32) return kWsSmallSamples;
  if (blk == kFusedBlockQuadLanes) return kQuadLanesBlock / kQuadLanes;
  if (blk == kFusedBlockQuadWs) return kQwsSamples;
  return blk == kFusedBlockRegen ? kFusedBlockLarge : blk;
}

template <class Sys, int BLK, bool REGEN>
static cudaError_t launch_fused_t(const CtrlParams &p, const float *x0, const CtrlState *st, const float *U, float *S,
                                  float *ps, BlockPartial *part, cudaStream_t s) {
  const bool gen = p.gen != nullptr;
  const size_t smem = rollout_smem_bytes(p.T, Sys::M, p.n_obs, BLK, REGEN, false, gen, quad_grid_bytes(p));
  const int grid = (shard_samples(p) + BLK - 1) / BLK;
  if (gen) {
    if (REGEN) return cudaErrorInvalidValue;
    k_rollout_fused<Sys, BLK, false, true><<<grid, BLK, smem, s>>>(p, x0, st, U, S, ps, part);
  } else {
    k_rollout_fused<Sys, BLK, REGEN><<<grid, BLK, smem, s>>>(p, x0, st, U, S, ps, part);
  }
  return cudaGetLastError();
}

template <class Sys>
static cudaError_t launch_fused_sys(int blk, const CtrlParams &p, const float *x0, const CtrlState *st, const float *U,
                                    float *S, float *ps, BlockPartial *part, cudaStream_t s) {
  if (blk == kFusedBlockLarge) return launch_fused_t<Sys, kFusedBlockLarge, false>(p, x0, st, U, S, ps, part, s);
  if (blk == kFusedBlockSmall) return launch_fused_t<Sys, kFusedBlockSmall, false>(p, x0, st, U, S, ps, part, s);
  if (blk == kFusedBlockRegen) return launch_fused_t<Sys, kFusedBlockLarge, true>(p, x0, st, U, S, ps, part, s);
  return cudaErrorInvalidValue;
}

template <int NS>
static cudaError_t launch_car_ws(const CtrlParams &p, const float *x0, const CtrlState *st, const float *U, float *S,
                                 float *ps, BlockPartial *part, cudaStream_t s) {
  const size_t smem = car_ws_smem_bytes(p.T, NS, false, p.gen != nullptr);
  const int grid = (shard_samples(p) + NS - 1) / NS;
  if (p.gen)
    k_rollout_car_ws<NS, true><<<grid, kWsRoles * NS, smem, s>>>(p, x0, st, U, S, ps, part);
  else
    k_rollout_car_ws<NS><<<grid, kWsRoles * NS, smem, s>>>(p, x0, st, U, S, ps, part);
  return cudaGetLastError();
}

cudaError_t launch_rollout_fused(int sys, int blk, const CtrlParams &p, const float *x0, const CtrlState *st,
                                 const float *U, float *S, float *part_sums, BlockPartial *part, cudaStream_t s) {
  switch (sys) {
    case 0: return launch_fused_sys<CartPole>(blk, p, x0, st, U, S, part_sums, part, s);
    case 4: return launch_fused_sys<CartPoleVel>(blk, p, x0, st, U, S, part_sums, part, s);
    case 1:
      if (blk == kFusedBlockCarWs) return launch_car_ws<kWsSamples>(p, x0, st, U, S, part_sums, part, s);
      if (blk == kFusedBlockCarWs32) return launch_car_ws<kWsSmallSamples>(p, x0, st, U, S, part_sums, part, s);
      return launch_fused_sys<Car>(blk, p, x0, st, U, S, part_sums, part, s);
    case 2:
      if (blk == kFusedBlockQuadWs) {
        const size_t smem = fused_smem_bytes(p, kFusedBlockQuadWs);
        const int grid = (shard_samples(p) + kQwsSamples - 1) / kQwsSamples;
        if (p.gen)
          k_rollout_quad_ws<kQwsSamples, true><<<grid, 3 * kQwsSamples, smem, s>>>(p, x0, st, U, S, part_sums, part);
        else
          k_rollout_quad_ws<kQwsSamples><<<grid, 3 * kQwsSamples, smem, s>>>(p, x0, st, U, S, part_sums, part);
        return cudaGetLastError();
      }
      if (blk == kFusedBlockQuadLanes) {
        const size_t smem = quad_lanes_smem_bytes(p.T, p.n_obs, kQuadLanesBlock / kQuadLanes);
        const int grid = (shard_samples(p) + kQuadLanesBlock / kQuadLanes - 1) / (kQuadLanesBlock / kQuadLanes);
        k_rollout_quad_lanes<kQuadLanesBlock, kQuadLanes><<<grid, kQuadLanesBlock, smem, s>>>(p, x0, st, U, S,
                                                                                              part_sums, part);
        return cudaGetLastError();
      }
      return launch_fused_sys<Quad>(blk, p, x0, st, U, S, part_sums, part, s);
    default: return cudaErrorInvalidValue;
  }
}

int fused_block_size_to_go(int sys, const CtrlParams &p) {
  const bool gen = p.gen != nullptr;
  if (sys == 1 && p.T <= kWsChunk * kWsMaxChunks && car_ws_smem_bytes(p.T, kWsSamples, true, gen) <= kBigWsSmemLimit)
    return kFusedBlockCarWs;
  if (sys == 2 && !gen && p.T <= kQwsChunk * kQwsMaxChunks &&
      quad_ws_smem_bytes(p.T, p.n_obs, kQwsSamples, quad_grid_bytes(p), false, true) <= kBigWsSmemLimit)
    return kFusedBlockQuadWs;
  if (rollout_smem_bytes(p.T, p.m, p.n_obs, kFusedBlockLarge, false, true, gen, quad_grid_bytes(p)) <= kFusedSmemLimit)
    return kFusedBlockLarge;
  if (rollout_smem_bytes(p.T, p.m, p.n_obs, kFusedBlockSmall, false, true, gen, quad_grid_bytes(p)) <= kFusedSmemLimit)
    return kFusedBlockSmall;
  return 0;
}

template <class Sys, int BLK>
static cudaError_t launch_to_go_t(const CtrlParams &p, const float *x0, const CtrlState *st, const float *U, float *S,
                                  float *ps, BlockPartial *part, float *prho, DF *peta, cudaStream_t s) {
  const bool gen = p.gen != nullptr;
  const size_t smem = rollout_smem_bytes(p.T, Sys::M, p.n_obs, BLK, false, true, gen, quad_grid_bytes(p));
  const int grid = (p.K + BLK - 1) / BLK;
  if (gen)
    k_rollout_to_go<Sys, BLK, true><<<grid, BLK, smem, s>>>(p, x0, st, U, S, ps, part, prho, peta);
  else
    k_rollout_to_go<Sys, BLK><<<grid, BLK, smem, s>>>(p, x0, st, U, S, ps, part, prho, peta);
  return cudaGetLastError();
}

template <class Sys>
static cudaError_t launch_to_go_sys(int blk, const CtrlParams &p, const float *x0, const CtrlState *st,
                                    const float *U, float *S, float *ps, BlockPartial *part, float *prho,
                                    DF *peta, cudaStream_t s) {
  if (blk == kFusedBlockLarge) return launch_to_go_t<Sys, kFusedBlockLarge>(p, x0, st, U, S, ps, part, prho, peta, s);
  if (blk == kFusedBlockSmall) return launch_to_go_t<Sys, kFusedBlockSmall>(p, x0, st, U, S, ps, part, prho, peta, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_rollout_to_go(int sys, int blk, const CtrlParams &p, const float *x0, const CtrlState *st,
                                 const float *U, float *S, float *part_sums, BlockPartial *part, float *part_rho,
                                 DF *part_eta, cudaStream_t s) {
  switch (sys) {
    case 0: return launch_to_go_sys<CartPole>(blk, p, x0, st, U, S, part_sums, part, part_rho, part_eta, s);
    case 4: return launch_to_go_sys<CartPoleVel>(blk, p, x0, st, U, S, part_sums, part, part_rho, part_eta, s);
    case 1:
      if (blk == kFusedBlockCarWs) {
        const size_t smem = car_ws_smem_bytes(p.T, kWsSamples, true, p.gen != nullptr);
        const int grid = (p.K + kWsSamples - 1) / kWsSamples;
        if (p.gen)
          k_rollout_car_ws_to_go<kWsSamples, true><<<grid, kWsRoles * kWsSamples, smem, s>>>(
              p, x0, st, U, S, part_sums, part, part_rho, part_eta);
        else
          k_rollout_car_ws_to_go<kWsSamples><<<grid, kWsRoles * kWsSamples, smem, s>>>(p, x0, st, U, S, part_sums,
                                                                                     part, part_rho, part_eta);
        return cudaGetLastError();
      }
      return launch_to_go_sys<Car>(blk, p, x0, st, U, S, part_sums, part, part_rho, part_eta, s);
    case 2:
      if (blk == kFusedBlockQuadWs) {
        const size_t smem = quad_ws_smem_bytes(p.T, p.n_obs, kQwsSamples, quad_grid_bytes(p), false, true);
        const int grid = (p.K + kQwsSamples - 1) / kQwsSamples;
        k_rollout_quad_ws_to_go<kQwsSamples><<<grid, 3 * kQwsSamples, smem, s>>>(p, x0, st, U, S, part_sums, part,
                                                                                 part_rho, part_eta);
        return cudaGetLastError();
      }
      return launch_to_go_sys<Quad>(blk, p, x0, st, U, S, part_sums, part, part_rho, part_eta, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_merge_to_go(int nblk, const CtrlParams &p, const float *part_sums, const float *part_rho,
                               const DF *part_eta, const BlockPartial *part, float *U, float *u0_out,
                               float *dU_dbg, StepDebug *dbg, cudaStream_t s, bool shift, const float *u_init,
                               CtrlState *st, float *U_next, unsigned int *u0_ready) {
  const int TM = p.T * p.m;
  if (shift && (U_next == nullptr || U_next == U || u_init == nullptr || st == nullptr)) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((TM + kMergeOutputs - 1) / kMergeOutputs, 1, 1);
  cfg.blockDim = dim3(kMergeThreads, 1, 1);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const int T = p.T, m = p.m;
  const float il = p.inv_lambda;
  if (shift)
    return cudaLaunchKernelEx(&cfg, k_merge_to_go<true>, nblk, T, m, il, part_sums, part_rho, part_eta, part, U,
                              U_next, u0_out, dU_dbg, dbg, u_init, st, u0_ready);
  float *no_next = nullptr;
  const float *no_uinit = nullptr;
  CtrlState *no_st = nullptr;
  return cudaLaunchKernelEx(&cfg, k_merge_to_go<false>, nblk, T, m, il, part_sums, part_rho, part_eta, part, U,
                            no_next, u0_out, dU_dbg, dbg, no_uinit, no_st, u0_ready);
}

cudaError_t prepare_kernels() {
  // dynamic shared memory above the 48 KB default, set once (outside any capture)
  const int big = 220 * 1024;
  const void *fns[] = {
      reinterpret_cast<const void *>(k_rollout_fused<CartPole, kFusedBlockLarge, false>),
      reinterpret_cast<const void *>(k_rollout_fused<CartPole, kFusedBlockSmall, false>),
      reinterpret_cast<const void *>(k_rollout_fused<CartPole, kFusedBlockLarge, true>),
      reinterpret_cast<const void *>(k_rollout_fused<CartPoleVel, kFusedBlockLarge, false>),
      reinterpret_cast<const void *>(k_rollout_fused<CartPoleVel, kFusedBlockSmall, false>),
      reinterpret_cast<const void *>(k_rollout_fused<CartPoleVel, kFusedBlockLarge, true>),
      reinterpret_cast<const void *>(k_rollout_to_go<CartPoleVel, kFusedBlockLarge>),
      reinterpret_cast<const void *>(k_rollout_to_go<CartPoleVel, kFusedBlockSmall>),
#define MPPI_GEN_KERNELS(S)                                                              \
  reinterpret_cast<const void *>(k_rollout_fused<S, kFusedBlockLarge, false, true>),   \
      reinterpret_cast<const void *>(k_rollout_fused<S, kFusedBlockSmall, false, true>), \
      reinterpret_cast<const void *>(k_rollout_to_go<S, kFusedBlockLarge, true>),      \
      reinterpret_cast<const void *>(k_rollout_to_go<S, kFusedBlockSmall, true>)
      MPPI_GEN_KERNELS(CartPole), MPPI_GEN_KERNELS(Car), MPPI_GEN_KERNELS(Quad), MPPI_GEN_KERNELS(CartPoleVel),
#undef MPPI_GEN_KERNELS
      reinterpret_cast<const void *>(k_rollout_fused<Car, kFusedBlockLarge, false>),
      reinterpret_cast<const void *>(k_rollout_fused<Car, kFusedBlockSmall, false>),
      reinterpret_cast<const void *>(k_rollout_fused<Car, kFusedBlockLarge, true>),
      reinterpret_cast<const void *>(k_rollout_car_ws<kWsSamples>),
      reinterpret_cast<const void *>(k_rollout_car_ws<kWsSamples, true>),
      reinterpret_cast<const void *>(k_rollout_car_ws_to_go<kWsSamples>),
      reinterpret_cast<const void *>(k_rollout_car_ws_to_go<kWsSamples, true>),
      reinterpret_cast<const void *>(k_rollout_to_go<CartPole, kFusedBlockLarge>),
      reinterpret_cast<const void *>(k_rollout_to_go<CartPole, kFusedBlockSmall>),
      reinterpret_cast<const void *>(k_rollout_to_go<Car, kFusedBlockLarge>),
      reinterpret_cast<const void *>(k_rollout_to_go<Car, kFusedBlockSmall>),
      reinterpret_cast<const void *>(k_rollout_to_go<Quad, kFusedBlockLarge>),
      reinterpret_cast<const void *>(k_rollout_to_go<Quad, kFusedBlockSmall>),
      reinterpret_cast<const void *>(k_rollout_quad_lanes<kQuadLanesBlock, kQuadLanes>),
      reinterpret_cast<const void *>(k_rollout_quad_ws<kQwsSamples>),
      reinterpret_cast<const void *>(k_rollout_quad_ws<kQwsSamples, true>),
      reinterpret_cast<const void *>(k_rollout_quad_ws_to_go<kQwsSamples>),
      reinterpret_cast<const void *>(k_rollout_fused<Quad, kFusedBlockLarge, false>),
      reinterpret_cast<const void *>(k_rollout_fused<Quad, kFusedBlockSmall, false>),
      reinterpret_cast<const void *>(k_rollout_fused<Quad, kFusedBlockLarge, true>),
      reinterpret_cast<const void *>(k_merge_update<false>),
      reinterpret_cast<const void *>(k_merge_update<true>),
      reinterpret_cast<const void *>(k_rollout_car_ws<kWsSmallSamples>),
      reinterpret_cast<const void *>(k_rollout_car_ws<kWsSmallSamples, true>),
  };
  for (const void *f : fns) {
    const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

namespace {
// The path-weighting merge: one CTA per 32 outputs, launched as a programmatic dependent of
// the rollout (its CTAs start while the rollout drains and wait, griddepcontrol.wait, for its
// results).  No thread-block cluster: the shift writes the other control buffer.
template <bool SHIFT>
cudaError_t launch_merge(int nblk, const CtrlParams &p, const float *part_sums, const BlockPartial *part, float *U,
                         float *U_next, float *u0_out, float *dU_dbg, StepDebug *dbg, const float *u_init,
                         CtrlState *st, cudaStream_t s, unsigned int *u0_ready) {
  const int TM = p.T * p.m;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((TM + kMergeOutputs - 1) / kMergeOutputs, 1, 1);
  cfg.blockDim = dim3(kMergeUpdateThreads, 1, 1);
  cfg.dynamicSmemBytes = (sizeof(double) + sizeof(float)) * static_cast<size_t>(nblk);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const int m = p.m;
  const float il = p.inv_lambda;
  return cudaLaunchKernelEx(&cfg, k_merge_update<SHIFT>, nblk, TM, m, il, part_sums, part, U, U_next, u0_out, dU_dbg,
                            dbg, u_init, st, u0_ready);
}
}  // namespace

cudaError_t launch_merge_update(int nblk, const CtrlParams &p, const float *part_sums, const BlockPartial *part,
                                float *U, float *u0_out, float *dU_dbg, StepDebug *dbg, cudaStream_t s,
                                unsigned int *u0_ready) {
  return launch_merge<false>(nblk, p, part_sums, part, U, nullptr, u0_out, dU_dbg, dbg, nullptr, nullptr, s, u0_ready);
}

cudaError_t launch_shard_partial(int nblk, const CtrlParams &p, const float *part_sums, const BlockPartial *part,
                                 double *out, cudaStream_t s) {
  const int TM = p.T * p.m;
  k_shard_partial<<<(TM + kMergeOutputs - 1) / kMergeOutputs, kMergeThreads,
                    (sizeof(double) + sizeof(float)) * static_cast<size_t>(nblk), s>>>(nblk, TM, p.inv_lambda,
                                                                                       part_sums, part, out);
  return cudaGetLastError();
}

cudaError_t launch_shard_update(const CtrlParams &p, const double *all, int n_ranks, float *U, float *u0_out,
                                float *dU_dbg, StepDebug *dbg, cudaStream_t s) {
  const int TM = p.T * p.m;
  k_shard_update<<<(TM + 255) / 256, 256, 0, s>>>(all, n_ranks, TM, p.m, 1.0 / static_cast<double>(p.lambda), U,
                                                  u0_out, dU_dbg, dbg);
  return cudaGetLastError();
}

cudaError_t launch_merge_update_shift(int nblk, const CtrlParams &p, const float *part_sums, const BlockPartial *part,
                                      float *U, float *U_next, float *u0_out, float *dU_dbg, StepDebug *dbg,
                                      const float *u_init, CtrlState *st, cudaStream_t s, unsigned int *u0_ready) {
  if (U_next == nullptr || U_next == U || u_init == nullptr || st == nullptr) return cudaErrorInvalidValue;
  return launch_merge<true>(nblk, p, part_sums, part, U, U_next, u0_out, dU_dbg, dbg, u_init, st, s, u0_ready);
}

cudaError_t launch_shift(const CtrlParams &p, const float *U, float *U_next, const float *u_init, CtrlState *st,
                         cudaStream_t s) {
  if (U_next == nullptr || U_next == U) return cudaErrorInvalidValue;
  const int TM = p.T * p.m;
  k_shift<<<(TM + 1023) / 1024, 1024, 0, s>>>(U, U_next, u_init, TM, p.m, st);
  return cudaGetLastError();
}

cudaError_t launch_plain_noise(const CtrlParams &p, const uint32_t *counter, float *du, cudaStream_t s) {
  const int nb = (p.T * p.m + 3) / 4;
  const dim3 grid((p.K + 255) / 256, nb);
  switch (p.m) {
    case 1: k_plain_noise<1><<<grid, 256, 0, s>>>(p, counter, du); break;
    case 2: k_plain_noise<2><<<grid, 256, 0, s>>>(p, counter, du); break;
    case 4: k_plain_noise<4><<<grid, 256, 0, s>>>(p, counter, du); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_plain_rollout(int sys, const CtrlParams &p, const CtrlState *st, const float *U, const float *du,
                                 float *S, cudaStream_t s) {
  const int grid = (p.K + 127) / 128;
  switch (sys) {
    case 0: k_plain_rollout<CartPole><<<grid, 128, 0, s>>>(p, st, U, du, S); break;
    case 4: k_plain_rollout<CartPoleVel><<<grid, 128, 0, s>>>(p, st, U, du, S); break;
    case 1: k_plain_rollout<Car><<<grid, 128, 0, s>>>(p, st, U, du, S); break;
    case 2: k_plain_rollout<Quad><<<grid, 128, 0, s>>>(p, st, U, du, S); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

size_t plain_scratch_doubles(const CtrlParams &p) {
  const size_t TM = static_cast<size_t>(p.T) * p.m;
  const size_t n_eta = (p.K + kPlainBlock - 1) / kPlainBlock, n_split = (p.K + kPlainSplitK - 1) / kPlainSplitK;
  return static_cast<size_t>(p.K) + n_eta + n_split * TM;
}

cudaError_t launch_plain_reduce_update(const CtrlParams &p, const float *S, const float *du, float *U, float *u0_out,
                                       float *dU_dbg, StepDebug *dbg, double *scratch, cudaStream_t s) {
  const int TM = p.T * p.m;
  const int n_eta = (p.K + kPlainBlock - 1) / kPlainBlock, n_split = (p.K + kPlainSplitK - 1) / kPlainSplitK;
  float *w = reinterpret_cast<float *>(scratch);
  double *eta_part = scratch + p.K, *part = eta_part + n_eta;
  k_plain_min<<<1, 1024, 0, s>>>(S, p.K, dbg);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_plain_weights<<<n_eta, kPlainBlock, 0, s>>>(S, p.K, p.lambda, dbg, w, eta_part);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_plain_wsum<<<dim3(n_split, (TM + kPlainRows - 1) / kPlainRows), kPlainBlock, 0, s>>>(du, w, p.K, TM, part);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_plain_finalize<<<(TM + kPlainBlock - 1) / kPlainBlock, kPlainBlock, 0, s>>>(eta_part, n_eta, part, n_split, TM, p.m,
                                                                                 dbg, U, u0_out, dU_dbg);
  return cudaGetLastError();
}

cudaError_t launch_philox_words(uint32_t key_lo, uint32_t key_hi, int K, int n_blocks, uint32_t counter,
                                uint32_t gid, uint32_t *out, cudaStream_t s) {
  const dim3 grid((K + 255) / 256, n_blocks);
  k_philox_words<<<grid, 256, 0, s>>>(key_lo, key_hi, K, n_blocks, counter, gid, out);
  return cudaGetLastError();
}

}  // namespace mppi
