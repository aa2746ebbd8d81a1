// The cross-block reduction of the update (Eq. App_PI with the min shift; Algorithm 1's
// weighted sum and normaliser) in one fixed arithmetic order, independent of the launch
// shape, so that every path through the merge gives the same bits.
//
// Given the block partials (rho_b, k*_b, eta_b) and the FP32 block sums P_b[o] of
// w_k du_k over the block's samples (w relative to rho_b):
//   rho = min_b rho_b, k* = the lowest index attaining it;
//   s_b = exp(-(rho_b - rho) / lambda) in FP32 (0 when either minimum is not finite);
//   eta = sum_b s_b eta_b in FP64: lane l of one warp sums b = l, l + 32, ... in ascending
//         order, a butterfly adds the lanes, lane 0's sum is taken;
//   N[o] = sum_b s_b P_b[o]: the blocks split into kMergeRanges contiguous ranges of
//         ceil(nblk / kMergeRanges); within a range the terms are added in ascending b, and
//         the range sums in ascending range order, all in double-FP32 arithmetic (each
//         product s_b P_b[o] exact as a float pair through the FMA residual, each sum
//         error-free by Knuth's TwoSum, the residuals gathered in a second float): about
//         48 significant bits, which on B300 costs far less than FP64 (the FP64 pipe runs
//         about 2 FMAs per clock per SM);
//   du[o] = (N.hi + N.lo) / eta in FP64, stored as FP32; U[o] += du[o].
// The explicitly rounded intrinsics keep the compiler from contracting the TwoSum steps
// into FMAs, which would break their exactness.
#pragma once
#include <climits>

#include "mppi_device.cuh"

namespace mppi {

constexpr int kMergeRanges = 8;

// hi + lo, an unevaluated sum of two floats
struct DF {
  float hi, lo;
};

// a += s * x
__device__ __forceinline__ void df_add_prod(DF &a, float s, float x) {
  const float p = __fmul_rn(s, x);
  const float e = __fmaf_rn(s, x, -p);  // s x = p + e exactly
  const float t = __fadd_rn(a.hi, p);
  const float bp = __fsub_rn(t, a.hi);
  const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(t, bp)), __fsub_rn(p, bp));  // a.hi + p = t + err
  a.hi = t;
  a.lo = __fadd_rn(a.lo, __fadd_rn(err, e));
}

// a += b
__device__ __forceinline__ void df_add(DF &a, DF b) {
  const float t = __fadd_rn(a.hi, b.hi);
  const float bp = __fsub_rn(t, a.hi);
  const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(t, bp)), __fsub_rn(b.hi, bp));
  a.hi = t;
  a.lo = __fadd_rn(a.lo, __fadd_rn(err, b.lo));
}

__host__ __device__ __forceinline__ int merge_range_len(int nblk) {
  return (nblk + kMergeRanges - 1) / kMergeRanges;
}

__device__ __forceinline__ float merge_scale(float rho_b, float rho, float inv_lambda) {
  return (isfinite(rho) && isfinite(rho_b)) ? expf(-(rho_b - rho) * inv_lambda) : 0.0f;
}

// eta in the fixed order above; every lane of the calling warp takes part and gets lane 0's sum
__device__ __forceinline__ double merge_eta_warp(const float *s_sc, const double *s_eb, int nblk, int lane) {
  double e = 0.0;
  for (int b = lane; b < nblk; b += 32) e = fma(static_cast<double>(s_sc[b]), s_eb[b], e);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) e = __dadd_rn(e, __shfl_xor_sync(0xffffffffu, e, off));
  return __shfl_sync(0xffffffffu, e, 0);
}

// du[o] from the combined range sums
__device__ __forceinline__ double merge_du(DF tot, double inv_eta) {
  return __dmul_rn(__dadd_rn(static_cast<double>(tot.hi), static_cast<double>(tot.lo)), inv_eta);
}

}  // namespace mppi
