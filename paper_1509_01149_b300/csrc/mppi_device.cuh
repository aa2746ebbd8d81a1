// Device primitives of the MPPI hot path: counter-based noise, compensated sums,
// warp reductions and the kernel argument blocks.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mppi {

constexpr int kMaxM = 4;   // largest control dimension of the built-in systems
constexpr int kMaxN = 16;  // largest state dimension (padded)

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64-bit
// multiplies on the counter, key bumped by the Weyl increments between rounds.
// ---------------------------------------------------------------------------
struct Words4 {
  uint32_t x, y, z, w;
};

__device__ __forceinline__ Words4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  return Words4{c0, c1, c2, c3};
}

// 23 random bits, centred in their cell: exact in FP32, inside [2^-24, 1 - 2^-24].
__device__ __forceinline__ float unit_uniform(uint32_t w) {
  return (static_cast<float>(w >> 9) + 0.5f) * 1.1920928955078125e-07f;  // 2^-23
}

// Box-Muller on one pair of words: rad = sqrt(-2 ln ua), angle 2 pi ub.  The radicand is at
// least 2^-23 (ua <= 1 - 2^-24), a normal number, so the square root is taken as s * rsqrt(s)
// (a few ulp, no special-case branch).  The angle is taken half a turn back,
// 2 pi (ub - 1/2) in [-pi, pi) (ub - 1/2 is exact), where the special-function-unit sine and
// cosine are accurate to about 2^-21 absolute: cos(2 pi ub) = -cos(2 pi (ub - 1/2)), and the
// same for the sine.  The normals are then within ~rad * 6e-7 absolute.
__device__ __forceinline__ void box_muller(uint32_t wa, uint32_t wb, float &e0, float &e1) {
  const float s2 = -2.0f * logf(unit_uniform(wa));
  const float rad = s2 * rsqrtf(s2);
  float s, c;
  __sincosf(6.28318530717958648f * (unit_uniform(wb) - 0.5f), &s, &c);
  e0 = -rad * c;
  e1 = -rad * s;
}

// Four standard normals of Philox block (b, k, counter, gid).
__device__ __forceinline__ void normals4(uint32_t b, uint32_t k, uint32_t counter, uint32_t gid,
                                         uint32_t key_lo, uint32_t key_hi, float e[4]) {
  const Words4 w = philox4x32_10(b, k, counter, gid, key_lo, key_hi);
  box_muller(w.x, w.y, e[0], e[1]);
  box_muller(w.z, w.w, e[2], e[3]);
}

// ---------------------------------------------------------------------------
// Packed FP32 (sm_100 and later): one instruction carries two independent round-to-nearest
// FP32 operations, each rounding exactly as the scalar fmaf / + / * of its own operands.
// Pairing two independent chains halves their issue slots and changes no result.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }

// Kahan-compensated FP32 accumulator for the path cost.
struct KahanSum {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float v) {
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
};

// ---------------------------------------------------------------------------
// warp helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// (value, index) minimum, lowest index on ties; +inf values never win over finite ones.
__device__ __forceinline__ void warp_argmin(float &v, int &idx) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float ov = __shfl_xor_sync(0xffffffffu, v, o);
    const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
    if (ov < v || (ov == v && oi < idx)) {
      v = ov;
      idx = oi;
    }
  }
}

// ---------------------------------------------------------------------------
// argument blocks
// ---------------------------------------------------------------------------
// Per-controller constants (by value in the kernel argument space).
struct CtrlParams {
  int K, T, m, n;
  float dt, nu, lambda, inv_lambda;
  float is_du;              // (1 - 1/nu) / 2: weight of du^T R du in q~
  float Lnu[kMaxM * kMaxM]; // sqrt(nu) * chol(Sigma), row-major lower triangle
  float R[kMaxM * kMaxM];   // control-cost matrix, row-major
  uint32_t key_lo, key_hi, gid;
  // environment
  const float *map;         // car cost map [H][W]
  int map_w, map_h;
  float map_ox, map_oy, map_inv_cell;
  const float *obs;         // quadrotor cylinders [n_obs][3]
  int n_obs;
  // quadrotor: uniform grid of nearest-cylinder candidate lists over the forest (built on the
  // host, forest_grid.h); grid_nx == 0: none, every query searches all cylinders
  const unsigned short *grid_off;  // [grid_nx * grid_ny + 1] list starts in grid_idx
  const unsigned char *grid_idx;   // [grid_nidx] cylinder indices, cell by cell
  int grid_nx, grid_ny, grid_nidx;
  float grid_ox, grid_oy, grid_inv_h;  // cell (ix, iy) covers [ox + ix/inv_h, ox + (ix+1)/inv_h) x ...
  float goal[3];
  const void *mlp;          // learned dynamics weights (car_mlp)
  const float *gen;         // general sampling covariance: [T][2][m][m] = (chol(Sigma_E,i),
                            // R - lambda Sigma_E,i^-1) per step, row-major; null: nu Sigma
  // K-sharding: this context rolls out the samples [k_begin, k_begin + k_count) of the K
  // (global sample indices, so the noise is the unsharded controller's); k_count 0: to K
  int k_begin, k_count;
};

// Samples this context rolls out.
__host__ __device__ inline int shard_samples(const CtrlParams &p) {
  return p.k_count > 0 ? p.k_count : p.K - p.k_begin;
}

// Per-controller mutable device state.
struct CtrlState {
  float x0[kMaxN];   // current state (written by the step's H2D copy)
  uint32_t counter;  // iteration counter c (Philox counter word 2)
  uint32_t pad[3];
};

// Per-block partial of the fused rollout (flash-softmax style merge later).
struct BlockPartial {
  double eta;    // sum over the block of exp(-(S~ - rho_b)/lambda), FP64
  float rho;     // block minimum of S~ (+inf if none finite)
  int kstar;     // lowest sample index attaining rho
};

// Learned-dynamics weights on the device (BF16 tiles in the K-major core-matrix layout
// the tensor-core kernel copies verbatim into shared memory).
struct MlpDev {
  const unsigned char *w1;  // 256 x 16 tile
  const unsigned char *w2;  // 256 x 256 tile
  const unsigned char *w3;  // 16 x 256 tile
  const float *b1, *b2, *b3;
  float out_scale[8];
  float w_scale[4];         // per-tensor weight scales of W1, W2, W3 (1 for BF16)
  int *err;                 // set to 1 when a bounded tensor-core wait runs out
  int precision, pad;
};

// Results of the last iteration for the debug ABI.
struct StepDebug {
  double eta;
  float rho;
  int kstar;
};

}  // namespace mppi
