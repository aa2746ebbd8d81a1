// Quadrotor rollout with each sample held by a group of LANES consecutive lanes (LANES = 2 measured
// fastest at K = 8192, T = 150: 173 us per iteration, against 183 us with 4 lanes and 245 us with one).
//
// At K = 8192 one thread per sample gives 256 warps for 592 SM sub-partitions, and most of
// a step is the nearest-cylinder search (64 cylinders) on the path from one state to the
// next (a crash freezes the state).  Here the LANES lanes of a sample all run the same
// RK4 step, split the cylinder search among themselves and combine it with shuffles, and
// take turns drawing the Philox blocks (one per step for m = 4), handed round by shuffles:
// LANES times more warps, a search and a noise share LANES times shorter.  Each lane stores
// M / LANES of the perturbations into the block's du table; lane 0 owns the sample in the
// block softmax partial.  Arithmetic and summation order are those of the one-thread kernel.
#pragma once
#include "rollout_body.cuh"

namespace mppi {

// Shared-memory bytes of rollout_block_quad_lanes (dynamic part) for NS samples per block.
__host__ __device__ inline size_t quad_lanes_smem_bytes(int T, int n_obs, int ns) {
  const size_t TM = static_cast<size_t>(T) * Quad::M;
  return 16 + sizeof(float) * (4 * static_cast<size_t>(n_obs) + 2 * TM + T + ns + TM * ns);
}

template <int BLK, int LANES>
__device__ __forceinline__ void rollout_block_quad_lanes(const CtrlParams &p, const float *__restrict__ x0,
                                                         uint32_t ctr, const float *__restrict__ U, int k0,
                                                         float *__restrict__ S_out, float *__restrict__ part_sums,
                                                         BlockPartial *__restrict__ part, float *smem) {
  constexpr int M = Quad::M, N = Quad::N, NS = BLK / LANES;
  static_assert(M % LANES == 0, "each lane of the group stores M / LANES perturbations");
  static_assert(32 % LANES == 0 && NS % 32 == 0, "lane groups inside a warp; 32-sample columns");
  const int T = p.T, TM = T * M, tid = threadIdx.x;
  float *sObs = smem;              // [n_obs][4] cylinders (16-byte aligned, first)
  float *sU = sObs + 4 * p.n_obs;  // [TM]
  float *sRu = sU + TM;            // [TM]
  float *sHu = sRu + TM;           // [T]
  float *sW = sHu + T;             // [NS]
  float *sDu = sW + NS;            // [TM][NS]
  __shared__ float sx0[N];

  for (int o = tid; o < TM; o += BLK) sU[o] = U[o];
  for (int o = tid; o < 4 * p.n_obs; o += BLK) sObs[o] = (o & 3) == 3 ? 0.0f : p.obs[3 * (o >> 2) + (o & 3)];
  if (tid < N) sx0[tid] = x0[tid];
  __syncthreads();
  for (int i = tid; i < T; i += BLK) {
    float h = 0.0f;
#pragma unroll
    for (int j = 0; j < M; ++j) {
      float ru = 0.0f;
#pragma unroll
      for (int l = 0; l < M; ++l) ru = fmaf(p.R[j * M + l], sU[i * M + l], ru);
      sRu[i * M + j] = ru;
      h = fmaf(sU[i * M + j], ru, h);
    }
    sHu[i] = 0.5f * h;
  }
  __syncthreads();

  const Env env = make_env(p, sObs, 1);
  const int slot = tid / LANES, sub = tid % LANES;
  const int k = k0 + slot;
  float Lnu[M * M], R[M * M];
#pragma unroll
  for (int a = 0; a < M * M; ++a) {
    Lnu[a] = p.Lnu[a];
    R[a] = p.R[a];
  }
  float x[N];
#pragma unroll
  for (int a = 0; a < N; ++a) x[a] = sx0[a];
  Quad::Aux aux;
  aux.crashed = false;
  aux.d = Quad::obstacle_distance_lanes(env, x[0], x[1], sub, LANES);
  KahanSum S;
  // S~ gains q(x_{i+1}) + is_i once per step, in step order (as the one-thread kernel)
  // The normals of step i are Philox block i; lane s of a group draws block i0 + s for the
  // group of LANES steps starting at i0 and hands the others theirs by shuffles.
  const int base = (threadIdx.x & 31) & ~(LANES - 1);
  float eps_mine[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  for (int i = 0; i < T; ++i) {
    const int j = i % LANES;
    if (j == 0)
      normals4(static_cast<uint32_t>(i + sub), static_cast<uint32_t>(k), ctr, p.gid, p.key_lo, p.key_hi, eps_mine);
    float eps[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) eps[c] = __shfl_sync(0xffffffffu, eps_mine[c], base + j);
    float du[M], v[M];
    scale_noise<M>(Lnu, eps, du);
    float duRdu = 0.0f, uRdu = 0.0f;
#pragma unroll
    for (int j = 0; j < M; ++j) {
      v[j] = sU[i * M + j] + du[j];
      uRdu = fmaf(sRu[i * M + j], du[j], uRdu);
      float rd = 0.0f;
#pragma unroll
      for (int l = 0; l < M; ++l) rd = fmaf(R[j * M + l], du[l], rd);
      duRdu = fmaf(du[j], rd, duRdu);
    }
#pragma unroll
    for (int q = 0; q < M / LANES; ++q) {
      float mine = du[0];
#pragma unroll
      for (int j = 1; j < M; ++j) mine = (sub + q * LANES) == j ? du[j] : mine;
      sDu[(i * M + sub + q * LANES) * NS + slot] = mine;
    }
    Quad::step_lanes(x, v, aux, env, p.dt, sub, LANES);
    S.add(Quad::cost(x, aux, env) + (p.is_du * duRdu + uRdu + sHu[i]));
  }
  S.add(Quad::cost(x, aux, env));  // phi(x_T) = q(x_T)
  // the update kernel may start launching now (it waits for this grid's results itself)
  asm volatile("griddepcontrol.launch_dependents;");
  block_partial<M, BLK, false, NS>(p, sub == 0 ? k : INT_MAX, ctr, S.s, Lnu, S_out, part_sums, part, sW, sDu,
                                   sub == 0 ? slot : -1);
}

}  // namespace mppi
