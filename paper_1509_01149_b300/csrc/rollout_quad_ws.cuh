// Quadrotor rollout with each sample's work split over warps in three roles (warp
// specialisation), for the forest task of Sec. V-B.
//
// A crash freezes the state at its last valid value (the step that would cross a cylinder
// surface, the ground or the pitch limit is discarded) and the dynamics never read the
// obstacles.  So the RK4 chain can run ahead unconditionally: a role that integrates
// x_{i+1} = RK4(x_i, u_i + du_i) for every step, crashed or not, hands each new state to a
// role that takes every crash decision itself (nearest cylinder, ground, pitch limit,
// finiteness) and keeps its own copy of the frozen state.  The states the dynamics produce
// after a crash are simply never used, so the costs are those of the sequential step:
// same arithmetic, same order.
//
// A CTA owns NS samples with 3 NS threads in three warp-uniform roles:
//   noise     (threads 0..NS-1)        Philox block i -> du_i = sqrt(nu) L eps (m = 4),
//                                      ahead of the others;
//   dynamics  (threads NS..2NS-1)      the RK4 chain, nothing else;
//   cost      (threads 2NS..3NS-1)     the nearest cylinder (searched over its grid cell's
//                                      candidate list, forest_grid.h), crash logic, q(x),
//                                      the importance-sampling terms and S~ (Kahan).
// Shared memory carries the hand-offs in chunks of C steps:
//   du   [T*M][NS]       noise -> dynamics and cost, one single-use mbarrier per chunk (also
//                        the operand of the block sums)
//   ring [R][C][P][NS]   dynamics -> cost: per step the P = 8 state values the cost role
//                        reads (p, v, pitch, yaw; px replaced by NaN when any component of
//                        the new state is not finite), full/empty mbarriers
// With TOGO (the per-time-step cost-to-go weighting) the cost role also keeps each step's
// term of S~ in sC [T][NS] and its terminal cost, and the block forms per-step partials; the
// hand-off chunks are then 4 steps, so that the table fits beside du.
// With GEN (a general sampling covariance per step, Theorem 1) the noise role scales step
// i's normals by chol(Sigma_E,i) and the cost role's IS term is 1/2 du^T (R - lambda
// Sigma_E,i^-1) du + u^T R du + 1/2 u^T R u, the per-step matrices staged in sGen.
// Every wait is bounded; a thread whose wait runs out stops and its sample's cost is +inf.
#pragma once
#include "rollout_body.cuh"
#include "tc_common.cuh"

namespace mppi {

constexpr int kQwsSamples = 64;  // samples per CTA (3x threads)
constexpr int kQwsChunk = 8;     // steps per hand-off (4 with the cost-to-go weighting)
constexpr int kQwsRing = 3;      // chunks in the state ring (2 with the per-step tables)
constexpr int kQwsMaxChunks = 32;  // noise barriers: T <= 256 (64 barriers of 4 steps with TOGO)
__host__ __device__ constexpr int quad_ws_chunk(bool to_go) { return to_go ? kQwsChunk / 2 : kQwsChunk; }
__host__ __device__ constexpr int quad_ws_ring(bool to_go, bool gen) { return (to_go || gen) ? kQwsRing - 1 : kQwsRing; }
constexpr int kQwsPass = 8;      // values per step handed from the dynamics to the cost role

__host__ __device__ inline size_t quad_ws_smem_bytes(int T, int n_obs, int ns, size_t grid_bytes, bool gen = false,
                                                     bool to_go = false) {
  const size_t TM = 4 * static_cast<size_t>(T);
  return sizeof(float) * (4 * static_cast<size_t>(n_obs) + 2 * TM + T + 2 * static_cast<size_t>(ns) + TM * ns +
                          static_cast<size_t>(quad_ws_ring(to_go, gen)) * quad_ws_chunk(to_go) * kQwsPass * ns +
                          (gen ? 2 * TM * 4 : 0) + (to_go ? (static_cast<size_t>(T) + 1) * ns : 0)) +
         grid_bytes;
}

template <int NS, bool GEN = false, bool TOGO = false>
__device__ __forceinline__ void rollout_block_quad_ws(const CtrlParams &p, const float *__restrict__ x0, uint32_t ctr,
                                                      const float *__restrict__ U, int k0,
                                                      float *__restrict__ S_out, float *__restrict__ part_sums,
                                                      BlockPartial *__restrict__ part, float *smem,
                                                      float *__restrict__ part_rho = nullptr,
                                                      DF *__restrict__ part_eta = nullptr) {
  static_assert(NS % 32 == 0, "roles must be warp-uniform");
  constexpr int M = Quad::M, N = Quad::N, C = quad_ws_chunk(TOGO), R = quad_ws_ring(TOGO, GEN), P = kQwsPass,
                NT = 3 * NS;
  static_assert(C % 2 == 0, "chunk 0 splits into two halves");
  __shared__ uint64_t bar_noise[kQwsMaxChunks * kQwsChunk / C], bar_full[R], bar_empty[R];
  __shared__ float sx0[N];
  const int T = p.T, TM = T * M, tid = threadIdx.x;
  const int nch = (T + C - 1) / C;
  float *sObs = smem;                                    // [n_obs][4] cylinders (16-byte aligned, first)
  float *sU = sObs + 4 * p.n_obs;                        // [TM]  nominal controls
  float *sRu = sU + TM;                                  // [TM]  R u_i
  float *sHu = sRu + TM;                                 // [T]   1/2 u_i^T R u_i
  float *sW = sHu + T;                                   // [NS]  weights
  float *sS = sW + NS;                                   // [NS]  path costs (cost role -> block partial)
  float *sDu = sS + NS;                                  // [TM][NS] perturbations
  float *sRing = sDu + static_cast<size_t>(TM) * NS;     // [R][C][P][NS]
  float *sGen = sRing + R * C * P * NS;                  // GEN: [T][2][M][M] (chol(Sigma_E,i), R_IS,i)
  float *sC = sGen + (GEN ? 2 * TM * M : 0);             // TOGO: [T][NS] step terms of S~
  float *sPhi = sC + (TOGO ? static_cast<size_t>(T) * NS : 0);  // TOGO: [NS] terminal costs
  unsigned short *sOff = reinterpret_cast<unsigned short *>(sPhi + (TOGO ? NS : 0));  // [cells + 1]
  const int ncell = p.grid_nx * p.grid_ny;
  unsigned char *sIdx = reinterpret_cast<unsigned char *>(sOff + (ncell + 1));       // [grid_nidx]

  for (int o = tid; o < TM; o += NT) sU[o] = U[o];
  if (GEN)
    for (int o = tid; o < 2 * TM * M; o += NT) sGen[o] = p.gen[o];
  for (int o = tid; o < 4 * p.n_obs; o += NT) sObs[o] = (o & 3) == 3 ? 0.0f : p.obs[3 * (o >> 2) + (o & 3)];
  if (p.grid_nx > 0) {
    for (int o = tid; o <= ncell; o += NT) sOff[o] = p.grid_off[o];
    for (int o = tid; o < p.grid_nidx; o += NT) sIdx[o] = p.grid_idx[o];
  }
  if (tid < N) sx0[tid] = x0[tid];
  if (tid == 0) {
    // chunk 0's noise is drawn by the dynamics and cost roles together (2 NS arrivals)
    for (int c = 0; c < nch; ++c) tc::mbar_init(&bar_noise[c], c == 0 ? 2 * NS : NS);
    for (int r = 0; r < R; ++r) {
      tc::mbar_init(&bar_full[r], NS);
      tc::mbar_init(&bar_empty[r], NS);
    }
  }
  __syncthreads();
  for (int i = tid; i < T; i += NT) {
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

  float Lnu[M * M];
#pragma unroll
  for (int a = 0; a < M * M; ++a) Lnu[a] = p.Lnu[a];
  bool ok = true;
  // Philox block i -> du_i (four controls) of sample k0 + slot
  auto block = [&](int i, int slot) {
    float e[4];
    normals4(static_cast<uint32_t>(i), static_cast<uint32_t>(k0 + slot), ctr, p.gid, p.key_lo, p.key_hi, e);
    float du[M];
    scale_noise<M>(GEN ? sGen + static_cast<size_t>(i) * 2 * M * M : Lnu, e, du);
#pragma unroll
    for (int a = 0; a < M; ++a) sDu[(i * M + a) * NS + slot] = du[a];
  };
  // Chunk 0's noise: the dynamics and the cost role would otherwise wait for the noise role's
  // first chunk, so they draw its steps themselves, half each, while the noise role starts on
  // chunk 1.
  if (tid >= NS) {
    const int slot = tid % NS, i0 = tid < 2 * NS ? 0 : C / 2;
#pragma unroll 1
    for (int i = i0; i < min(i0 + C / 2, T); ++i) block(i, slot);
    tc::mbar_arrive(&bar_noise[0]);
  }
  if (tid < NS) {
    // ---- noise: du of chunks 1.. into sDu (Philox block i covers step i's four controls) --
    const int slot = tid;
    for (int c = 1; c < nch; ++c) {
      const int i0 = c * C;
      if (i0 + C <= T) {
#pragma unroll
        for (int j = 0; j < C; ++j) block(i0 + j, slot);
      } else {
#pragma unroll 1
        for (int i = i0; i < T; ++i) block(i, slot);
      }
      tc::mbar_arrive(&bar_noise[c]);
    }
  } else if (tid < 2 * NS) {
    // ---- dynamics: the RK4 chain, run ahead whether or not the sample has crashed --------
    const int slot = tid - NS;
    float x[N];
#pragma unroll
    for (int a = 0; a < N; ++a) x[a] = sx0[a];
    for (int c = 0; c < nch; ++c) {
      ok = tc::mbar_wait(&bar_noise[c], 0u);
      if (ok && c >= R) ok = tc::mbar_wait(&bar_empty[c % R], static_cast<uint32_t>((c / R - 1) & 1));
      if (!ok) break;
      float *ring = sRing + (c % R) * (C * P * NS);
      const int i0 = c * C, steps = min(C, T - i0);
#pragma unroll 1
      for (int j = 0; j < steps; ++j) {
        const int i = i0 + j;
        float v[M];
#pragma unroll
        for (int a = 0; a < M; ++a) v[a] = sU[i * M + a] + sDu[(i * M + a) * NS + slot];
        float y[N];
        const bool finite = Quad::rk4(x, v, p.dt, y);
        float *out = ring + j * (P * NS) + slot;
        out[0] = finite ? y[0] : __int_as_float(0x7fc00000);
        out[NS] = y[1];
        out[2 * NS] = y[2];
        out[3 * NS] = y[3];
        out[4 * NS] = y[4];
        out[5 * NS] = y[5];
        out[6 * NS] = y[7];
        out[7 * NS] = y[8];
#pragma unroll
        for (int a = 0; a < N; ++a) x[a] = y[a];
      }
      tc::mbar_arrive(&bar_full[c % R]);
    }
  } else {
    // ---- cost: crash decisions, q(x), IS terms, S~ ------------------------------------------
    const int slot = tid - 2 * NS;
    const Env env = make_env(p, sObs, 1, p.grid_nx > 0 ? sOff : nullptr, sIdx);
    float Rm[M * M];
#pragma unroll
    for (int a = 0; a < M * M; ++a) Rm[a] = p.R[a];
    float x[N];
#pragma unroll
    for (int a = 0; a < N; ++a) x[a] = sx0[a];
    Quad::Aux aux;
    aux.crashed = false;
    aux.d = Quad::nearest(env, x[0], x[1]);
    KahanSum S;
    for (int c = 0; c < nch; ++c) {
      // the noise wait is already satisfied (the dynamics waited on it before publishing
      // this chunk); taking it here makes the du writes visible to this thread directly
      ok = tc::mbar_wait(&bar_full[c % R], static_cast<uint32_t>((c / R) & 1)) && tc::mbar_wait(&bar_noise[c], 0u);
      if (!ok) break;
      const float *ring = sRing + (c % R) * (C * P * NS);
      const int i0 = c * C, steps = min(C, T - i0);
#pragma unroll 1
      for (int j = 0; j < steps; ++j) {
        const int i = i0 + j;
        const float *in = ring + j * (P * NS) + slot;
        const float px = in[0], py = in[NS], pz = in[2 * NS], vx = in[3 * NS], vy = in[4 * NS], vz = in[5 * NS];
        const float pitch = in[6 * NS], yaw = in[7 * NS];
        float du[M];
#pragma unroll
        for (int a = 0; a < M; ++a) du[a] = sDu[(i * M + a) * NS + slot];
        const float *Rg = sGen + static_cast<size_t>(i) * 2 * M * M + M * M;  // GEN: R_IS,i
        float duRdu = 0.0f, uRdu = 0.0f;
#pragma unroll
        for (int a = 0; a < M; ++a) {
          uRdu = fmaf(sRu[i * M + a], du[a], uRdu);
          float rd = 0.0f;
#pragma unroll
          for (int l = 0; l < M; ++l) rd = fmaf(GEN ? Rg[a * M + l] : Rm[a * M + l], du[l], rd);
          duRdu = fmaf(du[a], rd, duRdu);
        }
        // the sequential step's crash test on the new state (a crashed sample keeps its state
        // whatever the test says, and the states handed over after its crash can be far
        // outside the forest, so it skips the search)
        float d = aux.crashed ? 0.0f : Quad::nearest(env, px, py);
        const bool finite = isfinite(px);
        if (!finite) d = -1.0f;
        const bool hit = !finite || d < 0.0f || pz < 0.0f || (Quad::pitch_limit - fabsf(pitch)) <= 0.0f;
        if (!aux.crashed && !hit) {
          x[0] = px;
          x[1] = py;
          x[2] = pz;
          x[3] = vx;
          x[4] = vy;
          x[5] = vz;
          x[7] = pitch;
          x[8] = yaw;
          aux.d = d;
        }
        aux.crashed = aux.crashed || hit;
        const float cv = Quad::cost(x, aux, env) + ((GEN ? 0.5f : p.is_du) * duRdu + uRdu + sHu[i]);
        S.add(cv);
        if (TOGO) sC[i * NS + slot] = cv;
      }
      tc::mbar_arrive(&bar_empty[c % R]);
    }
    float phi = INFINITY;
    if (ok) {
      phi = Quad::cost(x, aux, env);
      S.add(phi);  // phi(x_T) = q(x_T)
    }
    sS[slot] = ok ? S.s : INFINITY;
    if (TOGO) sPhi[slot] = phi;
  }
  __syncthreads();
  // the update kernel may start launching now (it waits for this grid's results itself)
  asm volatile("griddepcontrol.launch_dependents;");
  const bool owner = tid < NS;
  if (TOGO) {
    if (owner && k0 + tid < p.K) S_out[k0 + tid] = isfinite(sS[tid]) ? sS[tid] : INFINITY;
    block_partial_to_go<M, NT, NS>(p, k0, owner ? sPhi[tid] : 0.0f, sC, sDu, part_sums, part_rho, part_eta, part);
    return;
  }
  block_partial<M, NT, false, NS>(p, owner ? k0 + tid : INT_MAX, ctr, owner ? sS[tid] : INFINITY, Lnu, S_out,
                                  part_sums, part, sW, sDu);
}

}  // namespace mppi
