// Car rollout with each sample's work split over three threads in different warps
// (warp specialisation).
//
// With one thread per sample, K = 16384 samples make 512 warps: at most one per SM
// sub-partition, so every dependency latency of the step is exposed.  The car step
// separates into
//   the velocity recurrence (vx, vy, r, delta): slip angles, tyre forces and the steering
//       actuator; it reads only itself and the control v_i = u_i + du_i;
//   the pose sums (X, Y, psi), the cost map and the importance-sampling terms, which read
//       the velocities and du but never feed back into them;
//   the noise du_i, which depends on nothing of the state.
// A CTA owns NS samples with 3 NS threads in three warp-uniform roles:
//   core  (threads 0..NS-1)      the recurrence;
//   noise (threads NS..2NS-1)    Philox normals -> du = sqrt(nu) L eps, ahead of the core;
//   pose  (threads 2NS..3NS-1)   pose, q(x), IS terms and S~ (Kahan), in the same order
//                                and arithmetic as the one-thread kernel.
// Shared memory carries the hand-offs, in chunks of C steps:
//   du  [T*M][NS]      noise -> core and pose, one single-use mbarrier per chunk (also the
//                      operand of the block sums)
//   vel [R][C][3][NS]  core -> pose, (vx, vy, r) after each step, a ring of R chunks (car_ws_ring) with
//                      full/empty mbarriers
// With TOGO (the per-time-step cost-to-go weighting) the pose role also keeps each step's
// term of S~ in sC [T][NS] and its terminal cost, and the block forms per-step partials.
// With GEN (a general sampling covariance per step, Theorem 1) the noise role scales step
// i's normals by chol(Sigma_E,i) and the pose role's IS term is 1/2 du^T (R - lambda
// Sigma_E,i^-1) du + u^T R du + 1/2 u^T R u, the per-step matrices staged in sGen.
// Every wait is bounded; a thread whose wait runs out stops and its sample's cost is +inf.
#pragma once
#include <type_traits>

#include "rollout_body.cuh"
#include "tc_common.cuh"

namespace mppi {

constexpr int kWsSamples = 128;   // samples per CTA (3x threads)
constexpr int kWsRoles = 3;
constexpr int kWsChunk = 8;       // steps per hand-off
// Chunks in the velocity ring.  Two keep the shared memory of the path weighting (127 KB at
// T = 100) and of the cost-to-go weighting inside smaller shared-memory configurations of the
// SM, which leaves more L1 to the cost-map lookups.  With the general sampling covariance two
// and four measured the same; four are kept there.
__host__ __device__ constexpr int car_ws_ring(bool to_go, bool gen) { return gen && !to_go ? 4 : 2; }
constexpr int kWsMaxChunks = 32;  // noise barriers: T <= kWsChunk * kWsMaxChunks

__host__ __device__ inline size_t car_ws_smem_bytes(int T, int ns, bool to_go = false, bool gen = false) {
  const size_t TM = 2 * static_cast<size_t>(T);
  return sizeof(float) * (2 * TM + T + 2 * static_cast<size_t>(ns) + TM * ns +
                          static_cast<size_t>(car_ws_ring(to_go, gen)) * kWsChunk * 3 * ns +
                          (to_go ? (static_cast<size_t>(T) + 1) * ns : 0) + (gen ? 2 * TM * 2 : 0));
}

// The car's velocity state (vx, vy, r, delta), passed by value.
struct CarVel {
  float x[4];
};

// Steps i0 .. i0+n-1 of the velocity recurrence in the arctangent form (Car::vel_step) from x,
// controls u_i + du_i re-read from shared memory, velocities stored to the ring slot: the
// rare redo of a chunk whose slip ratios left their domain.  Not inlined, so that the hot
// loop's code holds only the call.
static __device__ __noinline__ CarVel car_vel_chunk_atan(CarVel x, const float *sU, const float *sDu, float *vel, int i0,
                                                        int n, int NS, int slot, float dt) {
  constexpr int M = Car::M;
  for (int j = 0; j < n; ++j) {
    const int i = i0 + j;
    const float v[M] = {sU[i * M] + sDu[(i * M) * NS + slot], sU[i * M + 1] + sDu[(i * M + 1) * NS + slot]};
    Car::vel_step(x.x, v, dt);
    vel[(3 * j) * NS + slot] = x.x[0];
    vel[(3 * j + 1) * NS + slot] = x.x[1];
    vel[(3 * j + 2) * NS + slot] = x.x[2];
  }
  return x;
}

template <int NS, bool TOGO = false, bool GEN = false>
__device__ __forceinline__ void rollout_block_car_ws(const CtrlParams &p, const float *__restrict__ x0, uint32_t ctr,
                                                     const float *__restrict__ U, int k0, float *__restrict__ S_out,
                                                     float *__restrict__ part_sums, BlockPartial *__restrict__ part,
                                                     float *smem, float *__restrict__ part_rho = nullptr,
                                                     DF *__restrict__ part_eta = nullptr) {
  static_assert(NS % 32 == 0, "roles must be warp-uniform");
  static_assert(kWsChunk % 4 == 0, "chunk 0 splits into two halves of whole Philox blocks");
  constexpr int M = 2, C = kWsChunk, R = car_ws_ring(TOGO, GEN), NT = kWsRoles * NS;
  __shared__ uint64_t bar_noise[kWsMaxChunks], bar_full[R], bar_empty[R];
  const int T = p.T, TM = T * M, tid = threadIdx.x;
  const int nch = (T + C - 1) / C;
  float *sU = smem;         // [TM]  nominal controls
  float *sRu = sU + TM;     // [TM]  R u_i
  float *sHu = sRu + TM;    // [T]   1/2 u_i^T R u_i
  float *sW = sHu + T;      // [NS]  weights
  float *sS = sW + NS;      // [NS]  path costs (pose -> owner of the block partial)
  float *sDu = sS + NS;     // [TM][NS] perturbations
  float *sVel = sDu + static_cast<size_t>(TM) * NS;  // [R][C][3][NS]
  float *sC = sVel + R * C * 3 * NS;                 // TOGO: [T][NS] step terms of S~
  float *sPhi = sC + static_cast<size_t>(T) * NS;    // TOGO: [NS] terminal costs
  float *sGen = TOGO ? sPhi + NS : sC;              // GEN: [T][2][M][M] (chol(Sigma_E,i), R_IS,i)

  __shared__ float sx0[Car::N];  // x0 staged once (it may live in mapped host memory)
  for (int o = tid; o < TM; o += NT) sU[o] = U[o];
  if (GEN)
    for (int o = tid; o < 2 * TM * M; o += NT) sGen[o] = p.gen[o];
  if (tid < Car::N) sx0[tid] = x0[tid];
  if (tid == 0) {
    // chunk 0's noise is drawn by the core and pose roles together (2 NS arrivals)
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

  const int role = tid / NS;
  const int slot = tid - role * NS;
  const int k = k0 + slot;
  bool ok = true;

  // Philox block b -> du of steps 2b and 2b+1 (those < T) of this thread's sample
  auto noise_block = [&](int b, const float *Lnu) {
    float e[4];
    normals4(static_cast<uint32_t>(b), static_cast<uint32_t>(k), ctr, p.gid, p.key_lo, p.key_hi, e);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int i = 2 * b + s;
      float du[M];
      scale_noise<M>(GEN ? sGen + static_cast<size_t>(min(i, T - 1)) * 2 * M * M : Lnu, e + s * M, du);
      if (i < T) {
#pragma unroll
        for (int a = 0; a < M; ++a) sDu[(i * M + a) * NS + slot] = du[a];
      }
    }
  };
  // Chunk 0's noise: the core and the pose role would otherwise wait for the noise role's
  // first chunk, so they draw its blocks themselves, half each, while the noise role starts
  // on chunk 1.
  if (role != 1) {
    float Lnu[M * M];
#pragma unroll
    for (int a = 0; a < M * M; ++a) Lnu[a] = p.Lnu[a];
    const int bq = role == 0 ? 0 : C / 4;
#pragma unroll 1
    for (int b = bq; b < bq + C / 4 && 2 * b < T; ++b) noise_block(b, Lnu);
    tc::mbar_arrive(&bar_noise[0]);
  }

  // Each role runs whole chunks through one fully unrolled body (one basic block, so the
  // compiler can interleave the steps) and the ragged last chunk through a small rolled
  // loop: three roles share each sub-partition's instruction cache.
  if (role == 0) {
    // ---- core: the velocity recurrence ----------------------------------------------
    float xv[4] = {sx0[3], sx0[4], sx0[5], sx0[6]};
    for (int c = 0; c < nch; ++c) {
      ok = tc::mbar_wait(&bar_noise[c], 0u);
      if (ok && c >= R) ok = tc::mbar_wait(&bar_empty[c % R], static_cast<uint32_t>((c / R - 1) & 1));
      if (!ok) break;
      float *vel = sVel + (c % R) * (C * 3 * NS);
      const int i0 = c * C;
      // CN steps of the chunk through one unrolled body (the half chunk not with the cost-to-go
      // weighting, whose rollout that made 1.7 us slower)
      auto core_chunk = [&](auto cn) {
        constexpr int CN = decltype(cn)::value;
        // the controls of all CN steps first: the compiler cannot move a shared load above
        // the velocity stores of earlier steps
        float vv[CN][M];
#pragma unroll
        for (int j = 0; j < CN; ++j) {
          const int i = i0 + j;
          vv[j][0] = sU[i * M] + sDu[(i * M) * NS + slot];
          vv[j][1] = sU[i * M + 1] + sDu[(i * M + 1) * NS + slot];
        }
        // the chunk through the slip ratios; a lane that leaves their domain (rare: an extreme
        // slide or steering angle) redoes the chunk from its start with the arctangent form,
        // under a warp vote so that the common case carries no second path
        const float xs[4] = {xv[0], xv[1], xv[2], xv[3]};
        bool in = true;
#pragma unroll
        for (int j = 0; j < CN; ++j) {
          in &= Car::vel_step_ratio(xv, vv[j], p.dt);
          vel[(3 * j) * NS + slot] = xv[0];
          vel[(3 * j + 1) * NS + slot] = xv[1];
          vel[(3 * j + 2) * NS + slot] = xv[2];
        }
        if (__any_sync(__activemask(), !in) && !in) {
          const CarVel r = car_vel_chunk_atan(CarVel{{xs[0], xs[1], xs[2], xs[3]}}, sU, sDu, vel, i0, CN, NS, slot, p.dt);
#pragma unroll
          for (int q = 0; q < 4; ++q) xv[q] = r.x[q];
        }
      };
      if (i0 + C <= T) {
        core_chunk(std::integral_constant<int, C>{});
      } else if (!TOGO && T - i0 == C / 2) {  // a half chunk at the end (T = 100): unrolled as well
        core_chunk(std::integral_constant<int, C / 2>{});
      } else {
#pragma unroll 1
        for (int j = 0; j < T - i0; ++j) {
          const int i = i0 + j;
          const float v[M] = {sU[i * M] + sDu[(i * M) * NS + slot], sU[i * M + 1] + sDu[(i * M + 1) * NS + slot]};
          Car::vel_step(xv, v, p.dt);
          vel[(3 * j) * NS + slot] = xv[0];
          vel[(3 * j + 1) * NS + slot] = xv[1];
          vel[(3 * j + 2) * NS + slot] = xv[2];
        }
      }
      tc::mbar_arrive(&bar_full[c % R]);
    }
  } else if (role == 1) {
    // ---- noise: du of chunks 1.. into sDu (block b of the generator covers steps 2b, 2b+1)
    float Lnu[M * M];
#pragma unroll
    for (int a = 0; a < M * M; ++a) Lnu[a] = p.Lnu[a];
    for (int c = 1; c < nch; ++c) {
      const int b0 = c * (C / 2);
      if ((c + 1) * C <= T) {
#pragma unroll
        for (int q = 0; q < C / 2; ++q) noise_block(b0 + q, Lnu);
      } else {
#pragma unroll 1
        for (int b = b0; 2 * b < T; ++b) noise_block(b, Lnu);
      }
      tc::mbar_arrive(&bar_noise[c]);
    }
  } else {
    // ---- pose: heading and position sums, q(x), IS terms, S~ ------------------------
    const Env env = make_env(p, nullptr);
    float Rm[M * M];
#pragma unroll
    for (int a = 0; a < M * M; ++a) Rm[a] = p.R[a];
    float X = sx0[0], Y = sx0[1], psi = sx0[2], vx = sx0[3], vy = sx0[4], r = sx0[5];
    Car::Aux aux;
    aux.cX = aux.cY = aux.cpsi = 0.0f;
    KahanSum S;
    auto is_term = [&](int i) {  // importance-sampling running term of step i
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
      return (GEN ? 0.5f : p.is_du) * duRdu + uRdu + sHu[i];
    };
    // S~ gains q(x_{i+1}) + is_i one step late (the cost-map loads of a step are issued
    // before they are needed).  The pending term starts as an exact zero, whose Kahan
    // addition leaves the sum unchanged, so no step needs a first-step test.
    Car::Pending pend{0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    float pend_is = 0.0f;
    for (int c = 0; c < nch; ++c) {
      // the noise wait is already satisfied (the core waited on it before publishing this
      // chunk); taking it here makes the du writes visible to this thread directly
      ok = tc::mbar_wait(&bar_full[c % R], static_cast<uint32_t>((c / R) & 1)) && tc::mbar_wait(&bar_noise[c], 0u);
      if (!ok) break;
      const float *vel = sVel + (c % R) * (C * 3 * NS);
      const int i0 = c * C;
      // CN steps of the chunk through one unrolled body
      auto pose_chunk = [&](auto cn) {
        constexpr int CN = decltype(cn)::value;
        float nv[CN][3], is[CN];
#pragma unroll
        for (int j = 0; j < CN; ++j) {
          nv[j][0] = vel[(3 * j) * NS + slot];
          nv[j][1] = vel[(3 * j + 1) * NS + slot];
          nv[j][2] = vel[(3 * j + 2) * NS + slot];
        }
        tc::mbar_arrive(&bar_empty[c % R]);
#pragma unroll
        for (int j = 0; j < CN; ++j) is[j] = is_term(i0 + j);
        // all CN poses and their map loads first, then the CN cost additions in step order
        Car::Pending pq[CN];
#pragma unroll
        for (int j = 0; j < CN; ++j) {
          Car::pose_step(X, Y, psi, aux, vx, vy, r, p.dt);
          vx = nv[j][0];
          vy = nv[j][1];
          r = nv[j][2];
          const float xq[Car::N] = {X, Y, psi, vx, vy, r, 0.0f};
          pq[j] = Car::cost_issue(xq, aux, env);
        }
#pragma unroll
        for (int j = 0; j < CN; ++j) {
          const float cv = Car::cost_finish(pend, env) + pend_is;  // the term of step i0 + j - 1
          S.add(cv);
          if (TOGO && i0 + j > 0) sC[(i0 + j - 1) * NS + slot] = cv;
          pend = pq[j];
          pend_is = is[j];
        }
      };
      if (i0 + C <= T) {
        pose_chunk(std::integral_constant<int, C>{});
      } else if (!TOGO && T - i0 == C / 2) {  // a half chunk at the end (T = 100): unrolled as well
        pose_chunk(std::integral_constant<int, C / 2>{});
      } else {
#pragma unroll 1
        for (int j = 0; j < T - i0; ++j) {
          Car::pose_step(X, Y, psi, aux, vx, vy, r, p.dt);
          vx = vel[(3 * j) * NS + slot];
          vy = vel[(3 * j + 1) * NS + slot];
          r = vel[(3 * j + 2) * NS + slot];
          const float cv = Car::cost_finish(pend, env) + pend_is;
          S.add(cv);
          if (TOGO && i0 + j > 0) sC[(i0 + j - 1) * NS + slot] = cv;
          const float xq[Car::N] = {X, Y, psi, vx, vy, r, 0.0f};
          pend = Car::cost_issue(xq, aux, env);
          pend_is = is_term(i0 + j);
        }
        tc::mbar_arrive(&bar_empty[c % R]);
      }
    }
    float phi = INFINITY;
    if (ok) {
      const float cv = Car::cost_finish(pend, env) + pend_is;
      S.add(cv);
      if (TOGO) sC[(T - 1) * NS + slot] = cv;
      const float xq[Car::N] = {X, Y, psi, vx, vy, r, 0.0f};
      phi = Car::cost(xq, aux, env);
      S.add(phi);  // phi(x_T) = q(x_T)
    }
    sS[slot] = ok ? S.s : INFINITY;
    if (TOGO) sPhi[slot] = phi;
  }
  __syncthreads();
  // the update kernel may start launching now (it waits for this grid's results itself)
  asm volatile("griddepcontrol.launch_dependents;");
  const bool owner = role == 0;
  if (TOGO) {
    if (owner && k < p.K) S_out[k] = isfinite(sS[tid]) ? sS[tid] : INFINITY;
    block_partial_to_go<M, NT, NS>(p, k0, owner ? sPhi[tid] : 0.0f, sC, sDu, part_sums, part_rho, part_eta, part);
    return;
  }
  float Lnu_unused[M * M] = {0.0f, 0.0f, 0.0f, 0.0f};
  block_partial<M, NT, false, NS>(p, owner ? k : INT_MAX, ctr, owner ? sS[tid] : INFINITY, Lnu_unused, S_out,
                                  part_sums, part, sW, sDu);
}

}  // namespace mppi
