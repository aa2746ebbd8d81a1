// Per-block body of the fused MPPI rollout, shared by the single-controller kernel
// and the batched (serving) kernel.
//
// One thread per sample k.  For i = 0..T-1: Philox normals -> du_i = Lnu eps ->
// x_{i+1} = F(x_i, u_i + du_i) -> S~ += q(x_{i+1}) + IS running cost (Kahan FP32);
// then S~ += phi(x_T).  The block then forms its softmax partial:
//   rho_b = min_k S~_k (lowest k on ties), w_k = exp(-(S~_k - rho_b)/lambda),
//   eta_b = sum_k w_k (double-FP32), part_b[i][j] = sum_k w_k du_{i,j,k} (FP32 block sum).
// Two ways to get du back for the block sums:
//   STORE: du kept in shared memory during the rollout ([T*M][BLK] floats);
//   REGEN: du regenerated from the counter-based generator after the rollout (no
//          shared memory, so many blocks fit on an SM), reduced with a transposed
//          butterfly across the warp (31 shuffles per 32 outputs).
#pragma once
#include <climits>

#include "merge_common.cuh"
#include "systems.cuh"

namespace mppi {

// du_j = sum_{l <= j} Lnu[j][l] eps_l  (Lnu = sqrt(nu) chol(Sigma), lower triangular)
template <int M>
__device__ __forceinline__ void scale_noise(const float *Lnu, const float *eps, float *du) {
#pragma unroll
  for (int j = 0; j < M; ++j) {
    float a = 0.0f;
#pragma unroll
    for (int l = 0; l <= j; ++l) a = fmaf(Lnu[j * M + l], eps[l], a);
    du[j] = a;
  }
}

// grid_off / grid_idx: the nearest-cylinder grid staged in shared memory (or null: none)
__device__ __forceinline__ Env make_env(const CtrlParams &p, const float *obs, int packed = 0,
                                        const unsigned short *grid_off = nullptr,
                                        const unsigned char *grid_idx = nullptr) {
  Env e;
  e.obs_packed = packed;
  e.map = p.map;
  e.map_w = p.map_w;
  e.map_h = p.map_h;
  e.map_ox = p.map_ox;
  e.map_oy = p.map_oy;
  e.map_inv_cell = p.map_inv_cell;
  e.obs = obs;
  e.n_obs = p.n_obs;
  e.gx = p.goal[0];
  e.gy = p.goal[1];
  e.gz = p.goal[2];
  e.grid_off = grid_off;
  e.grid_idx = grid_idx;
  e.grid_nx = grid_off ? p.grid_nx : 0;
  e.grid_ny = p.grid_ny;
  e.grid_ox = p.grid_ox;
  e.grid_oy = p.grid_oy;
  e.grid_inv_h = p.grid_inv_h;
  return e;
}

// Sum over the 32 lanes of each of 32 per-lane values: afterwards lane l holds the
// warp total of value l (recursive halving; 31 shuffles in all).
__device__ __forceinline__ float transpose_reduce32(float v[32]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    const bool upper = (lane & s) != 0;
#pragma unroll
    for (int i = 0; i < s; ++i) {
      const float send = upper ? v[i] : v[i + s];
      const float keep = upper ? v[i + s] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, s);
    }
  }
  return v[0];
}

// Bytes of the quadrotor's nearest-cylinder grid in shared memory (offsets, then indices,
// 16-byte padded; 0 without a grid).
__host__ __device__ inline size_t quad_grid_bytes(int nx, int ny, int nidx) {
  if (nx <= 0) return 0;
  return (sizeof(unsigned short) * (static_cast<size_t>(nx) * ny + 1) + static_cast<size_t>(nidx) + 15) &
         ~static_cast<size_t>(15);
}
__host__ __device__ inline size_t quad_grid_bytes(const CtrlParams &p) {
  return quad_grid_bytes(p.grid_nx, p.grid_ny, p.grid_nidx);
}

// Shared-memory bytes of rollout_block (dynamic part) for T*M outputs; to_go adds the
// per-step costs [T][blk] of the cost-to-go weighting, grid_bytes the nearest-cylinder grid.
__host__ __device__ inline size_t rollout_smem_bytes(int T, int M, int n_obs, int blk, bool regen, bool to_go = false,
                                                   bool gen = false, size_t grid_bytes = 0) {
  const size_t TM = static_cast<size_t>(T) * M;
  return 16 + sizeof(float) * (2 * TM + T + 4 * static_cast<size_t>(n_obs) + blk + (regen ? 0 : TM * blk) +
                               (to_go ? static_cast<size_t>(T) * blk : 0) + (gen ? 2 * TM * M : 0)) +
         (grid_bytes ? grid_bytes + 16 : 0);
}

// Per-time-step block partials of the cost-to-go weighting (Eq. App_PI read literally: u_i
// weighted by each rollout's cost from t_i onward).  sC [T][BLK] holds each thread's step
// costs c_i (the terms its path sum added); the block turns them into costs-to-go
// S_i = c_i + ... + c_{T-1} + phi (compensated, backward, in place), then per step i, one warp
// per step:
//   rho_{b,i} = min_k S_i,  eta_{b,i} = sum_k exp(-(S_i - rho_{b,i})/lambda) (double-FP32 sums),
//   part_sums[i*M+j] = sum_k w_{i,k} du_{i,j,k} (FP32),
// and `part` gets step 0's (rho, k*, eta) (the total path cost's, for the debug surface).
// Samples k >= K and non-finite costs count as +inf.
//
// BLK threads run it; the block's NS samples (k0 + column) are sC's and sDu's columns, and
// threads 0..NS-1 own them (phi: the owner's terminal cost).
template <int M, int BLK, int NS = BLK>
__device__ __forceinline__ void block_partial_to_go(const CtrlParams &p, int k0, float phi, float *sC,
                                                    const float *sDu, float *__restrict__ part_sums,
                                                    float *__restrict__ part_rho, DF *__restrict__ part_eta,
                                                    BlockPartial *__restrict__ part) {
  static_assert(NS % 32 == 0 && NS <= BLK, "samples per block");
  constexpr int NW = BLK / 32, CPL = NS / 32;
  const int T = p.T, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid < NS) {
    const bool valid = k0 + tid < p.K;
    KahanSum s;
    s.s = phi;
    for (int i = T - 1; i >= 0; --i) {
      s.add(sC[i * NS + tid]);
      sC[i * NS + tid] = valid && isfinite(s.s) ? s.s : INFINITY;
    }
  }
  __syncthreads();
  for (int i = warp; i < T; i += NW) {
    float sv[CPL];
    float mv = INFINITY;
    int mi = INT_MAX;
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
      sv[c] = sC[i * NS + lane + 32 * c];
      const int kk = k0 + lane + 32 * c;  // sample of that column
      if (sv[c] < mv || (sv[c] == mv && kk < mi)) {
        mv = sv[c];
        mi = isfinite(sv[c]) ? kk : INT_MAX;
      }
    }
    warp_argmin(mv, mi);
    const float rho = mv;
    // eta in double-FP32 (error-free sums: ~48 bits, as FP64 would give, without B300's slow
    // FP64 pipe, which a per-step normaliser would otherwise keep busy)
    DF ed{0.0f, 0.0f};
    float acc[M];
#pragma unroll
    for (int j = 0; j < M; ++j) acc[j] = 0.0f;
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
      const float w = (isfinite(rho) && isfinite(sv[c])) ? expf(-(sv[c] - rho) * p.inv_lambda) : 0.0f;
      df_add(ed, DF{w, 0.0f});
#pragma unroll
      for (int j = 0; j < M; ++j) acc[j] = fmaf(w, sDu[(i * M + j) * NS + lane + 32 * c], acc[j]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
      df_add(ed, DF{__shfl_xor_sync(0xffffffffu, ed.hi, o), __shfl_xor_sync(0xffffffffu, ed.lo, o)});
    const double e = static_cast<double>(ed.hi) + static_cast<double>(ed.lo);  // lane 0's is used
#pragma unroll
    for (int j = 0; j < M; ++j) acc[j] = warp_sum_f(acc[j]);
    if (lane == 0) {
#pragma unroll
      for (int j = 0; j < M; ++j) part_sums[i * M + j] = acc[j];
      part_rho[i] = rho;
      part_eta[i] = ed;
      if (i == 0) {
        BlockPartial bp;
        bp.eta = e;
        bp.rho = rho;
        bp.kstar = mi;
        *part = bp;
      }
    }
  }
}

// The block's softmax partial from each thread's path cost Sk_raw (sample k):
//   rho_b = min_k S~_k (lowest k on ties), w_k = exp(-(S~_k - rho_b)/lambda),
//   eta_b = sum_k w_k (double-FP32), part_sums[i*M+j] = sum_k w_k du_{i,j,k} (FP32)
// with du from shared memory (STORE: sDu [T*M][BLK]) or regenerated (REGEN).
// Non-finite costs and samples k >= K count as +inf (weight 0); k == INT_MAX marks a thread
// that owns no sample (it only takes part in the block reduction).  BLK is the thread count;
// in STORE mode threads 0..NS-1 own the NS samples of sDu's columns (NS = BLK unless some
// threads hold no sample).
// slot: the column of sDu (and of sW) this thread's sample owns in STORE mode, -1 for a
// thread that owns none; by default thread t < NS owns column t.
template <int M, int BLK, bool REGEN, int NS = BLK>
__device__ __forceinline__ void block_partial(const CtrlParams &p, int k, uint32_t ctr, float Sk_raw, const float *Lnu,
                                              float *__restrict__ S_out, float *__restrict__ part_sums,
                                              BlockPartial *__restrict__ part, float *sW, const float *sDu,
                                              int slot = -2) {
  constexpr int SPB = 4 / M, NW = BLK / 32;
  __shared__ float s_min[NW];
  __shared__ int s_idx[NW];
  __shared__ DF s_eta[NW];
  __shared__ float s_red[NW][32];
  const int TM = p.T * M, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool valid = k < p.K;
  float Sk = Sk_raw;
  if (!valid || !isfinite(Sk)) Sk = INFINITY;
  if (valid) S_out[k] = Sk;

  float mv = Sk;
  int mi = valid ? k : INT_MAX;
  warp_argmin(mv, mi);
  if (lane == 0) {
    s_min[warp] = mv;
    s_idx[warp] = mi;
  }
  __syncthreads();
  if (warp == 0) {
    float v = lane < NW ? s_min[lane] : INFINITY;
    int ii = lane < NW ? s_idx[lane] : INT_MAX;
    warp_argmin(v, ii);
    if (lane == 0) {
      s_min[0] = v;
      s_idx[0] = ii;
    }
  }
  __syncthreads();
  const float rho_b = s_min[0];
  const float w = (isfinite(rho_b) && isfinite(Sk)) ? expf(-(Sk - rho_b) * p.inv_lambda) : 0.0f;
  // eta_b in double-FP32 (error-free sums, ~48 bits) rather than on B300's slow FP64 pipe;
  // warps whose threads own no sample skip the shuffles
  DF e{w, 0.0f};
  if (__any_sync(0xffffffffu, k != INT_MAX)) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
      df_add(e, DF{__shfl_xor_sync(0xffffffffu, e.hi, o), __shfl_xor_sync(0xffffffffu, e.lo, o)});
  } else {
    e = DF{0.0f, 0.0f};
  }
  if (lane == 0) s_eta[warp] = e;

  if (!REGEN) {
    static_assert(NS % 32 == 0 && NS <= BLK, "samples per block");
    constexpr int CPL = NS / 32;  // samples per lane
    if (slot == -2) slot = tid < NS ? tid : -1;
    if (slot >= 0) sW[slot] = w;
    __syncthreads();
    // warp per 32 outputs: lane l sums its CPL samples of each output (conflict-free rows of
    // sDu), then the transposed butterfly leaves output g*32 + l's block sum in lane l (FP32)
    float wl[CPL];
#pragma unroll
    for (int c = 0; c < CPL; ++c) wl[c] = sW[lane + 32 * c];
    for (int g = warp; g * 32 < TM; g += NW) {
      float v[32];
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const int o = g * 32 + q;
        float acc = 0.0f;
        if (o < TM) {
#pragma unroll
          for (int c = 0; c < CPL; ++c) acc = fmaf(wl[c], sDu[o * NS + lane + 32 * c], acc);
        }
        v[q] = acc;
      }
      const float tot = transpose_reduce32(v);
      const int o = g * 32 + lane;
      if (o < TM) part_sums[o] = tot;
    }
  } else {
    const int nb = (TM + 3) >> 2;
    // The samples of the block with a weight not exactly 0 (exp underflows beyond ~103 lambda
    // above rho_b), listed in sample order.  With sharp weights they are few: then the block's
    // threads share their regeneration, each forming whole Philox blocks of outputs summed over
    // the listed samples in order (FP32, at most kLive deep); otherwise each warp with a live
    // sample regenerates its 32 samples' du and the warps' sums are added.
    constexpr int kLive = 32;
    __shared__ int s_live_k[kLive];
    __shared__ float s_live_w[kLive];
    __shared__ int s_nlive[NW];
    const bool live = w != 0.0f;  // implies a valid sample with a finite cost
    const unsigned live_bits = __ballot_sync(0xffffffffu, live);
    if (lane == 0) s_nlive[warp] = __popc(live_bits);
    __syncthreads();
    int before = 0, n_live = 0;
    for (int q = 0; q < NW; ++q) {
      before += q < warp ? s_nlive[q] : 0;
      n_live += s_nlive[q];
    }
    if (n_live <= kLive) {
      if (live) {
        const int pos = before + __popc(live_bits & ((1u << lane) - 1u));
        s_live_k[pos] = k;
        s_live_w[pos] = w;
      }
      __syncthreads();
      for (int b = tid; b < nb; b += BLK) {
        float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        for (int j = 0; j < n_live; ++j) {
          float eps[4];
          normals4(static_cast<uint32_t>(b), static_cast<uint32_t>(s_live_k[j]), ctr, p.gid, p.key_lo, p.key_hi, eps);
          const float wj = s_live_w[j];
#pragma unroll
          for (int s = 0; s < SPB; ++s) {
            float du[M];
            scale_noise<M>(Lnu, eps + s * M, du);
#pragma unroll
            for (int q = 0; q < M; ++q) acc[s * M + q] = fmaf(wj, du[q], acc[s * M + q]);
          }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (4 * b + q < TM) part_sums[4 * b + q] = acc[q];
      }
    } else {
      const bool warp_live = live_bits != 0u;
      // regenerate du, weight it, transpose-reduce 32 outputs (8 Philox blocks) at a time
      for (int g = 0; g < nb; g += 8) {
        float v[32];
#pragma unroll
        for (int q = 0; q < 32; ++q) v[q] = 0.0f;
        if (warp_live) {
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            float eps[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            if (g + q < nb && k != INT_MAX)  // k == INT_MAX: a thread that owns no sample
              normals4(static_cast<uint32_t>(g + q), static_cast<uint32_t>(k), ctr, p.gid, p.key_lo, p.key_hi, eps);
#pragma unroll
            for (int s = 0; s < SPB; ++s) {
              float du[M];
              scale_noise<M>(Lnu, eps + s * M, du);
#pragma unroll
              for (int j = 0; j < M; ++j) v[q * 4 + s * M + j] = w * du[j];
            }
          }
        }
        const float wsum = warp_live ? transpose_reduce32(v) : 0.0f;
        s_red[warp][lane] = wsum;
        __syncthreads();
        if (warp == 0) {
          float t = 0.0f;
#pragma unroll
          for (int q = 0; q < NW; ++q) t += s_red[q][lane];
          const int o = 4 * g + lane;
          if (o < TM) part_sums[o] = t;
        }
        __syncthreads();
      }
    }
  }
  __syncthreads();
  if (tid == 0) {
    DF eb = s_eta[0];
#pragma unroll
    for (int q = 1; q < NW; ++q) df_add(eb, s_eta[q]);
    BlockPartial bp;
    bp.eta = static_cast<double>(eb.hi) + static_cast<double>(eb.lo);
    bp.rho = rho_b;
    bp.kstar = s_idx[0];
    *part = bp;
  }
}

// One block of BLK samples of one controller.
//   p        controller constants; x0/ctr the state and iteration counter
//   U        [T][M] nominal controls (global)
//   k0       first sample index of this block
//   S_out    [K] path costs (global), part_sums [T*M] and part: this block's partial
//   smem     dynamic shared memory of rollout_smem_bytes(...)
//   du_ext   STORE only: if not null, the [TM][BLK] perturbation buffer lives there (a
//            global-memory slab owned by this CTA) instead of in shared memory
//   TOGO     cost-to-go weighting (STORE only): per-step partials into part_sums, part_rho
//            [T] and part_eta [T] of this block (block_partial_to_go)
//   GEN      general sampling covariance (STORE only): du_i = chol(Sigma_E,i) eps and the
//            running term 1/2 du^T (R - lambda Sigma_E,i^-1) du + u^T R du + 1/2 u^T R u, the
//            per-step matrices from p.gen
template <class Sys, int BLK, bool REGEN, bool TOGO = false, bool GEN = false>
__device__ __forceinline__ void rollout_block(const CtrlParams &p, const float *__restrict__ x0, uint32_t ctr,
                                              const float *__restrict__ U, int k0, float *__restrict__ S_out,
                                              float *__restrict__ part_sums, BlockPartial *__restrict__ part,
                                              float *smem, float *du_ext = nullptr, float *part_rho = nullptr,
                                              DF *part_eta = nullptr) {
  static_assert(!(TOGO && REGEN), "the cost-to-go weighting keeps du in shared memory");
  static_assert(!(GEN && REGEN), "the general sampling covariance keeps du in shared memory");
  constexpr int M = Sys::M, N = Sys::N, SPB = 4 / M;
  static_assert(4 % M == 0, "controls per Philox block must divide 4");
  const int T = p.T, TM = T * M, tid = threadIdx.x;
  float *sObs = smem;               // [n_obs][4] cylinders (16-byte aligned, first)
  float *sU = sObs + 4 * p.n_obs;   // [TM]  nominal controls
  float *sRu = sU + TM;             // [TM]  R u_i
  float *sHu = sRu + TM;            // [T]   1/2 u_i^T R u_i
  float *sW = sHu + T;              // [BLK] weights
  float *sDu = du_ext ? du_ext : sW + BLK;  // STORE only: [TM][BLK] perturbations of this block
  float *sC = sW + BLK + static_cast<size_t>(TM) * BLK;  // TOGO only: [T][BLK] step costs
  float *sGen = sC + (TOGO ? static_cast<size_t>(T) * BLK : 0);  // GEN only: [T][2][M][M]
  // the nearest-cylinder grid follows the arrays in use (du in shared memory or not)
  float *tail = (REGEN || du_ext) ? sW + BLK : sGen + (GEN ? 2 * TM * M : 0);
  unsigned short *sOff = reinterpret_cast<unsigned short *>((reinterpret_cast<uintptr_t>(tail) + 15) & ~uintptr_t(15));
  const int ncell = p.grid_nx * p.grid_ny;
  unsigned char *sIdx = reinterpret_cast<unsigned char *>(sOff + (ncell + 1));
  const bool grid = p.grid_nx > 0 && p.n_obs > 0;

  __shared__ float sx0[N];  // x0 staged once per block (it may live in mapped host memory)
  for (int o = tid; o < TM; o += BLK) sU[o] = U[o];
  for (int o = tid; o < 4 * p.n_obs; o += BLK) sObs[o] = (o & 3) == 3 ? 0.0f : p.obs[3 * (o >> 2) + (o & 3)];
  if (tid < N) sx0[tid] = x0[tid];
  if (GEN)
    for (int o = tid; o < 2 * TM * M; o += BLK) sGen[o] = p.gen[o];
  if (grid) {
    for (int o = tid; o <= ncell; o += BLK) sOff[o] = p.grid_off[o];
    for (int o = tid; o < p.grid_nidx; o += BLK) sIdx[o] = p.grid_idx[o];
  }
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

  const Env env = make_env(p, sObs, 1, grid ? sOff : nullptr, grid ? sIdx : nullptr);
  const int k = k0 + tid;
  float Lnu[M * M], R[M * M];
#pragma unroll
  for (int a = 0; a < M * M; ++a) {
    Lnu[a] = p.Lnu[a];
    R[a] = p.R[a];
  }
  float x[N];
#pragma unroll
  for (int a = 0; a < N; ++a) x[a] = sx0[a];
  typename Sys::Aux aux;
  Sys::init(x, aux, env);
  KahanSum S;

  // One time step: noise -> control -> dynamics; the cost of the new state is issued now
  // and finished after the next step's dynamics (same summation order as q_i + is_i).
  typename Sys::Pending pend;
  float pend_is = 0.0f;
  bool have = false;
  auto step_at = [&](int i, const float *e) {
    float du[M], v[M];
    const float *Lg = sGen + static_cast<size_t>(i) * 2 * M * M;  // GEN: chol(Sigma_E,i), then R_IS,i
    scale_noise<M>(GEN ? Lg : Lnu, e, du);
    float duRdu = 0.0f, uRdu = 0.0f;
#pragma unroll
    for (int j = 0; j < M; ++j) {
      v[j] = sU[i * M + j] + du[j];
      if (!REGEN) sDu[(i * M + j) * BLK + tid] = du[j];
      uRdu = fmaf(sRu[i * M + j], du[j], uRdu);
      float rd = 0.0f;
#pragma unroll
      for (int l = 0; l < M; ++l) rd = fmaf(GEN ? Lg[M * M + j * M + l] : R[j * M + l], du[l], rd);
      duRdu = fmaf(du[j], rd, duRdu);
    }
    Sys::step(x, v, aux, env, p.dt);
    if (have) {
      const float c = Sys::cost_finish(pend, env) + pend_is;
      S.add(c);
      if (TOGO) sC[(i - 1) * BLK + tid] = c;
    }
    pend = Sys::cost_issue(x, aux, env);
    pend_is = (GEN ? 0.5f : p.is_du) * duRdu + uRdu + sHu[i];
    have = true;
  };

  // Philox blocks: the normals of block b+1 are drawn while block b's steps run
  const int nb = (TM + 3) >> 2;
  const int nb_full = T / SPB;  // blocks whose SPB steps are all inside the horizon
  float eps[4];
  normals4(0u, static_cast<uint32_t>(k), ctr, p.gid, p.key_lo, p.key_hi, eps);
  for (int b = 0; b < nb_full; ++b) {
    float nxt[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    if (b + 1 < nb) normals4(static_cast<uint32_t>(b + 1), static_cast<uint32_t>(k), ctr, p.gid, p.key_lo, p.key_hi, nxt);
#pragma unroll
    for (int s = 0; s < SPB; ++s) step_at(b * SPB + s, eps + s * M);
#pragma unroll
    for (int j = 0; j < 4; ++j) eps[j] = nxt[j];
  }
  if (nb_full < nb) {  // the last block holds fewer than SPB steps
#pragma unroll
    for (int s = 0; s < SPB; ++s) {
      const int i = nb_full * SPB + s;
      if (i < T) step_at(i, eps + s * M);
    }
  }
  if (have) {
    const float c = Sys::cost_finish(pend, env) + pend_is;
    S.add(c);
    if (TOGO) sC[(T - 1) * BLK + tid] = c;
  }
  const float phi = Sys::cost(x, aux, env);
  S.add(phi);  // phi(x_T) = q(x_T)
  // the update kernel may start launching now (it waits for this grid's results itself)
  asm volatile("griddepcontrol.launch_dependents;");
  if (TOGO) {
    if (k < p.K) S_out[k] = isfinite(S.s) ? S.s : INFINITY;
    block_partial_to_go<M, BLK>(p, k0, phi, sC, sDu, part_sums, part_rho, part_eta, part);
    return;
  }
  block_partial<M, BLK, REGEN>(p, k, ctr, S.s, Lnu, S_out, part_sums, part, sW, sDu);
}

}  // namespace mppi
