// Fused MPPI rollout with the learned car dynamics on the tensor cores (sm_103a).
//
// One CTA owns 128 samples (the MMA tile's M) with nine warps:
//   epilogue warps 0..7  warp w reads TMEM lane quadrant w % 4 (rows 32 (w % 4) .. +31) and
//                        the column half (w / 4) * 128 of each hidden layer, 32 columns at
//                        a time; threads 0..127 also own one sample each (noise, features,
//                        state update, cost);
//   MMA warp 8           one thread issues every tcgen05.mma and commit.
// The weights are copied once into shared memory in the K-major core-matrix layout (bulk
// asynchronous copies completing on an mbarrier the MMA thread waits for).  TMEM
// (512 columns) holds the FP32 accumulators: layer 1 in columns 0..255, layer 2 in
// 256..511, the output layer in 0..15.  Per time step:
//   owners: noise du_i (Philox), v = u_i + du_i, features z(x, v) -> X tile    [bar_x]
//   MMA  D1 = X W1^T  (M=128, N=256, K=16)                                     [bar_l1]
//   epilogue 1: H[:, 32 c .. 32 c + 31] = tanh(D1 + b1) chunk by chunk        [hb[c]]
//   MMA  D2 = H W2^T, one 32-deep K chunk as soon as its H chunk is written    [bar_l2]
//   epilogue 2: H = tanh(D2 + b2) chunk by chunk (H overwritten in place)      [hb[c]]
//   MMA  D3 = H W3^T  (N=16), again one K chunk per H chunk                    [bar_l3]
//   owners: x += (D3 + b3) * out_scale, S~ += q(x) + IS running cost (Kahan FP32, the
//           cost-map loads of a step finished during the next step)
// so the second and third products run under the epilogues (tanh on the special-function
// unit) instead of after them.  tanh.approx's error (~2^-11) is below the BF16 step of the
// activations it feeds.  After the horizon the block forms its softmax partial with du
// regenerated from the counter-based generator (shared memory is full of weights).
// Every mbarrier wait is bounded; a thread whose wait runs out stops waiting, the kernel
// flags the error, the MMA thread drains its MMAs (bounded) and TMEM is freed.
// FP8 variant (kind::f8f6f4): weights, features and hidden activations in E4M3 (weights
// with a per-tensor scale s_l, so a layer's pre-activation is s_l * acc + b), K padded to
// 32 in the first layer, one 32-deep MMA per 32 bytes of K.
#include <cstdint>
#include <cuda_fp8.h>

#include "kernels.cuh"
#include "mlp_model.cuh"
#include "rollout_body.cuh"
#include "tc_common.cuh"

namespace mppi {

namespace {
constexpr int kMlpThreads = 288;   // 8 epilogue warps (two per TMEM lane quadrant) + 1 MMA warp
constexpr int kMlpMmaWarp = 8;
constexpr int kMlpSamples = 128;   // rows of the MMA tile; threads 0..127 own one sample each

// Shared-memory layout (bytes) for element size E (2 = BF16, 1 = E4M3); the first layer's
// K is 16 (BF16) or 32 (E4M3, zero padded) so that one MMA covers it.
template <int E>
struct MlpLayout {
  static constexpr uint32_t K1 = E == 2 ? 16 : 32;
  static constexpr uint32_t W2 = 0;                           // 256 x 256
  static constexpr uint32_t W1 = W2 + 256 * 256 * E;          // 256 x K1
  static constexpr uint32_t W3 = W1 + 256 * K1 * E;           // 16 x 256
  static constexpr uint32_t H = W3 + 16 * 256 * E;            // 128 x 256
  static constexpr uint32_t X = H + 128 * 256 * E;            // 128 x K1
  static constexpr uint32_t B = X + 128 * K1 * E;             // b1, b2, b3, out_scale, w_scale (f32)
  static constexpr uint32_t U = B + (256 + 256 + 16 + 8 + 4) * 4;  // sU, sRu, sHu (f32)
  static constexpr uint32_t kTmemCols = 512;
  static constexpr uint32_t D1 = 0, D2 = 256, D3 = 0;         // TMEM columns of the three products
  static constexpr int KK = E;                                // MMAs per 32 columns of K (16-bit: K = 16 per MMA)
};

// byte offset of element (r, k) in a K-major no-swizzle tile of R rows, element size E
template <int E>
__device__ __forceinline__ uint32_t tile_offset(int r, int k, int R) {
  constexpr int per = 16 / E;  // elements per 16-byte core-matrix row
  return static_cast<uint32_t>((((k / per) * (R >> 3) + (r >> 3)) << 7) + ((r & 7) << 4) + ((k % per) * E));
}

__device__ __forceinline__ uint32_t pack_e4m3x4(float a, float b, float c, float d) {
  const __nv_fp8x2_storage_t lo = __nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE, __NV_E4M3);
  const __nv_fp8x2_storage_t hi = __nv_cvt_float2_to_fp8x2(make_float2(c, d), __NV_SATFINITE, __NV_E4M3);
  return static_cast<uint32_t>(lo) | (static_cast<uint32_t>(hi) << 16);
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float v[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t *>(&h);
}

// H row `row`, columns [c0, c0 + 32) = tanh(scale * v + bias) in the tile format (v: the 32
// accumulator columns of this thread's lane, already loaded from TMEM).  The scale-and-bias
// FMAs go two columns per packed instruction (the same roundings as one fmaf per column).
template <int E>
__device__ __forceinline__ void hidden_store(float v[32], const float *bias, float scale, unsigned char *smem, int row,
                                             int c0) {
  static_assert(MlpLayout<E>::B % 16 == 0, "the biases are read as float4 vectors");
  const float2 sc = make_float2(scale, scale);
#pragma unroll
  for (int j = 0; j < 32; j += 4) {
    const float4 b = *reinterpret_cast<const float4 *>(bias + c0 + j);
    const float2 z0 = fma2(make_float2(v[j], v[j + 1]), sc, make_float2(b.x, b.y));
    const float2 z1 = fma2(make_float2(v[j + 2], v[j + 3]), sc, make_float2(b.z, b.w));
    v[j] = tc::tanh_approx(z0.x);
    v[j + 1] = tc::tanh_approx(z0.y);
    v[j + 2] = tc::tanh_approx(z1.x);
    v[j + 3] = tc::tanh_approx(z1.y);
  }
  if (E == 2) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint4 w = make_uint4(pack_bf16(v[q * 8], v[q * 8 + 1]), pack_bf16(v[q * 8 + 2], v[q * 8 + 3]),
                                 pack_bf16(v[q * 8 + 4], v[q * 8 + 5]), pack_bf16(v[q * 8 + 6], v[q * 8 + 7]));
      *reinterpret_cast<uint4 *>(smem + MlpLayout<E>::H + tile_offset<E>(row, c0 + q * 8, 128)) = w;
    }
  } else {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const float *f = v + q * 16;
      const uint4 w = make_uint4(pack_e4m3x4(f[0], f[1], f[2], f[3]), pack_e4m3x4(f[4], f[5], f[6], f[7]),
                                 pack_e4m3x4(f[8], f[9], f[10], f[11]), pack_e4m3x4(f[12], f[13], f[14], f[15]));
      *reinterpret_cast<uint4 *>(smem + MlpLayout<E>::H + tile_offset<E>(row, c0 + q * 16, 128)) = w;
    }
  }
}

// order in which the MMA thread consumes the 32-column chunks of H: the two column halves
// are written side by side (warps 0..3 and 4..7), so chunks c and c + 4 complete together
__device__ __forceinline__ int chunk_at(int n) { return (n >> 1) + ((n & 1) << 2); }

template <int E>
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if (E == 2)
    tc::mma_bf16(d, a, b, idesc, acc);
  else
    tc::mma_e4m3(d, a, b, idesc, acc);
}

}  // namespace

template <int E>
__global__ void __launch_bounds__(kMlpThreads, 1) k_rollout_mlp(const CtrlParams p, const float *__restrict__ x0,
                                                                const CtrlState *__restrict__ st,
                                                                const float *__restrict__ U, float *__restrict__ S_out,
                                                                float *__restrict__ part_sums,
                                                                BlockPartial *__restrict__ part) {
  constexpr int M = 2, N = 7;
  using L = MlpLayout<E>;
  extern __shared__ __align__(1024) unsigned char smem[];
  // bar_x: X tile written (128 owner threads); bar_l1/l2/l3: products done (MMA commits);
  // hb[c]: H columns 32c..32c+31 written (128 threads of one column half), twice per step;
  // bar_drain: the MMA thread's last commit before TMEM is freed
  __shared__ uint64_t bar_x, bar_l1, bar_l2, bar_l3, bar_drain, hb[8], bar_w;
  __shared__ uint32_t tmem_base;
  const MlpDev *md = static_cast<const MlpDev *>(p.mlp);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int T = p.T, TM = T * M;
  float *sb1 = reinterpret_cast<float *>(smem + L::B);
  float *sb2 = sb1 + 256;
  float *sb3 = sb2 + 256;
  float *sscale = sb3 + 16;
  float *swscale = sscale + 8;
  float *sU = reinterpret_cast<float *>(smem + L::U);
  float *sRu = sU + TM;
  float *sHu = sRu + TM;

  if (warp == 0) tc::tmem_alloc(&tmem_base, L::kTmemCols);
  if (tid == 0) {
    tc::mbar_init(&bar_x, kMlpSamples);
    tc::mbar_init(&bar_l1, 1);
    tc::mbar_init(&bar_l2, 1);
    tc::mbar_init(&bar_l3, 1);
    tc::mbar_init(&bar_drain, 1);
    for (int c = 0; c < 8; ++c) tc::mbar_init(&hb[c], 128);
    tc::mbar_init(&bar_w, 1);
    tc::fence_mbar_init();
    // weights (already in tile layout): three bulk copies completing on bar_w, read only by
    // the MMAs (which wait for them)
    constexpr uint32_t b2 = 256 * 256 * E, b1 = 256 * L::K1 * E, b3 = 16 * 256 * E;
    tc::mbar_arrive_expect_tx(&bar_w, b1 + b2 + b3);
    tc::bulk_g2s(smem + L::W2, md->w2, b2, &bar_w);
    tc::bulk_g2s(smem + L::W1, md->w1, b1, &bar_w);
    tc::bulk_g2s(smem + L::W3, md->w3, b3, &bar_w);
  }
  // biases and scales
  {
    for (int i = tid; i < 256; i += kMlpThreads) {
      sb1[i] = md->b1[i];
      sb2[i] = md->b2[i];
    }
    if (tid < 16) sb3[tid] = md->b3[tid];
    if (tid < 8) sscale[tid] = md->out_scale[tid];
    if (tid < 3) swscale[tid] = md->w_scale[tid];
  }
  __shared__ float sx0[N];  // x0 staged once (it may live in mapped host memory)
  for (int o = tid; o < TM; o += kMlpThreads) sU[o] = U[o];
  if (tid < N) sx0[tid] = x0[tid];
  __syncthreads();
  for (int i = tid; i < T; i += kMlpThreads) {
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
  tc::fence_smem_to_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();

  const uint32_t tmem = tmem_base;
  const uint32_t ctr = st->counter;
  const bool owner = tid < kMlpSamples;
  const int k = blockIdx.x * kMlpSamples + tid;
  float Lnu[M * M];
#pragma unroll
  for (int a = 0; a < M * M; ++a) Lnu[a] = p.Lnu[a];
  bool ok = true;
  float Sk = INFINITY;

  if (warp == kMlpMmaWarp) {
    // ---- MMA issue ---------------------------------------------------------------------
    if ((tid & 31) == 0) {
      const uint32_t sbase = tc::smem_u32(smem);
      const uint32_t id256 = E == 2 ? tc::idesc_bf16_f32(128, 256) : tc::idesc_e4m3_f32(128, 256);
      const uint32_t id16 = E == 2 ? tc::idesc_bf16_f32(128, 16) : tc::idesc_e4m3_f32(128, 16);
      ok = tc::mbar_wait(&bar_w, 0u);  // the weight tiles are in shared memory
      for (int i = 0; i < T && ok; ++i) {
        const uint32_t ph = static_cast<uint32_t>(i & 1);
        ok = tc::mbar_wait(&bar_x, ph);
        if (!ok) break;
        tc::fence_after_sync();
        mma<E>(tmem + L::D1, tc::smem_desc(sbase + L::X, 128 * 16, 128), tc::smem_desc(sbase + L::W1, 256 * 16, 128),
               id256, 0u);
        tc::mma_commit(&bar_l1);
        // layer 2: K chunk c (32 columns of H) as soon as epilogue 1 wrote it
        for (int n = 0; n < 8 && ok; ++n) {
          const int c = chunk_at(n);
          ok = tc::mbar_wait(&hb[c], 0u);
          if (!ok) break;
          tc::fence_after_sync();
#pragma unroll
          for (int q = 0; q < L::KK; ++q) {
            const int kk = c * L::KK + q;
            mma<E>(tmem + L::D2, tc::smem_desc(sbase + L::H + kk * 2 * 2048, 2048, 128),
                   tc::smem_desc(sbase + L::W2 + kk * 2 * 4096, 4096, 128), id256, (n | q) ? 1u : 0u);
          }
        }
        if (!ok) break;
        tc::mma_commit(&bar_l2);
        // output layer: K chunk c as soon as epilogue 2 wrote it
        for (int n = 0; n < 8 && ok; ++n) {
          const int c = chunk_at(n);
          ok = tc::mbar_wait(&hb[c], 1u);
          if (!ok) break;
          tc::fence_after_sync();
#pragma unroll
          for (int q = 0; q < L::KK; ++q) {
            const int kk = c * L::KK + q;
            mma<E>(tmem + L::D3, tc::smem_desc(sbase + L::H + kk * 2 * 2048, 2048, 128),
                   tc::smem_desc(sbase + L::W3 + kk * 2 * 256, 256, 128), id16, (n | q) ? 1u : 0u);
          }
        }
        if (!ok) break;
        tc::mma_commit(&bar_l3);
      }
      // every MMA issued above has completed once this commit arrives
      tc::mma_commit(&bar_drain);
      if (!tc::mbar_wait(&bar_drain, 0u)) ok = false;
    }
  } else {
    // ---- epilogue warps (threads 0..127 also own the samples) ---------------------------
    const uint32_t tmem_row = tmem + (static_cast<uint32_t>(32 * (warp & 3)) << 16);
    const int erow = 32 * (warp & 3) + (tid & 31);  // epilogue row (= sample) of this thread
    const int half = warp >> 2;                     // column half of this warp
    const float s1 = swscale[0], s2 = swscale[1], s3 = swscale[2];
    const Env env = make_env(p, nullptr);
    float R[M * M];
#pragma unroll
    for (int a = 0; a < M * M; ++a) R[a] = p.R[a];
    float x[N];
#pragma unroll
    for (int a = 0; a < N; ++a) x[a] = sx0[a];
    KahanSum S;
    float eps[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    // control v_i = u_i + du_i and IS running term of step i (owners); step i+1's are
    // drawn during step i's second epilogue, off the step's critical path
    float v_cur[M] = {0.0f, 0.0f}, is_cur = 0.0f;
    auto noise_step = [&](int i, float v[M], float &is) {
      if ((i & 1) == 0)
        normals4(static_cast<uint32_t>(i >> 1), static_cast<uint32_t>(k), ctr, p.gid, p.key_lo, p.key_hi, eps);
      float du[M];
      {
        const float pair[2] = {(i & 1) ? eps[2] : eps[0], (i & 1) ? eps[3] : eps[1]};
        scale_noise<M>(Lnu, pair, du);
      }
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
      is = p.is_du * duRdu + uRdu + sHu[i];
    };
    // one hidden layer's epilogue for this warp's column half: the TMEM load of chunk q+1 is
    // in flight while chunk q is activated and stored; mid() runs after the second chunk
    auto epilogue = [&](uint32_t dcol, const float *bias, float scale, auto mid) {
      float va[32], vb[32];
      tmem_ld32(tmem_row + dcol + 32 * (half * 4), va);
      tc::tmem_ld_wait();
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int c = half * 4 + q;
        float *cur = (q & 1) ? vb : va;
        float *nxt = (q & 1) ? va : vb;
        if (q < 3) tmem_ld32(tmem_row + dcol + 32 * (c + 1), nxt);
        hidden_store<E>(cur, bias, scale, smem, erow, 32 * c);
        tc::fence_smem_to_async();
        tc::fence_before_sync();
        tc::mbar_arrive(&hb[c]);
        if (q == 1) mid();
        if (q < 3) tc::tmem_ld_wait();
      }
    };
    // the previous step's state cost is combined one step late (its map loads in flight meanwhile)
    bool have_pend = false;
    const float *pend_row = nullptr;
    float pend_tx = 0.0f, pend_ty = 0.0f, pend_speed = 0.0f, pend_is = 0.0f;
    if (owner) noise_step(0, v_cur, is_cur);
    for (int i = 0; i < T && ok; ++i) {
      const uint32_t ph = static_cast<uint32_t>(i & 1);
      if (owner) {
        float z[mlp::kIn];
        mlp::features(x, v_cur, z);
        if (E == 2) {
          const uint4 a = make_uint4(pack_bf16(z[0], z[1]), pack_bf16(z[2], z[3]), pack_bf16(z[4], z[5]),
                                     pack_bf16(z[6], z[7]));
          const uint4 b = make_uint4(pack_bf16(z[8], z[9]), pack_bf16(z[10], z[11]), pack_bf16(z[12], z[13]),
                                     pack_bf16(z[14], z[15]));
          *reinterpret_cast<uint4 *>(smem + L::X + tile_offset<E>(tid, 0, 128)) = a;
          *reinterpret_cast<uint4 *>(smem + L::X + tile_offset<E>(tid, 8, 128)) = b;
        } else {
          const uint4 a = make_uint4(pack_e4m3x4(z[0], z[1], z[2], z[3]), pack_e4m3x4(z[4], z[5], z[6], z[7]),
                                     pack_e4m3x4(z[8], z[9], z[10], z[11]), pack_e4m3x4(z[12], z[13], z[14], z[15]));
          *reinterpret_cast<uint4 *>(smem + L::X + tile_offset<E>(tid, 0, 128)) = a;
          *reinterpret_cast<uint4 *>(smem + L::X + tile_offset<E>(tid, 16, 128)) = make_uint4(0u, 0u, 0u, 0u);
        }
        tc::fence_smem_to_async();
        tc::fence_before_sync();
        tc::mbar_arrive(&bar_x);
        // the previous step's cost, its map loads issued a step ago
        if (have_pend) {
          const float m00 = __ldg(pend_row), m10 = __ldg(pend_row + 1);
          const float m01 = __ldg(pend_row + env.map_w), m11 = __ldg(pend_row + env.map_w + 1);
          const float aa = m00 + pend_tx * (m10 - m00);
          const float bb = m01 + pend_tx * (m11 - m01);
          S.add((aa + pend_ty * (bb - aa)) + pend_speed + pend_is);
        }
      }
      // epilogue 1
      ok = tc::mbar_wait(&bar_l1, ph);
      if (!ok) break;
      tc::fence_after_sync();
      epilogue(L::D1, sb1, s1, [] {});
      // epilogue 2 (H is overwritten only after every layer-2 MMA has read it)
      ok = tc::mbar_wait(&bar_l2, ph);
      if (!ok) break;
      tc::fence_after_sync();
      float v_nxt[M] = {0.0f, 0.0f}, is_nxt = 0.0f;
      epilogue(L::D2, sb2, s2, [&] {
        if (owner && i + 1 < T) noise_step(i + 1, v_nxt, is_nxt);
      });
      if (owner) {  // warps 0..3: TMEM lane quadrant = warp, row = sample
        ok = tc::mbar_wait(&bar_l3, ph);
        if (!ok) break;
        tc::fence_after_sync();
        float y[16];
        tc::tmem_ld8(tmem_row + L::D3, y);
        tc::tmem_ld8(tmem_row + L::D3 + 8, y + 8);
        tc::tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < N; ++j) x[j] += fmaf(y[j], s3, sb3[j]) * sscale[j];
        // cost of the new state: map loads issued now, combined next step (same sum order)
        const float fx = fminf(fmaxf((x[0] - env.map_ox) * env.map_inv_cell, 0.0f), static_cast<float>(env.map_w - 1));
        const float fy = fminf(fmaxf((x[1] - env.map_oy) * env.map_inv_cell, 0.0f), static_cast<float>(env.map_h - 1));
        const int ix = min(static_cast<int>(fx), env.map_w - 2);
        const int iy = min(static_cast<int>(fy), env.map_h - 2);
        pend_tx = fx - static_cast<float>(ix);
        pend_ty = fy - static_cast<float>(iy);
        pend_row = env.map + static_cast<size_t>(iy) * env.map_w + ix;
        const float dv = x[3] - Car::v_target;
        pend_speed = fmaf(dv, dv, position_nan(x[0], x[1]));
        pend_is = is_cur;
        have_pend = true;
        v_cur[0] = v_nxt[0];
        v_cur[1] = v_nxt[1];
        is_cur = is_nxt;
      }
    }
    if (ok && owner) {
      if (have_pend) {
        const float m00 = __ldg(pend_row), m10 = __ldg(pend_row + 1);
        const float m01 = __ldg(pend_row + env.map_w), m11 = __ldg(pend_row + env.map_w + 1);
        const float aa = m00 + pend_tx * (m10 - m00);
        const float bb = m01 + pend_tx * (m11 - m01);
        S.add((aa + pend_ty * (bb - aa)) + pend_speed + pend_is);
      }
      const float dv = x[3] - Car::v_target;
      S.add(map_bilinear(env, x[0], x[1]) + dv * dv);  // phi(x_T) = q(x_T)
      Sk = S.s;
    }
  }
  tc::fence_before_sync();
  if (!__syncthreads_and(ok)) {
    Sk = INFINITY;
    if (tid == 0) atomicExch(md->err, 1);
  }
  tc::fence_after_sync();
  // the update kernel may start launching now (it waits for this grid's results itself)
  asm volatile("griddepcontrol.launch_dependents;");
  block_partial<M, kMlpThreads, true>(p, owner ? k : INT_MAX, ctr, Sk, Lnu, S_out,
                                      part_sums + static_cast<size_t>(blockIdx.x) * TM, part + blockIdx.x, nullptr,
                                      nullptr);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, L::kTmemCols);
  if (tid == 0) tc::mbar_wait(&bar_w, 0u);  // no weight copy still in flight when the CTA exits
}

size_t mlp_rollout_smem_bytes(int T, int precision) {
  const size_t base = precision == 0 ? MlpLayout<2>::U : MlpLayout<1>::U;
  return base + sizeof(float) * (2 * static_cast<size_t>(T) * 2 + T);
}

cudaError_t launch_rollout_mlp(const CtrlParams &p, const float *x0, const CtrlState *st, const float *U, float *S,
                               float *part_sums, BlockPartial *part, int precision, cudaStream_t s) {
  const size_t smem = mlp_rollout_smem_bytes(p.T, precision);
  const int grid = (p.K + kMlpSamples - 1) / kMlpSamples;
  if (precision == 0)
    k_rollout_mlp<2><<<grid, kMlpThreads, smem, s>>>(p, x0, st, U, S, part_sums, part);
  else
    k_rollout_mlp<1><<<grid, kMlpThreads, smem, s>>>(p, x0, st, U, S, part_sums, part);
  return cudaGetLastError();
}

cudaError_t prepare_mlp_kernel() {
  cudaError_t e = cudaFuncSetAttribute(k_rollout_mlp<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(kMlpSmemLimit));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_rollout_mlp<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(kMlpSmemLimit));
  return e;
}

}  // namespace mppi
