// Generic BF16 tensor-core GEMM for sm_103a (tcgen05, accumulator in TMEM), with
// fused epilogues, used by the learned-dynamics training step.
//
//   C[M x N] = A[M x K] . B[K x N],   A(m, k) = A[m*sam + k*sak],  B(k, n) = B[k*sbk + n*sbn]
//
// One CTA (128 threads) per 128 x BN output tile.  Each 64-wide K slab of A and B is
// gathered from global memory by all threads (any strides, so transposed operands cost
// nothing extra) into the no-swizzle K-major core-matrix layout, then one elected
// thread issues the 16-deep tcgen05.mma instructions and commits them to an mbarrier.
// The epilogue reads the FP32 accumulator back with tcgen05.ld (warp w owns TMEM lanes
// 32w..32w+31, i.e. output rows) and applies the fused operation.
#include <cstdint>

#include "kernels.cuh"
#include "tc_common.cuh"
#include "tc_gemm.cuh"

namespace mppi {

namespace {
constexpr int kBM = 128, kKT = 64, kThreads = 128;
constexpr uint32_t kTmemCols = 512;
}  // namespace

__global__ void __launch_bounds__(kThreads, 1) k_gemm_bf16(const GemmArgs g) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * g.BN;
  const int BN = g.BN;
  unsigned char *sA = smem;               // [128 x 64] K-major
  unsigned char *sB = smem + 128 * kKT * 2;  // [BN x 64] K-major

  if (warp == 0) tc::tmem_alloc(&tmem_base, kTmemCols);
  if (tid == 0) tc::mbar_init(&bar, 1);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = tc::idesc_bf16_f32(kBM, BN);
  const uint32_t wait_limit = g.wait_limit ? g.wait_limit : tc::kWaitLimit;
  uint32_t phase = 0;
  bool ok = true;

  // split-K: this CTA reduces K in [kbeg, kend)
  const int nsplit = g.ksplit > 1 ? g.ksplit : 1;
  const int kchunk = ((g.K + nsplit - 1) / nsplit + kKT - 1) / kKT * kKT;
  const int kbeg = blockIdx.z * kchunk, kend = min(g.K, kbeg + kchunk);
  const int64_t csn = g.ldcn ? g.ldcn : 1;
  for (int k0 = kbeg; k0 < kend && ok; k0 += kKT) {
    const int klen = min(kKT, kend - k0);
    const int kpad = (klen + 15) & ~15;
    // gather the A slab
    for (int idx = tid; idx < kBM * kpad; idx += kThreads) {
      int r, c;
      if (g.sak == 1) {
        r = idx / kpad;
        c = idx % kpad;
      } else {
        r = idx % kBM;
        c = idx / kBM;
      }
      const int m = m0 + r, k = k0 + c;
      __nv_bfloat16 v = __float2bfloat16(0.0f);
      if (m < g.M && c < klen) v = g.A[static_cast<int64_t>(m) * g.sam + static_cast<int64_t>(k) * g.sak];
      *reinterpret_cast<__nv_bfloat16 *>(sA + tc::kmajor_offset(r, c, kBM)) = v;
    }
    // gather the B slab (rows = n)
    for (int idx = tid; idx < BN * kpad; idx += kThreads) {
      int r, c;
      if (g.sbk == 1) {
        r = idx / kpad;
        c = idx % kpad;
      } else {
        r = idx % BN;
        c = idx / BN;
      }
      const int n = n0 + r, k = k0 + c;
      __nv_bfloat16 v = __float2bfloat16(0.0f);
      if (n < g.N && c < klen) v = g.B[static_cast<int64_t>(k) * g.sbk + static_cast<int64_t>(n) * g.sbn];
      *reinterpret_cast<__nv_bfloat16 *>(sB + tc::kmajor_offset(r, c, BN)) = v;
    }
    tc::fence_smem_to_async();
    __syncthreads();
    if (tid == 0 && !g.debug_skip_mma) {
      tc::fence_after_sync();
      const uint32_t a0 = tc::smem_u32(sA), b0 = tc::smem_u32(sB);
      const uint32_t lbo_a = kBM * 16, lbo_b = BN * 16;
      for (int kk = 0; kk < kpad / 16; ++kk) {
        const uint64_t ad = tc::smem_desc(a0 + kk * 2 * lbo_a, lbo_a, 128);
        const uint64_t bd = tc::smem_desc(b0 + kk * 2 * lbo_b, lbo_b, 128);
        tc::mma_bf16(tmem, ad, bd, idesc, (k0 > kbeg || kk > 0) ? 1u : 0u);
      }
      tc::mma_commit(&bar);
    }
    const bool got = tc::mbar_wait(&bar, phase, wait_limit);
    phase ^= 1u;
    tc::fence_after_sync();
    ok = __syncthreads_and(got) != 0;  // block-uniform
  }

  if (!ok) {
    if (tid == 0) atomicExch(g.err, 1);
    tc::mbar_wait(&bar, phase ^ 1u, wait_limit);  // second, bounded chance for the MMAs in flight
  } else {
    // epilogue: row m = m0 + 32*warp + lane, columns n0 .. n0+BN
    const int m = m0 + 32 * warp + lane;
    const bool empty = kbeg >= kend;  // a split with no K range contributes nothing
    for (int c0 = 0; c0 < BN && !empty; c0 += 8) {
      float v[8];
      tc::tmem_ld8(tmem + (static_cast<uint32_t>(32 * warp) << 16) + static_cast<uint32_t>(c0), v);
      tc::tmem_ld_wait();
      if (m < g.M) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int n = n0 + c0 + j;
          if (n >= g.N) continue;
          float a = g.alpha * v[j];
          switch (g.mode) {
            case kEpiStoreF32:
              g.Cf[static_cast<int64_t>(m) * g.ldc + n * csn] = a;
              break;
            case kEpiAddF32:
              g.Cf[static_cast<int64_t>(m) * g.ldc + n * csn] += a;
              break;
            case kEpiAtomicF32:
              atomicAdd(&g.Cf[static_cast<int64_t>(m) * g.ldc + n * csn], a);
              break;
            case kEpiBiasTanh: {
              const float h = tanhf(a + g.bias[n]);
              g.Cb[static_cast<int64_t>(m) * g.ldcb + n] = __float2bfloat16(h);
              if (g.Cf) g.Cf[static_cast<int64_t>(m) * g.ldc + n * csn] = h;
              break;
            }
            case kEpiBiasF32:
              g.Cf[static_cast<int64_t>(m) * g.ldc + n * csn] = a + g.bias[n];
              break;
            case kEpiTanhGrad: {
              const float h = __bfloat162float(g.H[static_cast<int64_t>(m) * g.ldh + n]);
              g.Cb[static_cast<int64_t>(m) * g.ldcb + n] = __float2bfloat16(a * (1.0f - h * h));
              break;
            }
            default:
              break;
          }
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

size_t gemm_smem_bytes() { return kGemmSmemBytes; }

cudaError_t launch_gemm_bf16(const GemmArgs &g, cudaStream_t s) {
  static bool attr_set = false;
  if (!attr_set) {
    const cudaError_t e = cudaFuncSetAttribute(k_gemm_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               static_cast<int>(kGemmSmemBytes));
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  if (g.BN < 16 || g.BN > 256 || (g.BN & 15) != 0) return cudaErrorInvalidValue;
  const int nsplit = g.ksplit > 1 ? g.ksplit : 1;
  if (nsplit > 1 && g.mode != kEpiAtomicF32) return cudaErrorInvalidValue;
  const dim3 grid((g.M + kBM - 1) / kBM, (g.N + g.BN - 1) / g.BN, nsplit);
  k_gemm_bf16<<<grid, kThreads, kGemmSmemBytes, s>>>(g);
  return cudaGetLastError();
}

}  // namespace mppi

// ---------------------------------------------------------------------------
// C ABI check hook: C (FP32, row-major, ldc) = A . B on device buffers.
// ---------------------------------------------------------------------------
extern "C" int mppi_debug_gemm_bf16(int M, int N, int K, const void *dA, int64_t sam, int64_t sak, const void *dB,
                                    int64_t sbk, int64_t sbn, float *dC, int64_t ldc, int BN) {
  using namespace mppi;
  if (M < 1 || N < 1 || K < 1 || !dA || !dB || !dC || BN < 16 || BN > 256 || (BN & 15)) return -1;
  int *d_err = nullptr;
  if (cudaMalloc(&d_err, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return -2;
  }
  cudaMemset(d_err, 0, sizeof(int));
  GemmArgs g{};
  g.M = M;
  g.N = N;
  g.K = K;
  g.BN = BN;
  g.A = static_cast<const __nv_bfloat16 *>(dA);
  g.sam = sam;
  g.sak = sak;
  g.B = static_cast<const __nv_bfloat16 *>(dB);
  g.sbk = sbk;
  g.sbn = sbn;
  g.mode = kEpiStoreF32;
  g.alpha = 1.0f;
  g.Cf = dC;
  g.ldc = ldc;
  g.err = d_err;
  cudaError_t e = launch_gemm_bf16(g, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  int err = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&err, d_err, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(d_err);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return -3;
  }
  return err ? -4 : 0;
}

// ---------------------------------------------------------------------------
// C ABI check hook of the bounded-wait exit path: one GEMM CTA (128 x 128 x 128, zero
// operands) whose MMA issuer issues nothing, so its accumulator barrier never completes; the
// waits give up after `polls` polls, the kernel raises its error flag, frees its TMEM and
// returns.  Nothing asynchronous (no MMA, no bulk copy) is outstanding when it does.
// ---------------------------------------------------------------------------
extern "C" int mppi_debug_gemm_wait_timeout(uint32_t polls) {
  using namespace mppi;
  if (polls < 1 || polls > (1u << 20)) return -1;
  constexpr int M = 128, N = 128, K = 128;
  void *buf = nullptr;
  const size_t ab = sizeof(__nv_bfloat16) * M * K, cb = sizeof(float) * M * N;
  if (cudaMalloc(&buf, 2 * ab + cb + 256) != cudaSuccess) {
    cudaGetLastError();
    return -2;
  }
  cudaError_t e = cudaMemset(buf, 0, 2 * ab + cb + 256);
  GemmArgs g{};
  g.M = M;
  g.N = N;
  g.K = K;
  g.BN = N;
  g.A = static_cast<const __nv_bfloat16 *>(buf);
  g.sam = K;
  g.sak = 1;
  g.B = reinterpret_cast<const __nv_bfloat16 *>(static_cast<char *>(buf) + ab);
  g.sbk = N;
  g.sbn = 1;
  g.mode = kEpiStoreF32;
  g.alpha = 1.0f;
  g.Cf = reinterpret_cast<float *>(static_cast<char *>(buf) + 2 * ab);
  g.ldc = N;
  g.err = reinterpret_cast<int *>(static_cast<char *>(buf) + 2 * ab + cb);
  g.wait_limit = polls;
  g.debug_skip_mma = 1;
  if (e == cudaSuccess) e = launch_gemm_bf16(g, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  int err = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&err, g.err, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(buf);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return -3;
  }
  return err ? -4 : 0;
}
