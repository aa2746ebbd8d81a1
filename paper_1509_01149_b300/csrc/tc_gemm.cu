// Generic BF16 tensor-core GEMM for sm_103a (tcgen05, accumulator in TMEM), with
// fused epilogues, used by the learned-dynamics training step.
//
//   C[M x N] = A[M x K] . B[K x N],   A(m, k) = A[m*sam + k*sak],  B(k, n) = B[k*sbk + n*sbn]
//
// One CTA (128 threads) per 128 x BN output tile.  Each 64-wide K slab of A and B is
// gathered from global memory by all threads into the no-swizzle K-major core-matrix layout
// (any strides, so transposed operands need no copy): where 8 consecutive elements are
// contiguous in memory along K, one 16-byte asynchronous copy (cp.async) per core-matrix row,
// every copy of the slab in flight at once; where they are contiguous along the rows, every
// 16-byte load of the thread first, then each feeds 8 rows; element-wise loads otherwise.
// The CTA takes only the TMEM columns (BN, rounded up to a power of two) and the shared memory
// (two stages of 16 KB + BN x 128 B) its tile needs, so two or more CTAs share an SM and hide
// each other's gather latency.  Two shared-memory stages:
// while the tensor core multiplies slab s (one elected thread issues the 16-deep
// tcgen05.mma instructions and commits them to the stage's mbarrier), the threads gather slab
// s + 1 into the other stage, after the MMAs of slab s - 1 have released it.  The epilogue
// reads the FP32 accumulator back with tcgen05.ld (warp w owns TMEM lanes 32w..32w+31, i.e.
// output rows) and applies the fused operation.  Split-K (gridDim.z > 1) either adds into C
// atomically (kEpiAtomicF32) or stores each split's partial product to its own slice
// Cf + z * split_stride (kEpiStoreF32), for a reduction in a fixed order afterwards.
#include <cstdint>

#include "kernels.cuh"
#include "tc_common.cuh"
#include "tc_gemm.cuh"

namespace mppi {

namespace {
constexpr int kBM = 128, kKT = 64, kThreads = 128;
constexpr uint32_t kStageA = kBM * kKT * 2;     // 16 KB
__host__ __device__ constexpr uint32_t stage_bytes(int BN) { return kStageA + static_cast<uint32_t>(BN) * kKT * 2; }
static_assert(2 * stage_bytes(256) <= kGemmSmemBytes, "two stages of the widest tile fit the dynamic shared memory");
// TMEM columns of a 128 x BN FP32 accumulator: a power of two, at least 32
__device__ __forceinline__ uint32_t tmem_cols(int BN) {
  return BN <= 32 ? 32u : BN <= 64 ? 64u : BN <= 128 ? 128u : 256u;
}
constexpr int kMaxRowLoads = 16;  // 16-byte loads per thread of one operand slab (256 rows x 64 k)

__device__ __forceinline__ bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// 16-byte asynchronous global -> shared copy; src_bytes 0 fills the 16 bytes with zeros
__device__ __forceinline__ void cp_async16(void *dst, const void *src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(tc::smem_u32(dst)), "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// 32 consecutive FP32 accumulator columns of this thread's TMEM lane (wait with tmem_ld_wait)
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

// Rows [r0, r0 + Rn) x K slab [k0, k0 + klen) of X(r, k) = X[r*srow + k*sk] (rows >= nrows and
// k >= klen read as 0) into the K-major core-matrix tile `dst` with Rn rows and kpad columns.
// KIND: kGatherK (8 elements contiguous along K), kGatherRows (8 rows contiguous at one k), or
// kGatherAny (chosen per call from the strides and alignment, element-wise if neither).  The
// launcher picks the kind from the same conditions, so that the common kernels carry only the
// code of their own gathers (a smaller instruction footprint for the four warps of a CTA).
constexpr int kGatherK = 0, kGatherRows = 1, kGatherAny = 2;

template <int KIND>
__device__ __forceinline__ void gather_tile(const __nv_bfloat16 *__restrict__ X, int64_t srow, int64_t sk, int r0,
                                            int nrows, int Rn, int k0, int klen, int kpad, unsigned char *dst,
                                            int tid) {
  const __nv_bfloat16 zero = __float2bfloat16(0.0f);
  if (KIND == kGatherK || (KIND == kGatherAny && sk == 1 && (srow & 7) == 0 && aligned16(X))) {
    // eight consecutive k of one row: one 16-byte asynchronous copy per core-matrix row (zeros
    // past the last row or past klen); a chunk that klen cuts is gathered element-wise
    const int cpr = kpad >> 3;
    for (int idx = tid; idx < Rn * cpr; idx += kThreads) {
      const int r = idx / cpr, c = (idx - r * cpr) << 3;
      const int row = r0 + r;
      unsigned char *d = dst + tc::kmajor_offset(r, c, Rn);
      const __nv_bfloat16 *src = X + static_cast<int64_t>(row) * srow + k0 + c;
      if (row >= nrows || c >= klen) {
        cp_async16(d, X, 0u);
      } else if (c + 8 <= klen) {
        cp_async16(d, src, 16u);
      } else {
        __nv_bfloat16 t[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) t[e] = c + e < klen ? src[e] : zero;
        *reinterpret_cast<uint4 *>(d) = *reinterpret_cast<const uint4 *>(t);
      }
    }
  } else if (KIND == kGatherRows ||
             (KIND == kGatherAny && srow == 1 && (sk & 7) == 0 && (r0 & 7) == 0 && aligned16(X) &&
              (Rn >> 3) * kpad <= kMaxRowLoads * kThreads)) {
    // eight consecutive rows at one k: every 16-byte load of the thread is issued first, then
    // each feeds eight core-matrix rows
    const int groups = Rn >> 3, total = groups * kpad;
    uint4 v[kMaxRowLoads];
#pragma unroll
    for (int it = 0; it < kMaxRowLoads; ++it) {
      const int idx = tid + it * kThreads;
      v[it] = make_uint4(0u, 0u, 0u, 0u);
      if (idx < total) {
        const int c = idx / groups, r = (idx - c * groups) << 3;
        const int row = r0 + r;
        if (c < klen) {
          const __nv_bfloat16 *src = X + row + static_cast<int64_t>(k0 + c) * sk;
          if (row + 8 <= nrows) {
            v[it] = *reinterpret_cast<const uint4 *>(src);
          } else {
            __nv_bfloat16 t[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) t[e] = row + e < nrows ? src[e] : zero;
            v[it] = *reinterpret_cast<const uint4 *>(t);
          }
        }
      }
    }
#pragma unroll
    for (int it = 0; it < kMaxRowLoads; ++it) {
      const int idx = tid + it * kThreads;
      if (idx < total) {
        const int c = idx / groups, r = (idx - c * groups) << 3;
        const __nv_bfloat16 *e = reinterpret_cast<const __nv_bfloat16 *>(&v[it]);
#pragma unroll
        for (int i = 0; i < 8; ++i) *reinterpret_cast<__nv_bfloat16 *>(dst + tc::kmajor_offset(r + i, c, Rn)) = e[i];
      }
    }
  } else if (KIND == kGatherAny) {
    for (int idx = tid; idx < Rn * kpad; idx += kThreads) {
      int r, c;
      if (sk == 1) {
        r = idx / kpad;
        c = idx % kpad;
      } else {
        r = idx % Rn;
        c = idx / Rn;
      }
      const int row = r0 + r;
      __nv_bfloat16 v = zero;
      if (row < nrows && c < klen) v = X[static_cast<int64_t>(row) * srow + static_cast<int64_t>(k0 + c) * sk];
      *reinterpret_cast<__nv_bfloat16 *>(dst + tc::kmajor_offset(r, c, Rn)) = v;
    }
  }
}
}  // namespace

template <int GA, int GB>
__global__ void __launch_bounds__(kThreads, 1) k_gemm_bf16(const GemmArgs g) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint64_t bar[2];
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * g.BN;
  const int BN = g.BN;

  const uint32_t ncols = tmem_cols(g.BN);
  const uint32_t sbytes = stage_bytes(g.BN);
  if (warp == 0) tc::tmem_alloc(&tmem_base, ncols);
  if (tid == 0) {
    tc::mbar_init(&bar[0], 1);
    tc::mbar_init(&bar[1], 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = tc::idesc_bf16_f32(kBM, BN);
  const uint32_t wait_limit = g.wait_limit ? g.wait_limit : tc::kWaitLimit;
  bool ok = true;

  // split-K: this CTA reduces K in [kbeg, kend)
  const int nsplit = g.ksplit > 1 ? g.ksplit : 1;
  const int kchunk = ((g.K + nsplit - 1) / nsplit + kKT - 1) / kKT * kKT;
  const int kbeg = blockIdx.z * kchunk, kend = min(g.K, kbeg + kchunk);
  const int ns = kbeg < kend ? (kend - kbeg + kKT - 1) / kKT : 0;  // K slabs
  auto gather = [&](int s) {
    const int k0 = kbeg + s * kKT, klen = min(kKT, kend - k0), kpad = (klen + 15) & ~15;
    unsigned char *sA = smem + (s & 1) * sbytes, *sB = sA + kStageA;
    gather_tile<GA>(g.A, g.sam, g.sak, m0, g.M, kBM, k0, klen, kpad, sA, tid);
    gather_tile<GB>(g.B, g.sbn, g.sbk, n0, g.N, BN, k0, klen, kpad, sB, tid);
    cp_async_wait_all();  // this thread's asynchronous copies have landed
  };
  int last = -1;  // the last slab whose MMAs were committed
  if (ns > 0) {
    gather(0);
    tc::fence_smem_to_async();
    __syncthreads();
    for (int s = 0; s < ns; ++s) {
      if (tid == 0 && !g.debug_skip_mma) {
        tc::fence_after_sync();
        const int k0 = kbeg + s * kKT, klen = min(kKT, kend - k0), kpad = (klen + 15) & ~15;
        const uint32_t a0 = tc::smem_u32(smem + (s & 1) * sbytes), b0 = a0 + kStageA;
        const uint32_t lbo_a = kBM * 16, lbo_b = BN * 16;
        for (int kk = 0; kk < kpad / 16; ++kk) {
          const uint64_t ad = tc::smem_desc(a0 + kk * 2 * lbo_a, lbo_a, 128);
          const uint64_t bd = tc::smem_desc(b0 + kk * 2 * lbo_b, lbo_b, 128);
          tc::mma_bf16(tmem, ad, bd, idesc, (s > 0 || kk > 0) ? 1u : 0u);
        }
        tc::mma_commit(&bar[s & 1]);
      }
      last = s;
      if (s + 1 < ns) {
        if (s >= 1) {
          // the other stage was read by slab s - 1's MMAs: its commit is that barrier's
          // ((s - 1) / 2)-th completion
          const bool got = tc::mbar_wait(&bar[(s + 1) & 1], ((s - 1) >> 1) & 1u, wait_limit);
          ok = __syncthreads_and(got) != 0;  // block-uniform
          if (!ok) break;
        }
        gather(s + 1);
        tc::fence_smem_to_async();
      }
      __syncthreads();
    }
    if (ok) {
      const bool got = tc::mbar_wait(&bar[(ns - 1) & 1], ((ns - 1) >> 1) & 1u, wait_limit);
      ok = __syncthreads_and(got) != 0;
    }
    tc::fence_after_sync();
  }

  if (!ok) {
    if (tid == 0) atomicExch(g.err, 1);
    // second, bounded chance for the MMAs in flight (they complete in order: the last commit)
    if (last >= 0) tc::mbar_wait(&bar[last & 1], (last >> 1) & 1u, wait_limit);
  } else {
    // epilogue: row m = m0 + 32*warp + lane, columns n0 .. n0+BN, 32 at a time: one TMEM load of
    // 32 columns (inside the tile's allocation, which is at least BN rounded up to 32) and, for
    // the tanh gradient, the row's 32 values of H loaded before it completes
    const int m = m0 + 32 * warp + lane;
    const bool empty = ns == 0;  // a split with no K range contributes nothing
    const int64_t csn = g.ldcn ? g.ldcn : 1;
    float *Cf = g.Cf ? g.Cf + static_cast<int64_t>(blockIdx.z) * g.split_stride : nullptr;
    const bool vec_bf16 = ((g.mode == kEpiBiasTanh && !Cf) || g.mode == kEpiTanhGrad) && (g.ldcb & 7) == 0 &&
                          aligned16(g.Cb) && (g.mode != kEpiTanhGrad || ((g.ldh & 7) == 0 && aligned16(g.H)));
    for (int c0 = 0; c0 < BN; c0 += 32) {
      float v32[32];
      uint4 hv[4] = {make_uint4(0u, 0u, 0u, 0u), make_uint4(0u, 0u, 0u, 0u), make_uint4(0u, 0u, 0u, 0u),
                     make_uint4(0u, 0u, 0u, 0u)};
      if (!empty) {
        tmem_ld32(tmem + (static_cast<uint32_t>(32 * warp) << 16) + static_cast<uint32_t>(c0), v32);
        if (vec_bf16 && g.mode == kEpiTanhGrad && m < g.M) {
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (n0 + c0 + 8 * q + 8 <= g.N)
              hv[q] = *reinterpret_cast<const uint4 *>(g.H + static_cast<int64_t>(m) * g.ldh + n0 + c0 + 8 * q);
        }
        tc::tmem_ld_wait();
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) v32[j] = 0.0f;
        if (g.mode != kEpiStoreF32 || g.split_stride == 0) break;  // only a split slice must be written
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int cq = c0 + 8 * q;
        if (cq >= BN) break;
        const float *v = v32 + 8 * q;
        // BF16 outputs of 8 whole columns: one 16-byte store per row (and one 16-byte load of H)
        const int nb = n0 + cq;
        if (m < g.M && vec_bf16 && nb + 8 <= g.N) {
          float o[8];
          if (g.mode == kEpiBiasTanh) {
#pragma unroll
            for (int j = 0; j < 8; ++j) o[j] = tc::tanh_approx(g.alpha * v[j] + g.bias[nb + j]);
          } else {
            const __nv_bfloat16 *h = reinterpret_cast<const __nv_bfloat16 *>(&hv[q]);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const float hj = __bfloat162float(h[j]);
              o[j] = g.alpha * v[j] * (1.0f - hj * hj);
            }
          }
          __nv_bfloat16 ob[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) ob[j] = __float2bfloat16(o[j]);
          *reinterpret_cast<uint4 *>(g.Cb + static_cast<int64_t>(m) * g.ldcb + nb) = *reinterpret_cast<const uint4 *>(ob);
          if (g.Ct) {  // the warp's 32 rows of one column are 64 contiguous bytes
#pragma unroll
            for (int j = 0; j < 8; ++j) g.Ct[static_cast<int64_t>(nb + j) * g.ldct + m] = ob[j];
          }
        } else if (m < g.M && g.mode == kEpiStoreF32 && csn == 1 && nb + 8 <= g.N && (g.ldc & 3) == 0 &&
                   aligned16(Cf)) {
          // FP32 outputs of 8 whole contiguous columns: two 16-byte stores per row
          float4 *dst = reinterpret_cast<float4 *>(Cf + static_cast<int64_t>(m) * g.ldc + nb);
          dst[0] = make_float4(g.alpha * v[0], g.alpha * v[1], g.alpha * v[2], g.alpha * v[3]);
          dst[1] = make_float4(g.alpha * v[4], g.alpha * v[5], g.alpha * v[6], g.alpha * v[7]);
        } else if (m < g.M) {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int n = nb + j;
            if (n >= g.N || cq + j >= BN) continue;
            float a = g.alpha * v[j];
            switch (g.mode) {
              case kEpiStoreF32:
                Cf[static_cast<int64_t>(m) * g.ldc + n * csn] = a;
                break;
              case kEpiAddF32:
                Cf[static_cast<int64_t>(m) * g.ldc + n * csn] += a;
                break;
              case kEpiAtomicF32:
                atomicAdd(&Cf[static_cast<int64_t>(m) * g.ldc + n * csn], a);
                break;
              case kEpiBiasTanh: {
                const float h = tc::tanh_approx(a + g.bias[n]);
                g.Cb[static_cast<int64_t>(m) * g.ldcb + n] = __float2bfloat16(h);
                if (g.Ct) g.Ct[static_cast<int64_t>(n) * g.ldct + m] = __float2bfloat16(h);
                if (Cf) Cf[static_cast<int64_t>(m) * g.ldc + n * csn] = h;
                break;
              }
              case kEpiBiasF32:
                Cf[static_cast<int64_t>(m) * g.ldc + n * csn] = a + g.bias[n];
                break;
              case kEpiTanhGrad: {
                const float h = __bfloat162float(g.H[static_cast<int64_t>(m) * g.ldh + n]);
                g.Cb[static_cast<int64_t>(m) * g.ldcb + n] = __float2bfloat16(a * (1.0f - h * h));
                if (g.Ct) g.Ct[static_cast<int64_t>(n) * g.ldct + m] = __float2bfloat16(a * (1.0f - h * h));
                break;
              }
              default:
                break;
            }
          }
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, ncols);
}

size_t gemm_smem_bytes() { return kGemmSmemBytes; }

// gather kind of an operand X(r, k) = X[r*srow + k*sk] (the device conditions of gather_tile)
static int gather_kind(const void *X, int64_t srow, int64_t sk) {
  const bool a16 = (reinterpret_cast<uintptr_t>(X) & 15u) == 0;
  if (sk == 1 && (srow & 7) == 0 && a16) return kGatherK;
  if (srow == 1 && (sk & 7) == 0 && a16) return kGatherRows;
  return kGatherAny;
}

cudaError_t launch_gemm_bf16(const GemmArgs &g, cudaStream_t s) {
  using Kern = void (*)(const GemmArgs);
  static const Kern kernels[5] = {k_gemm_bf16<kGatherK, kGatherK>, k_gemm_bf16<kGatherK, kGatherRows>,
                                  k_gemm_bf16<kGatherRows, kGatherK>, k_gemm_bf16<kGatherRows, kGatherRows>,
                                  k_gemm_bf16<kGatherAny, kGatherAny>};
  static bool attr_set = false;
  if (!attr_set) {
    for (Kern k : kernels) {
      const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 static_cast<int>(kGemmSmemBytes));
      if (e != cudaSuccess) return e;
    }
    attr_set = true;
  }
  if (g.BN < 16 || g.BN > 256 || (g.BN & 15) != 0) return cudaErrorInvalidValue;
  const int nsplit = g.ksplit > 1 ? g.ksplit : 1;
  if (nsplit > 1 && g.mode != kEpiAtomicF32 && !(g.mode == kEpiStoreF32 && g.split_stride > 0))
    return cudaErrorInvalidValue;
  const int ga = gather_kind(g.A, g.sam, g.sak), gb = gather_kind(g.B, g.sbn, g.sbk);
  const Kern k = (ga == kGatherAny || gb == kGatherAny) ? kernels[4] : kernels[2 * ga + gb];
  const dim3 grid((g.M + kBM - 1) / kBM, (g.N + g.BN - 1) / g.BN, nsplit);
  k<<<grid, kThreads, 2 * stage_bytes(g.BN), s>>>(g);
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
