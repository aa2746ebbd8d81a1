// Host interface of the tcgen05 BF16 GEMM (tc_gemm.cu).
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace mppi {

enum GemmEpilogue {
  kEpiStoreF32 = 0,   // Cf = alpha * acc
  kEpiAddF32 = 1,     // Cf += alpha * acc
  kEpiBiasTanh = 2,   // Cb = bf16(tanh(alpha * acc + bias)); Cf (optional) = the same in FP32
  kEpiBiasF32 = 3,    // Cf = alpha * acc + bias
  kEpiTanhGrad = 4,   // Cb = bf16(alpha * acc * (1 - H^2))  (backward through tanh)
  kEpiAtomicF32 = 5,  // Cf += alpha * acc with atomicAdd (split-K partial sums)
};

struct GemmArgs {
  int M, N, K, BN;              // BN: output tile width (multiple of 16, <= 256)
  const __nv_bfloat16 *A;
  int64_t sam, sak;
  const __nv_bfloat16 *B;
  int64_t sbk, sbn;
  int mode;
  float alpha;
  float *Cf;
  int64_t ldc;                  // Cf(m, n) = Cf[m*ldc + n*ldcn]
  int64_t ldcn;                 // column stride of Cf (1 = row-major; 0 is read as 1)
  __nv_bfloat16 *Cb;
  int64_t ldcb;
  __nv_bfloat16 *Ct;            // optional transposed copy of the BF16 output: Ct[n*ldct + m]
  int64_t ldct;                 // (the batch-contiguous operand of a later weight-gradient GEMM)
  const float *bias;
  const __nv_bfloat16 *H;
  int64_t ldh;
  int *err;                     // set to 1 if a bounded wait ran out
  int ksplit;                   // K range split over gridDim.z CTAs (kEpiAtomicF32, or kEpiStoreF32 with
                                // split_stride > 0); 0/1 = no split
  int64_t split_stride;         // kEpiStoreF32 with splits: split z writes its partial to Cf + z * split_stride
  uint32_t wait_limit;          // mbarrier polls before a wait gives up (0: tc::kWaitLimit)
  int debug_skip_mma;           // check hook only: issue no MMA (so the waits run out, nothing in flight)
};

// Largest dynamic shared memory of a GEMM CTA: two stages of the widest (BN = 256) tile.  A
// launch requests two stages of its own tile width.
constexpr size_t kGemmSmemBytes = 96 * 1024;

cudaError_t launch_gemm_bf16(const GemmArgs &g, cudaStream_t s);

}  // namespace mppi
