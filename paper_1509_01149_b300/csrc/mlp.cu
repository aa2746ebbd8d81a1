// Training and one-step prediction of the learned car-dynamics surrogate on sm_103a.
//
// Data: for given (state, control) pairs, the analytic car step (systems.cuh) produces
// the next state on the GPU; the features are stored in BF16, the state increments in
// FP32, and out_scale = per-state standard deviation of the increments.
// Training step (batch B, all on one stream):
//   gather  (Philox-random rows) -> Xb [B][16] bf16, Tb [B][16] = increments / out_scale
//   forward H1 = tanh(Xb W1^T + b1), H2 = tanh(H1 W2^T + b2), Y = H2 W3^T + b3   (tcgen05 GEMMs)
//   loss    L = (1/B) sum_b sum_{i<7} (Y - Tb)^2, dY = 2 (Y - Tb) / B
//   backward gW3 = dY^T H2, dZ2 = (dY W3) * (1 - H2^2), gW2 = dZ2^T H1,
//            dZ1 = (dZ2 W2) * (1 - H1^2), gW1 = dZ1^T Xb  (weight gradients split over
//            the batch across CTAs, each split's partial stored to its own slice and the
//            slices summed in a fixed order, so training is bit-reproducible; their operands
//            are transposed copies [features][B] written by the producing GEMM epilogues, so
//            the batch, their K dimension, is contiguous), bias gradients = column sums
//   Adam    on FP32 master weights, BF16 copies (and W2, W3 transposed for the backward
//            data products) refreshed for the next step.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "nvtx_range.h"
#include "../../include/mppi.h"
#include "mlp_model.cuh"
#include "systems.cuh"
#include "tc_gemm.cuh"

namespace mppi {
namespace mlp {

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
// analytic transitions: features (bf16) and increments (f32) of x' = step(x, u)
__global__ void k_datagen(const float *__restrict__ xs, const float *__restrict__ us, int n, float dt,
                          __nv_bfloat16 *__restrict__ Xf, float *__restrict__ D) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float x[kState], u[kCtl], z[kIn];
#pragma unroll
  for (int j = 0; j < kState; ++j) x[j] = xs[static_cast<size_t>(i) * kState + j];
  u[0] = us[static_cast<size_t>(i) * kCtl];
  u[1] = us[static_cast<size_t>(i) * kCtl + 1];
  features(x, u, z);
#pragma unroll
  for (int j = 0; j < kIn; ++j) Xf[static_cast<size_t>(i) * kIn + j] = __float2bfloat16(z[j]);
  float y[kState];
#pragma unroll
  for (int j = 0; j < kState; ++j) y[j] = x[j];
  Car::Aux aux;
  Env env{};
  Car::init(y, aux, env);
  Car::step(y, u, aux, env, dt);
#pragma unroll
  for (int j = 0; j < kState; ++j) D[static_cast<size_t>(i) * kState + j] = y[j] - x[j];
}

// per-state sums of increments and their squares (FP64)
__global__ void k_moments(const float *__restrict__ D, int n, double *__restrict__ acc /*[gridDim.x][14]*/) {
  __shared__ double s[2 * kState][8];
  double a[2 * kState] = {0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
#pragma unroll
    for (int j = 0; j < kState; ++j) {
      const double d = D[static_cast<size_t>(i) * kState + j];
      a[j] += d;
      a[kState + j] += d * d;
    }
#pragma unroll
  for (int j = 0; j < 2 * kState; ++j) {
    double v = a[j];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s[j][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < 2 * kState) {
    double v = 0.0;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) v += s[threadIdx.x][w];
    acc[static_cast<size_t>(blockIdx.x) * 2 * kState + threadIdx.x] = v;  // this block's partial
  }
}

// random batch rows (Philox counter (b, step, 0x4d4c5000, 0) under the training seed)
__global__ void k_gather(const __nv_bfloat16 *__restrict__ Xf, const float *__restrict__ D, int n,
                         const float *__restrict__ out_scale, int B, uint32_t key_lo, uint32_t key_hi, uint32_t step,
                         __nv_bfloat16 *__restrict__ Xb, float *__restrict__ Tb) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const Words4 w = philox4x32_10(static_cast<uint32_t>(b), step, 0x4d4c5000u, 0u, key_lo, key_hi);
  const uint64_t r = (static_cast<uint64_t>(w.x) << 32) | w.y;
  const size_t i = static_cast<size_t>(r % static_cast<uint64_t>(n));
  static_assert(kIn == 16 && kOut == 16, "one 32-byte feature row, one 64-byte target row");
  const uint4 *xs = reinterpret_cast<const uint4 *>(Xf + i * kIn);
  uint4 *xd = reinterpret_cast<uint4 *>(Xb + static_cast<size_t>(b) * kIn);
  const uint4 x0 = xs[0], x1 = xs[1];
  float t[kOut];
#pragma unroll
  for (int j = 0; j < kOut; ++j) t[j] = j < kState ? D[i * kState + j] / out_scale[j] : 0.0f;
  xd[0] = x0;
  xd[1] = x1;
  float4 *td = reinterpret_cast<float4 *>(Tb + static_cast<size_t>(b) * kOut);
#pragma unroll
  for (int j = 0; j < kOut / 4; ++j) td[j] = make_float4(t[4 * j], t[4 * j + 1], t[4 * j + 2], t[4 * j + 3]);
}

// dY = 2 (Y - T) / B on the first 7 outputs, one thread per batch row (dYf and dYb row-major,
// dYt [16][B] transposed for the weight-gradient GEMM); the loss is summed in FP32 over each
// row and warp and added across warps in FP64
__global__ void k_loss_grad(const float *__restrict__ Y, const float *__restrict__ T, int B, float *__restrict__ dYf,
                            __nv_bfloat16 *__restrict__ dYb, __nv_bfloat16 *__restrict__ dYt,
                            double *__restrict__ loss) {
  static_assert(kOut == 16, "one 64-byte output row");
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.0f;
  if (b < B) {
    const float4 *y4 = reinterpret_cast<const float4 *>(Y + static_cast<size_t>(b) * kOut);
    const float4 *t4 = reinterpret_cast<const float4 *>(T + static_cast<size_t>(b) * kOut);
    float g[kOut];
#pragma unroll
    for (int q = 0; q < kOut / 4; ++q) {
      const float4 y = y4[q], t = t4[q];
      const float r[4] = {y.x - t.x, y.y - t.y, y.z - t.z, y.w - t.w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int jj = 4 * q + e;
        g[jj] = jj < kState ? 2.0f * r[e] / static_cast<float>(B) : 0.0f;
        if (jj < kState) l = fmaf(r[e], r[e], l);
      }
    }
    float4 *gf = reinterpret_cast<float4 *>(dYf + static_cast<size_t>(b) * kOut);
#pragma unroll
    for (int q = 0; q < kOut / 4; ++q) gf[q] = make_float4(g[4 * q], g[4 * q + 1], g[4 * q + 2], g[4 * q + 3]);
    __nv_bfloat16 gb[kOut];
#pragma unroll
    for (int jj = 0; jj < kOut; ++jj) gb[jj] = __float2bfloat16(g[jj]);
    uint4 *db = reinterpret_cast<uint4 *>(dYb + static_cast<size_t>(b) * kOut);
    db[0] = *reinterpret_cast<const uint4 *>(gb);
    db[1] = *reinterpret_cast<const uint4 *>(gb + 8);
#pragma unroll
    for (int jj = 0; jj < kOut; ++jj) dYt[static_cast<size_t>(jj) * B + b] = gb[jj];
  }
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if ((threadIdx.x & 31) == 0 && l != 0.0f) atomicAdd(loss, static_cast<double>(l) / B);
}

// Xt [16][B] = X [B][16] transposed (the batch-contiguous input of the first weight gradient)
__global__ void k_transpose16(const __nv_bfloat16 *__restrict__ X, int B, __nv_bfloat16 *__restrict__ Xt) {
  static_assert(kIn == 16, "one 32-byte feature row");
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const uint4 *xs = reinterpret_cast<const uint4 *>(X + static_cast<size_t>(b) * kIn);
  uint4 v[2] = {xs[0], xs[1]};
  const __nv_bfloat16 *e = reinterpret_cast<const __nv_bfloat16 *>(v);
#pragma unroll
  for (int jj = 0; jj < kIn; ++jj) Xt[static_cast<size_t>(jj) * B + b] = e[jj];
}

// column sums of a [rows][cols] matrix (f32 or bf16) into out[cols]: block (x, y) sums the rows
// r = y, y + 8 gridDim.y, ... of its 32 columns into part[y][cols]; the last block of each column
// group to finish (a ticket, reset for the next launch) adds the gridDim.y partials in a fixed
// order (eight warps over eight partials each, then the warps in order), so the result does not
// depend on which block finishes last
template <class T>
__global__ void k_colsum(const T *__restrict__ A, int rows, int cols, float *__restrict__ part,
                         float *__restrict__ out, unsigned int *__restrict__ tickets) {
  __shared__ float s[8][33];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, c = blockIdx.x * 32 + lane, ty = threadIdx.x >> 5;
  const int stride = 8 * gridDim.y;
  float a = 0.0f;
  if (c < cols) {
    // rows r = ty + 8 y, r + stride, ... added in that order, eight loads in flight at a time
    int r = ty + blockIdx.y * 8;
    for (; r + 7 * stride < rows; r += 8 * stride) {
      float v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = static_cast<float>(A[static_cast<size_t>(r + u * stride) * cols + c]);
#pragma unroll
      for (int u = 0; u < 8; ++u) a += v[u];
    }
    for (; r < rows; r += stride) a += static_cast<float>(A[static_cast<size_t>(r) * cols + c]);
  }
  s[ty][lane] = a;
  __syncthreads();
  if (ty == 0 && c < cols) {
    float t = 0.0f;
    for (int q = 0; q < 8; ++q) t += s[q][lane];
    part[static_cast<size_t>(blockIdx.y) * cols + c] = t;  // this block's partial
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(&tickets[blockIdx.x], 1u) == gridDim.y - 1;
  __syncthreads();
  if (!last) return;
  const int per = (gridDim.y + 7) / 8;  // partials per warp
  float w = 0.0f;
  if (c < cols) {
    for (int z = ty * per; z < min(static_cast<int>(gridDim.y), (ty + 1) * per); ++z)
      w += __ldcg(part + static_cast<size_t>(z) * cols + c);
  }
  s[ty][lane] = w;
  __syncthreads();
  if (ty == 0 && c < cols) {
    float t = 0.0f;
    for (int q = 0; q < 8; ++q) t += s[q][lane];
    out[c] = t;
  }
  if (threadIdx.x == 0) tickets[blockIdx.x] = 0u;
}

// out[i] = sum over z = 0 .. nsplit-1 (in that order) of part[z][i]: the fixed-order reduction of
// split-K partial products and of column-sum partials, so that training is bit-reproducible
__global__ void k_sum_splits(const float *__restrict__ part, int nsplit, size_t count, float *__restrict__ out) {
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < count;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    float a = 0.0f;
    int z = 0;
    for (; z + 8 <= nsplit; z += 8) {  // eight loads in flight, added in z order
      float v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = part[static_cast<size_t>(z + u) * count + i];
#pragma unroll
      for (int u = 0; u < 8; ++u) a += v[u];
    }
    for (; z < nsplit; ++z) a += part[static_cast<size_t>(z) * count + i];
    out[i] = a;
  }
}

// Adam step fused with the BF16 weight copies of the next step's GEMMs (the same conversions
// as refresh_bf16: W1, W2, W3 as stored and W2, W3 transposed)
__global__ void k_adam_bf16(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, size_t n, float lr, float b1, float b2, float c1, float c2, float eps,
                            __nv_bfloat16 *__restrict__ w1, __nv_bfloat16 *__restrict__ w2,
                            __nv_bfloat16 *__restrict__ w3, __nv_bfloat16 *__restrict__ w2t,
                            __nv_bfloat16 *__restrict__ w3t) {
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    const __nv_bfloat16 h = __float2bfloat16(pi);
    if (i < kOffB1) {
      w1[i - kOffW1] = h;
    } else if (i >= kOffW2 && i < kOffB2) {
      const size_t e = i - kOffW2, r = e / kHid, c = e % kHid;
      w2[e] = h;
      w2t[c * kHid + r] = h;
    } else if (i >= kOffW3 && i < kOffB3) {
      const size_t e = i - kOffW3, r = e / kHid, c = e % kHid;
      w3[e] = h;
      w3t[c * kOut + r] = h;
    }
  }
}

// dst [cols][rows] = src [rows][cols] transposed, in BF16 (the weights as the backward data
// GEMMs read them: their K dimension contiguous)
__global__ void k_to_bf16_t(const float *__restrict__ src, __nv_bfloat16 *__restrict__ dst, int rows, int cols) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows * cols; i += gridDim.x * blockDim.x) {
    const int r = i / cols, c = i - r * cols;
    dst[static_cast<size_t>(c) * rows + r] = __float2bfloat16(src[i]);
  }
}

__global__ void k_to_bf16(const float *__restrict__ src, __nv_bfloat16 *__restrict__ dst, size_t n) {
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * blockDim.x)
    dst[i] = __float2bfloat16(src[i]);
}

// uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases, zero padded rows/columns
__global__ void k_init(float *__restrict__ p, uint32_t key_lo, uint32_t key_hi) {
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < kNumParams;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const Words4 w = philox4x32_10(static_cast<uint32_t>(i), 0u, 0x494e4954u, 0u, key_lo, key_hi);
    const float u = 2.0f * unit_uniform(w.x) - 1.0f;
    float v = 0.0f;
    if (i < kOffB1) {
      const int col = static_cast<int>((i - kOffW1) % kIn);
      v = col < kState + kCtl ? u / 3.0f : 0.0f;           // fan_in 9
    } else if (i >= kOffW2 && i < kOffB2) {
      v = u / 16.0f;                                      // fan_in 256
    } else if (i >= kOffW3 && i < kOffB3) {
      const int row = static_cast<int>((i - kOffW3) / kHid);
      v = row < kState ? u / 16.0f : 0.0f;
    }
    p[i] = v;
  }
}

// x' = x + y[0:7] * out_scale from the FP32 network output Y [n][16]
__global__ void k_apply(const float *__restrict__ xs, const float *__restrict__ Y, const float *__restrict__ out_scale,
                        int n, float *__restrict__ xn) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * kState) return;
  const int i = idx / kState, j = idx % kState;
  xn[idx] = xs[idx] + Y[static_cast<size_t>(i) * kOut + j] * out_scale[j];
}

// the analytic car step (the learned model's fallback and the yardstick of its error)
__global__ void k_analytic_step(const float *__restrict__ xs, const float *__restrict__ us, int n, float dt,
                                float *__restrict__ xn) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float y[kState], u[kCtl];
#pragma unroll
  for (int j = 0; j < kState; ++j) y[j] = xs[static_cast<size_t>(i) * kState + j];
  u[0] = us[static_cast<size_t>(i) * kCtl];
  u[1] = us[static_cast<size_t>(i) * kCtl + 1];
  Car::Aux aux;
  Env env{};
  Car::init(y, aux, env);
  Car::step(y, u, aux, env, dt);
#pragma unroll
  for (int j = 0; j < kState; ++j) xn[static_cast<size_t>(i) * kState + j] = y[j];
}

__global__ void k_features(const float *__restrict__ xs, const float *__restrict__ us, int n,
                           __nv_bfloat16 *__restrict__ Xf) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float x[kState], u[kCtl], z[kIn];
#pragma unroll
  for (int j = 0; j < kState; ++j) x[j] = xs[static_cast<size_t>(i) * kState + j];
  u[0] = us[static_cast<size_t>(i) * kCtl];
  u[1] = us[static_cast<size_t>(i) * kCtl + 1];
  features(x, u, z);
#pragma unroll
  for (int j = 0; j < kIn; ++j) Xf[static_cast<size_t>(i) * kIn + j] = __float2bfloat16(z[j]);
}

}  // namespace mlp
}  // namespace mppi

using namespace mppi;
using namespace mppi::mlp;

namespace {
constexpr int kMaxSplit = 64;       // split-K partials of a weight-gradient GEMM
constexpr int kMomentBlocks = 512;  // blocks of the data-set moment kernel
}  // namespace

struct mppi_mlp {
  std::string err;
  cudaStream_t stream = nullptr;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;  // FP32 master, grads, Adam moments
  __nv_bfloat16 *w1 = nullptr, *w2 = nullptr, *w3 = nullptr;      // BF16 copies for the GEMMs
  __nv_bfloat16 *w2t = nullptr, *w3t = nullptr;                   // and W2, W3 transposed (backward)
  float *out_scale = nullptr;                                    // [16] (first 7 used)
  float h_out_scale[kOut] = {0};
  int adam_t = 0;
  // data
  __nv_bfloat16 *Xf = nullptr;
  float *D = nullptr;
  int n_data = 0;
  // batch workspace
  int cap = 0;
  __nv_bfloat16 *Xb = nullptr, *H1 = nullptr, *H2 = nullptr, *dYb = nullptr, *dZ2 = nullptr, *dZ1 = nullptr;
  // the same activations and errors transposed ([features][B]): the batch is the K dimension of
  // the weight-gradient GEMMs, which then read it contiguously
  __nv_bfloat16 *Xt = nullptr, *H1t = nullptr, *H2t = nullptr, *dYt = nullptr, *dZ2t = nullptr, *dZ1t = nullptr;
  float *Tb = nullptr, *Y = nullptr, *dYf = nullptr;
  double *loss = nullptr;
  int *d_err = nullptr;
  float *gsplit = nullptr;    // split-K and column-sum partials [splits][count]
  unsigned int *tickets = nullptr;  // column-sum completion tickets [kHid / 32], zero between launches
  double *moments = nullptr;  // per-block moment partials [kMomentBlocks][2 * kState]

  int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    err = buf;
    return code;
  }
  int cuda(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return MPPI_OK;
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? MPPI_ENOMEM : MPPI_ECUDA, "%s: %s", what, cudaGetErrorString(e));
  }
};

#define MLP_TRY(expr)               \
  do {                              \
    const int _rc = (expr);         \
    if (_rc != MPPI_OK) return _rc; \
  } while (0)

namespace {

int ensure_batch(mppi_mlp *q, int B) {
  if (B <= q->cap) return MPPI_OK;
  for (__nv_bfloat16 *t : {q->Xt, q->H1t, q->H2t, q->dYt, q->dZ2t, q->dZ1t}) cudaFree(t);
  q->Xt = q->H1t = q->H2t = q->dYt = q->dZ2t = q->dZ1t = nullptr;
  cudaFree(q->Xb);
  cudaFree(q->H1);
  cudaFree(q->H2);
  cudaFree(q->dYb);
  cudaFree(q->dZ2);
  cudaFree(q->dZ1);
  cudaFree(q->Tb);
  cudaFree(q->Y);
  cudaFree(q->dYf);
  q->cap = 0;
  const size_t b = static_cast<size_t>(B);
  MLP_TRY(q->cuda(cudaMalloc(&q->Xb, b * kIn * 2), "batch"));
  MLP_TRY(q->cuda(cudaMalloc(&q->H1, b * kHid * 2), "batch"));
  MLP_TRY(q->cuda(cudaMalloc(&q->H2, b * kHid * 2), "batch"));
  MLP_TRY(q->cuda(cudaMalloc(&q->dYb, b * kOut * 2), "batch"));
  MLP_TRY(q->cuda(cudaMalloc(&q->dZ2, b * kHid * 2), "batch"));
  MLP_TRY(q->cuda(cudaMalloc(&q->dZ1, b * kHid * 2), "batch"));
  MLP_TRY(q->cuda(cudaMalloc(&q->Tb, b * kOut * 4), "batch"));
  MLP_TRY(q->cuda(cudaMalloc(&q->Y, b * kOut * 4), "batch"));
  MLP_TRY(q->cuda(cudaMalloc(&q->dYf, b * kOut * 4), "batch"));
  MLP_TRY(q->cuda(cudaMalloc(&q->Xt, b * kIn * 2), "batch"));
  MLP_TRY(q->cuda(cudaMalloc(&q->H1t, b * kHid * 2), "batch"));
  MLP_TRY(q->cuda(cudaMalloc(&q->H2t, b * kHid * 2), "batch"));
  MLP_TRY(q->cuda(cudaMalloc(&q->dYt, b * kOut * 2), "batch"));
  MLP_TRY(q->cuda(cudaMalloc(&q->dZ2t, b * kHid * 2), "batch"));
  MLP_TRY(q->cuda(cudaMalloc(&q->dZ1t, b * kHid * 2), "batch"));
  q->cap = B;
  return MPPI_OK;
}

GemmArgs gemm(int M, int N, int K, int BN, const __nv_bfloat16 *A, int64_t sam, int64_t sak, const __nv_bfloat16 *B,
              int64_t sbk, int64_t sbn, int mode, int *err) {
  GemmArgs g{};
  g.M = M;
  g.N = N;
  g.K = K;
  g.BN = BN;
  g.A = A;
  g.sam = sam;
  g.sak = sak;
  g.B = B;
  g.sbk = sbk;
  g.sbn = sbn;
  g.mode = mode;
  g.alpha = 1.0f;
  g.err = err;
  g.ldcn = 1;
  return g;
}

int refresh_bf16(mppi_mlp *q) {
  k_to_bf16<<<64, 256, 0, q->stream>>>(q->p + kOffW1, q->w1, static_cast<size_t>(kHid) * kIn);
  k_to_bf16<<<256, 256, 0, q->stream>>>(q->p + kOffW2, q->w2, static_cast<size_t>(kHid) * kHid);
  k_to_bf16<<<64, 256, 0, q->stream>>>(q->p + kOffW3, q->w3, static_cast<size_t>(kOut) * kHid);
  k_to_bf16_t<<<256, 256, 0, q->stream>>>(q->p + kOffW2, q->w2t, kHid, kHid);
  k_to_bf16_t<<<16, 256, 0, q->stream>>>(q->p + kOffW3, q->w3t, kOut, kHid);
  return q->cuda(cudaGetLastError(), "bf16 copy");
}

// forward on Xb [B][16] into H1, H2 (bf16) and Y (f32); with `transposed` (training) also
// H1t, H2t for the weight gradients
int forward(mppi_mlp *q, const __nv_bfloat16 *X, int B, bool transposed) {
  GemmArgs g = gemm(B, kHid, kIn, 64, X, kIn, 1, q->w1, 1, kIn, kEpiBiasTanh, q->d_err);
  g.bias = q->p + kOffB1;
  g.Cb = q->H1;
  g.ldcb = kHid;
  g.Ct = transposed ? q->H1t : nullptr;
  g.ldct = B;
  MLP_TRY(q->cuda(launch_gemm_bf16(g, q->stream), "gemm h1"));
  g = gemm(B, kHid, kHid, 64, q->H1, kHid, 1, q->w2, 1, kHid, kEpiBiasTanh, q->d_err);
  g.bias = q->p + kOffB2;
  g.Cb = q->H2;
  g.ldcb = kHid;
  g.Ct = transposed ? q->H2t : nullptr;
  g.ldct = B;
  MLP_TRY(q->cuda(launch_gemm_bf16(g, q->stream), "gemm h2"));
  g = gemm(B, kOut, kHid, 16, q->H2, kHid, 1, q->w3, 1, kHid, kEpiBiasF32, q->d_err);
  g.bias = q->p + kOffB3;
  g.Cf = q->Y;
  g.ldc = kOut;
  return q->cuda(launch_gemm_bf16(g, q->stream), "gemm y");
}

// loss + gradients of the batch (Xb, Tb) into q->g and q->loss
int backward(mppi_mlp *q, const __nv_bfloat16 *X, const float *T, int B) {
  MLP_TRY(q->cuda(cudaMemsetAsync(q->loss, 0, sizeof(double), q->stream), "loss zero"));
  const int nthr = 256;
  mlp::k_loss_grad<<<(B + nthr - 1) / nthr, nthr, 0, q->stream>>>(q->Y, T, B, q->dYf, q->dYb, q->dYt, q->loss);
  mlp::k_transpose16<<<(B + nthr - 1) / nthr, nthr, 0, q->stream>>>(X, B, q->Xt);
  MLP_TRY(q->cuda(cudaGetLastError(), "loss"));
  // Weight gradients are sums over the batch: split-K GEMMs, each split storing its partial
  // product to its own slice of gsplit, then a fixed-order sum of the slices (no atomics: the
  // same data and seed give the same bits)
  const int split = std::max(1, std::min(kMaxSplit, B / 256));
  auto split_sum = [&](size_t count, float *out, const char *what) {
    mlp::k_sum_splits<<<static_cast<int>(std::min<size_t>(1024, (count + 255) / 256)), 256, 0, q->stream>>>(
        q->gsplit, split, count, out);
    return q->cuda(cudaGetLastError(), what);
  };
  // gW3 (stored [16][256]): C(m = hidden j, n = output i) = sum_b H2[b][j] dY[b][i]
  GemmArgs g = gemm(kHid, kOut, B, 16, q->H2t, B, 1, q->dYt, 1, B, kEpiStoreF32, q->d_err);
  g.Cf = q->gsplit;
  g.ldc = 1;
  g.ldcn = kHid;
  g.ksplit = split;
  g.split_stride = static_cast<int64_t>(kOut) * kHid;
  MLP_TRY(q->cuda(launch_gemm_bf16(g, q->stream), "gemm gW3"));
  MLP_TRY(split_sum(static_cast<size_t>(kOut) * kHid, q->g + kOffW3, "gW3 sum"));
  // dZ2 = (dY W3) * (1 - H2^2)
  g = gemm(B, kHid, kOut, 64, q->dYb, kOut, 1, q->w3t, 1, kOut, kEpiTanhGrad, q->d_err);
  g.H = q->H2;
  g.ldh = kHid;
  g.Cb = q->dZ2;
  g.ldcb = kHid;
  g.Ct = q->dZ2t;
  g.ldct = B;
  MLP_TRY(q->cuda(launch_gemm_bf16(g, q->stream), "gemm dZ2"));
  // gW2 [256][256] = dZ2^T H1
  g = gemm(kHid, kHid, B, 128, q->dZ2t, B, 1, q->H1t, 1, B, kEpiStoreF32, q->d_err);
  g.Cf = q->gsplit;
  g.ldc = kHid;
  g.ksplit = split;
  g.split_stride = static_cast<int64_t>(kHid) * kHid;
  MLP_TRY(q->cuda(launch_gemm_bf16(g, q->stream), "gemm gW2"));
  MLP_TRY(split_sum(static_cast<size_t>(kHid) * kHid, q->g + kOffW2, "gW2 sum"));
  // dZ1 = (dZ2 W2) * (1 - H1^2)
  g = gemm(B, kHid, kHid, 64, q->dZ2, kHid, 1, q->w2t, 1, kHid, kEpiTanhGrad, q->d_err);
  g.H = q->H1;
  g.ldh = kHid;
  g.Cb = q->dZ1;
  g.ldcb = kHid;
  g.Ct = q->dZ1t;
  g.ldct = B;
  MLP_TRY(q->cuda(launch_gemm_bf16(g, q->stream), "gemm dZ1"));
  // gW1 [256][16] = dZ1^T X
  g = gemm(kHid, kIn, B, 16, q->dZ1t, B, 1, q->Xt, 1, B, kEpiStoreF32, q->d_err);
  g.Cf = q->gsplit;
  g.ldc = kIn;
  g.ksplit = split;
  g.split_stride = static_cast<int64_t>(kHid) * kIn;
  MLP_TRY(q->cuda(launch_gemm_bf16(g, q->stream), "gemm gW1"));
  MLP_TRY(split_sum(static_cast<size_t>(kHid) * kIn, q->g + kOffW1, "gW1 sum"));
  // bias gradients: column sums, 64 row partials each, summed in a fixed order by the last block
  constexpr int kRowParts = 64;
  mlp::k_colsum<float><<<dim3(1, kRowParts), 256, 0, q->stream>>>(q->dYf, B, kOut, q->gsplit, q->g + kOffB3,
                                                                    q->tickets);
  mlp::k_colsum<__nv_bfloat16><<<dim3(kHid / 32, kRowParts), 256, 0, q->stream>>>(q->dZ2, B, kHid, q->gsplit,
                                                                                  q->g + kOffB2, q->tickets);
  mlp::k_colsum<__nv_bfloat16><<<dim3(kHid / 32, kRowParts), 256, 0, q->stream>>>(q->dZ1, B, kHid, q->gsplit,
                                                                                  q->g + kOffB1, q->tickets);
  return q->cuda(cudaGetLastError(), "bias grads");
}

int check_err(mppi_mlp *q) {
  int e = 0;
  MLP_TRY(q->cuda(cudaMemcpyAsync(&e, q->d_err, sizeof e, cudaMemcpyDeviceToHost, q->stream), "err"));
  MLP_TRY(q->cuda(cudaStreamSynchronize(q->stream), "sync"));
  return e ? q->fail(MPPI_ETIMEOUT, "a tensor-core wait ran out") : MPPI_OK;
}

}  // namespace

extern "C" {

const char *mppi_mlp_last_error(mppi_mlp *q) { return q ? q->err.c_str() : "null mlp"; }

int mppi_mlp_create(uint64_t seed, mppi_mlp **out) {
  if (!out) return MPPI_EINVAL;
  *out = nullptr;
  mppi_mlp *q = new (std::nothrow) mppi_mlp();
  if (!q) return MPPI_ENOMEM;
  int rc = q->cuda(cudaStreamCreateWithFlags(&q->stream, cudaStreamNonBlocking), "stream");
  const size_t pb = sizeof(float) * kNumParams;
  if (rc == MPPI_OK) rc = q->cuda(cudaMalloc(&q->p, pb), "params");
  if (rc == MPPI_OK) rc = q->cuda(cudaMalloc(&q->g, pb), "grads");
  if (rc == MPPI_OK) rc = q->cuda(cudaMalloc(&q->m, pb), "adam m");
  if (rc == MPPI_OK) rc = q->cuda(cudaMalloc(&q->v, pb), "adam v");
  if (rc == MPPI_OK) rc = q->cuda(cudaMalloc(&q->w1, sizeof(__nv_bfloat16) * kHid * kIn), "w1");
  if (rc == MPPI_OK) rc = q->cuda(cudaMalloc(&q->w2, sizeof(__nv_bfloat16) * kHid * kHid), "w2");
  if (rc == MPPI_OK) rc = q->cuda(cudaMalloc(&q->w3, sizeof(__nv_bfloat16) * kOut * kHid), "w3");
  if (rc == MPPI_OK) rc = q->cuda(cudaMalloc(&q->w2t, sizeof(__nv_bfloat16) * kHid * kHid), "w2t");
  if (rc == MPPI_OK) rc = q->cuda(cudaMalloc(&q->w3t, sizeof(__nv_bfloat16) * kOut * kHid), "w3t");
  if (rc == MPPI_OK) rc = q->cuda(cudaMalloc(&q->out_scale, sizeof(float) * kOut), "scale");
  if (rc == MPPI_OK) rc = q->cuda(cudaMalloc(&q->loss, sizeof(double) * 16), "loss");
  if (rc == MPPI_OK) rc = q->cuda(cudaMalloc(&q->d_err, sizeof(int)), "err");
  if (rc == MPPI_OK)
    rc = q->cuda(cudaMalloc(&q->gsplit, sizeof(float) * static_cast<size_t>(kMaxSplit) * kHid * kHid), "split partials");
  if (rc == MPPI_OK) rc = q->cuda(cudaMalloc(&q->tickets, sizeof(unsigned int) * (kHid / 32)), "tickets");
  if (rc == MPPI_OK) rc = q->cuda(cudaMemset(q->tickets, 0, sizeof(unsigned int) * (kHid / 32)), "tickets");
  if (rc == MPPI_OK)
    rc = q->cuda(cudaMalloc(&q->moments, sizeof(double) * static_cast<size_t>(kMomentBlocks) * 2 * kState), "moments");
  if (rc == MPPI_OK) rc = q->cuda(cudaMemsetAsync(q->d_err, 0, sizeof(int), q->stream), "err zero");
  if (rc == MPPI_OK) rc = q->cuda(cudaMemsetAsync(q->m, 0, pb, q->stream), "m zero");
  if (rc == MPPI_OK) rc = q->cuda(cudaMemsetAsync(q->v, 0, pb, q->stream), "v zero");
  if (rc == MPPI_OK) {
    for (int i = 0; i < kOut; ++i) q->h_out_scale[i] = 1.0f;
    rc = q->cuda(cudaMemcpyAsync(q->out_scale, q->h_out_scale, sizeof(float) * kOut, cudaMemcpyHostToDevice, q->stream),
                 "scale");
  }
  if (rc == MPPI_OK) {
    mlp::k_init<<<128, 256, 0, q->stream>>>(q->p, static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
    rc = q->cuda(cudaGetLastError(), "init");
  }
  if (rc == MPPI_OK) rc = refresh_bf16(q);
  if (rc == MPPI_OK) rc = q->cuda(cudaStreamSynchronize(q->stream), "sync");
  if (rc != MPPI_OK) {
    mppi_mlp_destroy(q);
    return rc;
  }
  *out = q;
  return MPPI_OK;
}

int mppi_mlp_destroy(mppi_mlp *q) {
  if (!q) return MPPI_OK;
  if (q->stream) cudaStreamSynchronize(q->stream);
  void *bufs[] = {q->p, q->g, q->m, q->v, q->w1, q->w2, q->w3, q->w2t, q->w3t, q->out_scale, q->Xf, q->D, q->Xb, q->H1, q->H2,
                  q->dYb, q->dZ2, q->dZ1, q->Tb, q->Y, q->dYf, q->loss, q->d_err, q->gsplit, q->moments,
                  q->Xt, q->H1t, q->H2t, q->dYt, q->dZ2t, q->dZ1t, q->tickets};
  for (void *b : bufs)
    if (b) cudaFree(b);
  if (q->stream) cudaStreamDestroy(q->stream);
  delete q;
  return MPPI_OK;
}

int mppi_mlp_set_params(mppi_mlp *q, const float *h_params, const float *h_out_scale) {
  if (!q || !h_params) return MPPI_EINVAL;
  MLP_TRY(q->cuda(cudaMemcpyAsync(q->p, h_params, sizeof(float) * kNumParams, cudaMemcpyHostToDevice, q->stream), "p"));
  if (h_out_scale) {
    for (int i = 0; i < kState; ++i) q->h_out_scale[i] = h_out_scale[i];
    MLP_TRY(q->cuda(cudaMemcpyAsync(q->out_scale, q->h_out_scale, sizeof(float) * kOut, cudaMemcpyHostToDevice,
                                    q->stream),
                    "scale"));
  }
  MLP_TRY(refresh_bf16(q));
  q->adam_t = 0;
  MLP_TRY(q->cuda(cudaMemsetAsync(q->m, 0, sizeof(float) * kNumParams, q->stream), "m"));
  MLP_TRY(q->cuda(cudaMemsetAsync(q->v, 0, sizeof(float) * kNumParams, q->stream), "v"));
  return q->cuda(cudaStreamSynchronize(q->stream), "sync");
}

int mppi_mlp_get_params(mppi_mlp *q, float *h_params, float *h_out_scale) {
  if (!q) return MPPI_EINVAL;
  if (h_params)
    MLP_TRY(q->cuda(cudaMemcpyAsync(h_params, q->p, sizeof(float) * kNumParams, cudaMemcpyDeviceToHost, q->stream),
                    "p"));
  MLP_TRY(q->cuda(cudaStreamSynchronize(q->stream), "sync"));
  if (h_out_scale)
    for (int i = 0; i < kState; ++i) h_out_scale[i] = q->h_out_scale[i];
  return MPPI_OK;
}

int mppi_mlp_set_data(mppi_mlp *q, const float *d_states, const float *d_controls, int n, float dt) {
  if (!q || !d_states || !d_controls || n < 1 || !(dt > 0.0f)) return MPPI_EINVAL;
  MLP_TRY(q->cuda(cudaStreamSynchronize(q->stream), "sync"));
  cudaFree(q->Xf);
  cudaFree(q->D);
  q->Xf = nullptr;
  q->D = nullptr;
  q->n_data = 0;
  MLP_TRY(q->cuda(cudaMalloc(&q->Xf, sizeof(__nv_bfloat16) * kIn * static_cast<size_t>(n)), "data X"));
  MLP_TRY(q->cuda(cudaMalloc(&q->D, sizeof(float) * kState * static_cast<size_t>(n)), "data D"));
  mlp::k_datagen<<<(n + 255) / 256, 256, 0, q->stream>>>(d_states, d_controls, n, dt, q->Xf, q->D);
  MLP_TRY(q->cuda(cudaGetLastError(), "datagen"));
  mlp::k_moments<<<kMomentBlocks, 256, 0, q->stream>>>(q->D, n, q->moments);
  MLP_TRY(q->cuda(cudaGetLastError(), "moments"));
  std::vector<double> part(static_cast<size_t>(kMomentBlocks) * 2 * kState);
  MLP_TRY(q->cuda(cudaMemcpyAsync(part.data(), q->moments, sizeof(double) * part.size(), cudaMemcpyDeviceToHost,
                                  q->stream),
                  "moments copy"));
  MLP_TRY(q->cuda(cudaStreamSynchronize(q->stream), "sync"));
  double acc[2 * kState] = {0};
  for (int b = 0; b < kMomentBlocks; ++b)  // block order: the same bits every time
    for (int j = 0; j < 2 * kState; ++j) acc[j] += part[static_cast<size_t>(b) * 2 * kState + j];
  for (int j = 0; j < kState; ++j) {
    const double mean = acc[j] / n, var = acc[kState + j] / n - mean * mean;
    q->h_out_scale[j] = static_cast<float>(std::sqrt(std::fmax(var, 0.0)) + 1e-9);
  }
  for (int j = kState; j < kOut; ++j) q->h_out_scale[j] = 1.0f;
  MLP_TRY(q->cuda(cudaMemcpyAsync(q->out_scale, q->h_out_scale, sizeof(float) * kOut, cudaMemcpyHostToDevice, q->stream),
                  "scale"));
  q->n_data = n;
  return q->cuda(cudaStreamSynchronize(q->stream), "sync");
}

int mppi_mlp_train(mppi_mlp *q, int steps, int batch, float lr, uint64_t seed, float *h_loss_trace) {
  const NvtxRange range("mppi_mlp_train (forward, backward GEMMs, Adam)");
  if (!q || steps < 0 || batch < 128 || (batch % 128) || !(lr > 0.0f)) return MPPI_EINVAL;
  if (q->n_data < 1) return q->fail(MPPI_ESTATE, "no training data (mppi_mlp_set_data)");
  MLP_TRY(ensure_batch(q, batch));
  const float b1 = 0.9f, b2 = 0.999f;
  std::vector<double> losses(steps);
  for (int s = 0; s < steps; ++s) {
    mlp::k_gather<<<(batch + 255) / 256, 256, 0, q->stream>>>(q->Xf, q->D, q->n_data, q->out_scale, batch,
                                                             static_cast<uint32_t>(seed),
                                                             static_cast<uint32_t>(seed >> 32), static_cast<uint32_t>(s),
                                                             q->Xb, q->Tb);
    MLP_TRY(q->cuda(cudaGetLastError(), "gather"));
    MLP_TRY(forward(q, q->Xb, batch, true));
    MLP_TRY(backward(q, q->Xb, q->Tb, batch));
    q->adam_t += 1;
    const float c1 = 1.0f - std::pow(b1, static_cast<float>(q->adam_t));
    const float c2 = 1.0f - std::pow(b2, static_cast<float>(q->adam_t));
    mlp::k_adam_bf16<<<296, 256, 0, q->stream>>>(q->p, q->g, q->m, q->v, kNumParams, lr, b1, b2, c1, c2, 1e-8f,
                                                  q->w1, q->w2, q->w3, q->w2t, q->w3t);
    MLP_TRY(q->cuda(cudaGetLastError(), "adam"));
    if (h_loss_trace) {
      double l = 0.0;
      MLP_TRY(q->cuda(cudaMemcpyAsync(&l, q->loss, sizeof l, cudaMemcpyDeviceToHost, q->stream), "loss"));
      MLP_TRY(q->cuda(cudaStreamSynchronize(q->stream), "sync"));
      h_loss_trace[s] = static_cast<float>(l);
    }
  }
  return check_err(q);
}

int mppi_mlp_grad(mppi_mlp *q, const void *d_X, const float *d_T, int B, float *h_grads, double *h_loss) {
  if (!q || !d_X || !d_T || B < 1 || !h_grads) return MPPI_EINVAL;
  if ((reinterpret_cast<uintptr_t>(d_X) | reinterpret_cast<uintptr_t>(d_T)) & 15u)
    return q->fail(MPPI_EINVAL, "d_X and d_T must be 16-byte aligned (their rows are read as 16-byte vectors)");
  MLP_TRY(ensure_batch(q, B));
  const __nv_bfloat16 *X = static_cast<const __nv_bfloat16 *>(d_X);
  MLP_TRY(forward(q, X, B, true));
  MLP_TRY(backward(q, X, d_T, B));
  MLP_TRY(q->cuda(cudaMemcpyAsync(h_grads, q->g, sizeof(float) * kNumParams, cudaMemcpyDeviceToHost, q->stream), "g"));
  double l = 0.0;
  MLP_TRY(q->cuda(cudaMemcpyAsync(&l, q->loss, sizeof l, cudaMemcpyDeviceToHost, q->stream), "loss"));
  MLP_TRY(check_err(q));
  if (h_loss) *h_loss = l;
  return MPPI_OK;
}

int mppi_mlp_predict(mppi_mlp *q, const float *d_states, const float *d_controls, int n, float *d_next) {
  const NvtxRange range("mppi_mlp_predict (tensor-core forward)");
  if (!q || !d_states || !d_controls || !d_next || n < 1) return MPPI_EINVAL;
  MLP_TRY(ensure_batch(q, ((n + 127) / 128) * 128));
  mlp::k_features<<<(n + 255) / 256, 256, 0, q->stream>>>(d_states, d_controls, n, q->Xb);
  MLP_TRY(q->cuda(cudaGetLastError(), "features"));
  MLP_TRY(forward(q, q->Xb, n, false));
  mlp::k_apply<<<(n * kState + 255) / 256, 256, 0, q->stream>>>(d_states, q->Y, q->out_scale, n, d_next);
  MLP_TRY(q->cuda(cudaGetLastError(), "apply"));
  return check_err(q);
}

int mppi_car_step(const float *d_states, const float *d_controls, int n, float dt, float *d_next, void *stream) {
  if (!d_states || !d_controls || !d_next || n < 1 || !(dt > 0.0f)) return MPPI_EINVAL;
  mlp::k_analytic_step<<<(n + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(d_states, d_controls, n, dt,
                                                                                         d_next);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? MPPI_OK : MPPI_ECUDA;
}

}  // extern "C"
