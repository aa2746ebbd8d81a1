// mppi_step_static: one MPPI iteration that allocates nothing.
//
// Who needs it: callers that may not allocate device memory once they are running.
// A real-time control loop must not call cudaMalloc after start-up (the call can
// synchronise the whole device and has no latency bound), and some hosts hand out
// every byte of device memory through their own pool, so a library may not take
// memory of its own.  Such callers pass every input and output buffer themselves;
// the per-iteration scratch (path costs, per-block softmax partials, the state
// block the kernels read) lives in the file-scope array below instead.
//
// The array is a static __device__ object: every GPU that loads this library holds
// it (kStaticScratchBytes) until the process exits.  Every call on a device uses
// the same array and leaves its contents behind, so two calls whose work overlaps
// on the GPU (different streams, or different host threads) race on it.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/mppi.h"
#include "kernels.cuh"

using namespace mppi;

namespace {

constexpr size_t kStaticScratchBytes = MPPI_STATIC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

// The scratch.  In host code this name is only a host-side stand-in for the device
// object: its device address comes from cudaGetSymbolAddress (see scratch_for_device).
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Writes the error text into the caller's buffer (if any) and returns the code.
struct ErrorSink {
  char *buf;
  size_t len;
  int operator()(int code, const std::string &msg) const {
    if (buf && len > 0) {
      const size_t k = msg.size() < len - 1 ? msg.size() : len - 1;
      std::memcpy(buf, msg.data(), k);
      buf[k] = '\0';
    }
    return code;
  }
};

// Device address of the scratch on the current device, looked up once per device.
struct DeviceSetup {
  std::once_flag once;
  unsigned char *ptr = nullptr;
  cudaError_t status = cudaSuccess;
};
DeviceSetup g_setup[kMaxDevices];

cudaError_t scratch_for_device(int dev, unsigned char **out) {
  DeviceSetup &s = g_setup[dev];
  std::call_once(s.once, [&s] {
    void *p = nullptr;
    s.status = cudaGetSymbolAddress(&p, g_static_scratch);
    if (s.status == cudaSuccess) s.status = prepare_kernels();
    s.ptr = static_cast<unsigned char *>(p);
  });
  *out = s.ptr;
  return s.status;
}

// Copies the caller's state into the scratch state block and sets the iteration
// counter (a kernel, so no host staging copy is involved).
__global__ void k_static_state(const float *__restrict__ d_state, int n, uint32_t counter, CtrlState *st) {
  const int t = threadIdx.x;
  if (t < kMaxN) st->x0[t] = t < n ? d_state[t] : 0.0f;
  if (t == 0) st->counter = counter;
}

int dims(int sys, int *n, int *m) {
  switch (sys) {
    case MPPI_CARTPOLE: *n = 4; *m = 1; return MPPI_OK;
    case MPPI_CAR: *n = 7; *m = 2; return MPPI_OK;
    case MPPI_QUAD: *n = 12; *m = 4; return MPPI_OK;
    case MPPI_CARTPOLE_VEL: *n = 4; *m = 1; return MPPI_OK;
    default: return MPPI_EINVAL;
  }
}

// Lower Cholesky factor of a symmetric positive semi-definite matrix (double).
bool chol(const double *S, int m, double *L) {
  for (int i = 0; i < m * m; ++i) L[i] = 0.0;
  for (int j = 0; j < m; ++j) {
    double d = S[j * m + j];
    for (int l = 0; l < j; ++l) d -= L[j * m + l] * L[j * m + l];
    if (d < -1e-9 * std::fmax(1.0, std::fabs(S[j * m + j]))) return false;
    L[j * m + j] = std::sqrt(std::fmax(d, 0.0));
    for (int i = j + 1; i < m; ++i) {
      double a = S[i * m + j];
      for (int l = 0; l < j; ++l) a -= L[i * m + l] * L[j * m + l];
      L[i * m + j] = L[j * m + j] > 0.0 ? a / L[j * m + j] : 0.0;
    }
  }
  return true;
}

// Inverse of an SPD matrix from its Cholesky factor (double).
void spd_inverse(const double *L, int m, double *Ai) {
  double Li[kMaxM * kMaxM] = {0};
  for (int j = 0; j < m; ++j) {
    Li[j * m + j] = 1.0 / L[j * m + j];
    for (int i = j + 1; i < m; ++i) {
      double a = 0.0;
      for (int l = j; l < i; ++l) a -= L[i * m + l] * Li[l * m + j];
      Li[i * m + j] = a / L[i * m + i];
    }
  }
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) {
      double a = 0.0;
      for (int l = 0; l < m; ++l) a += Li[l * m + i] * Li[l * m + j];
      Ai[i * m + j] = a;
    }
}

size_t round256(size_t b) { return (b + 255) & ~static_cast<size_t>(255); }

}  // namespace

extern "C" int mppi_step_static(mppi_system sys, int K, int T, float dt, float nu, float lambda, const float *h_Sigma,
                                const float *h_R, uint64_t seed, uint32_t gid, uint32_t counter,
                                const void *h_env_header, const float *d_env_payload, const float *d_state,
                                float *d_U, float *d_u0_out, void *cuda_stream, char *h_err, size_t err_len) {
  const ErrorSink fail{h_err, err_len};
  if (h_err && err_len > 0) h_err[0] = '\0';
  int n = 0, m = 0;
  if (dims(sys, &n, &m) != MPPI_OK) return fail(MPPI_EINVAL, "unknown or unsupported system");
  if (K < 1 || T < 1 || T > 1024) return fail(MPPI_EINVAL, "K must be >= 1 and T in [1, 1024]");
  if (!(dt > 0.0f) || !(nu > 0.0f) || !(lambda > 0.0f)) return fail(MPPI_EINVAL, "dt, nu, lambda must be > 0");
  if (!h_Sigma || !d_state || !d_U || !d_u0_out) return fail(MPPI_EINVAL, "null Sigma, state, U or u0 pointer");

  CtrlParams p{};
  p.K = K;
  p.T = T;
  p.m = m;
  p.n = n;
  p.dt = dt;
  p.nu = nu;
  p.lambda = lambda;
  p.inv_lambda = 1.0f / lambda;
  p.is_du = 0.5f * static_cast<float>(1.0 - 1.0 / static_cast<double>(nu));
  p.key_lo = static_cast<uint32_t>(seed & 0xffffffffu);
  p.key_hi = static_cast<uint32_t>(seed >> 32);
  p.gid = gid;
  p.map_w = p.map_h = 2;
  p.map_inv_cell = 1.0f;

  double S[kMaxM * kMaxM], L[kMaxM * kMaxM], Rd[kMaxM * kMaxM];
  for (int i = 0; i < m * m; ++i) S[i] = h_Sigma[i];
  if (!chol(S, m, L)) return fail(MPPI_EINVAL, "Sigma is not positive semi-definite");
  if (h_R) {
    for (int i = 0; i < m * m; ++i) Rd[i] = h_R[i];
    double LR[kMaxM * kMaxM];
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < i; ++j)
        if (std::fabs(Rd[i * m + j] - Rd[j * m + i]) > 1e-6 * (std::fabs(Rd[i * m + j]) + std::fabs(Rd[j * m + i])))
          return fail(MPPI_EINVAL, "R is not symmetric");
    if (!chol(Rd, m, LR)) return fail(MPPI_EINVAL, "R is not positive definite");
    for (int j = 0; j < m; ++j)
      if (!(LR[j * m + j] > 0.0)) return fail(MPPI_EINVAL, "R is not positive definite");
  } else {
    for (int j = 0; j < m; ++j)
      if (!(L[j * m + j] > 0.0)) return fail(MPPI_EINVAL, "R = lambda Sigma^-1 needs Sigma positive definite");
    double Si[kMaxM * kMaxM];
    spd_inverse(L, m, Si);
    for (int i = 0; i < m * m; ++i) Rd[i] = lambda * Si[i];
  }
  const double snu = std::sqrt(static_cast<double>(nu));
  for (int i = 0; i < m * m; ++i) {
    p.Lnu[i] = static_cast<float>(snu * L[i]);
    p.R[i] = static_cast<float>(Rd[i]);
  }

  // environment: a host header describing a device payload the caller owns
  if (sys == MPPI_CAR || sys == MPPI_QUAD) {
    if (!h_env_header || !d_env_payload) return fail(MPPI_EINVAL, "this system needs an environment");
    uint32_t kind;
    std::memcpy(&kind, h_env_header, sizeof kind);
    if (sys == MPPI_CAR) {
      mppi_env_map h;
      std::memcpy(&h, h_env_header, sizeof h);
      if (kind != MPPI_ENV_MAP || h.width < 2 || h.height < 2 || !(h.cell > 0.0f))
        return fail(MPPI_EINVAL, "bad cost-map header");
      p.map = d_env_payload;
      p.map_w = h.width;
      p.map_h = h.height;
      p.map_ox = h.origin_x;
      p.map_oy = h.origin_y;
      p.map_inv_cell = 1.0f / h.cell;
    } else {
      mppi_env_forest h;
      std::memcpy(&h, h_env_header, sizeof h);
      if (kind != MPPI_ENV_FOREST || h.n_obstacles < 0 || h.n_obstacles > 256)
        return fail(MPPI_EINVAL, "bad forest header");
      p.obs = d_env_payload;
      p.n_obs = h.n_obstacles;
      for (int i = 0; i < 3; ++i) p.goal[i] = h.goal[i];
    }
  }

  const int blk = fused_block_size(sys, p);
  if (blk == 0) return fail(MPPI_EINVAL, "T*m too large for the fused rollout's shared memory");
  const int nblk = (K + fused_block_samples(blk) - 1) / fused_block_samples(blk);
  const size_t TM = static_cast<size_t>(T) * m;
  const size_t need = round256(sizeof(CtrlState)) + round256(sizeof(StepDebug)) + round256(sizeof(float) * TM) +
                      round256(sizeof(float) * static_cast<size_t>(K)) +
                      round256(sizeof(float) * static_cast<size_t>(nblk) * TM) +
                      round256(sizeof(BlockPartial) * static_cast<size_t>(nblk));
  if (need > kStaticScratchBytes)
    return fail(MPPI_EINVAL, "scratch for K=" + std::to_string(K) + ", T=" + std::to_string(T) + " needs " +
                                 std::to_string(need) + " bytes; the static scratch holds " +
                                 std::to_string(kStaticScratchBytes));

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return fail(MPPI_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  unsigned char *base = nullptr;
  e = scratch_for_device(dev, &base);
  if (e != cudaSuccess || !base) return fail(MPPI_ECUDA, std::string("static scratch set-up: ") + cudaGetErrorString(e));

  // carve the scratch (nothing in it needs to start at zero: every slot below is
  // written by the kernels of this call before it is read)
  size_t off = 0;
  auto take = [&](size_t bytes) {
    unsigned char *q = base + off;
    off += round256(bytes);
    return q;
  };
  CtrlState *st = reinterpret_cast<CtrlState *>(take(sizeof(CtrlState)));
  StepDebug *dbg = reinterpret_cast<StepDebug *>(take(sizeof(StepDebug)));
  float *dU = reinterpret_cast<float *>(take(sizeof(float) * TM));
  float *Sk = reinterpret_cast<float *>(take(sizeof(float) * static_cast<size_t>(K)));
  float *psum = reinterpret_cast<float *>(take(sizeof(float) * static_cast<size_t>(nblk) * TM));
  BlockPartial *part = reinterpret_cast<BlockPartial *>(take(sizeof(BlockPartial) * static_cast<size_t>(nblk)));

  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  k_static_state<<<1, 32, 0, s>>>(d_state, n, counter, st);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = launch_rollout_fused(sys, blk, p, st->x0, st, d_U, Sk, psum, part, s);
  if (e == cudaSuccess) e = launch_merge_update(nblk, p, psum, part, d_U, d_u0_out, dU, dbg, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(MPPI_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
  }
  return MPPI_OK;
}
