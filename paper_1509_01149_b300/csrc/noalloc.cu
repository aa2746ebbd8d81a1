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
#include "host_params.h"
#include "nvtx_range.h"
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

// Device address of the scratch on the current device, looked up once per device.  Only a
// successful set-up is remembered: a failed one (for example a first call made during a
// stream capture) is tried again by the next call.
struct DeviceSetup {
  std::mutex mu;
  bool ready = false;
  unsigned char *ptr = nullptr;
};
DeviceSetup g_setup[kMaxDevices];

cudaError_t scratch_for_device(int dev, unsigned char **out) {
  DeviceSetup &s = g_setup[dev];
  std::lock_guard<std::mutex> lock(s.mu);
  if (!s.ready) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e == cudaSuccess) e = prepare_kernels();
    if (e != cudaSuccess) {
      cudaGetLastError();
      return e;
    }
    s.ptr = static_cast<unsigned char *>(p);
    s.ready = true;
  }
  *out = s.ptr;
  return cudaSuccess;
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

size_t round256(size_t b) { return (b + 255) & ~static_cast<size_t>(255); }

}  // namespace

extern "C" int mppi_step_static(mppi_system sys, int K, int T, float dt, float nu, float lambda, const float *h_Sigma,
                                const float *h_R, uint64_t seed, uint32_t gid, uint32_t counter,
                                const void *h_env_header, const float *d_env_payload, size_t env_payload_bytes,
                                const float *d_state,
                                float *d_U, float *d_u0_out, void *cuda_stream, char *h_err, size_t err_len) {
  const ErrorSink fail{h_err, err_len};
  if (h_err && err_len > 0) h_err[0] = '\0';
  const NvtxRange range("mppi_step_static (state copy, rollout, merge + update)");
  int n = 0, m = 0;
  if (dims(sys, &n, &m) != MPPI_OK)
    return fail(MPPI_EINVAL, "unknown or unsupported system (the learned-dynamics car is not served here)");
  if (K < 1 || K > (1 << 20) || T < 1 || T > 1024) return fail(MPPI_EINVAL, "K must be in [1, 1048576] and T in [1, 1024]");
  if (!d_state || !d_U || !d_u0_out) return fail(MPPI_EINVAL, "null state, U or u0 pointer");
  float Lnu[kMaxM * kMaxM], Rf[kMaxM * kMaxM];
  if (const char *why = host::control_constants(m, dt, nu, lambda, h_Sigma, h_R, Lnu, Rf))
    return fail(MPPI_EINVAL, why);

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
  for (int i = 0; i < m * m; ++i) {
    p.Lnu[i] = Lnu[i];
    p.R[i] = Rf[i];
  }

  // environment: a host header describing a device payload the caller owns
  if (sys == MPPI_CAR || sys == MPPI_QUAD) {
    if (!h_env_header || !d_env_payload) return fail(MPPI_EINVAL, "this system needs an environment");
    uint32_t kind;
    std::memcpy(&kind, h_env_header, sizeof kind);
    if (sys == MPPI_CAR) {
      mppi_env_map h;
      std::memcpy(&h, h_env_header, sizeof h);
      if (kind != MPPI_ENV_MAP || h.width < 2 || h.height < 2 || h.width > 16384 || h.height > 16384 ||
          !(h.cell > 0.0f) || !std::isfinite(h.cell) || !std::isfinite(h.origin_x) || !std::isfinite(h.origin_y))
        return fail(MPPI_EINVAL, "bad cost-map header");
      const size_t need = sizeof(float) * static_cast<size_t>(h.width) * static_cast<size_t>(h.height);
      if (env_payload_bytes < need)
        return fail(MPPI_EINVAL, "cost-map payload holds " + std::to_string(env_payload_bytes) + " bytes; the header needs " +
                                     std::to_string(need));
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
      const size_t need = sizeof(float) * 3 * static_cast<size_t>(h.n_obstacles);
      if (env_payload_bytes < need)
        return fail(MPPI_EINVAL, "forest payload holds " + std::to_string(env_payload_bytes) + " bytes; the header needs " +
                                     std::to_string(need));
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
  if (e != cudaSuccess) return fail(MPPI_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices)
    return fail(MPPI_EINVAL, "device " + std::to_string(dev) + " is beyond the " + std::to_string(kMaxDevices) +
                                 " devices this entry point keeps a scratch address for");
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
