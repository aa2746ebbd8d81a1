// Host runtime of the MPPI C ABI (include/mppi.h): controller contexts, device
// memory, the CUDA graph of one iteration, and the plain-loop baseline.
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>

#include <cstring>
#include <new>
#include <utility>
#include <string>
#include <vector>

#include "../../include/mppi.h"
#include "alloc_fault.h"
#include "forest_grid.h"
#include "host_params.h"
#include "nvtx_range.h"
#include "kernels.cuh"
#include "mlp_model.cuh"

namespace mppi {
std::atomic<int> g_alloc_fail_countdown{-1};
}

using namespace mppi;

namespace {

thread_local std::string g_create_error;

int state_dim(int sys) {
  switch (sys) {
    case MPPI_CARTPOLE: return 4;
    case MPPI_CAR: return 7;
    case MPPI_QUAD: return 12;
    case MPPI_CAR_MLP: return 7;
    case MPPI_CARTPOLE_VEL: return 4;
    default: return 0;
  }
}
int control_dim(int sys) {
  switch (sys) {
    case MPPI_CARTPOLE: return 1;
    case MPPI_CAR: return 2;
    case MPPI_QUAD: return 4;
    case MPPI_CAR_MLP: return 2;
    case MPPI_CARTPOLE_VEL: return 1;
    default: return 0;
  }
}

using host::cholesky_psd;
using host::invert;
using host::symmetric;

// Bump allocator over one device allocation (256-byte aligned slices).
struct Arena {
  char *base = nullptr;
  size_t size = 0, used = 0;
  template <class T>
  T *take(size_t count) {
    const size_t bytes = (sizeof(T) * count + 255) & ~static_cast<size_t>(255);
    if (used + bytes > size) return nullptr;
    T *p = reinterpret_cast<T *>(base + used);
    used += bytes;
    return p;
  }
};

}  // namespace

struct mppi_ctx {
  int sys = 0, K = 0, T = 0, m = 0, n = 0;
  int impl = MPPI_IMPL_FUSED;
  int weighting = MPPI_WEIGHT_PATH;
  float *d_gen = nullptr;    // general sampling covariance: [T][2][m][m] (chol, R - lambda Sigma_E^-1)
  float *d_prho = nullptr;   // cost-to-go weighting: per-step block minima [nblk_cap][T]
  DF *d_peta = nullptr;      // and normalisers [nblk_cap][T] (double-FP32 pairs)
  int blk = 0, nblk = 0;
  int nblk_cap = 0;  // block partials the arena holds
  CtrlParams p{};
  uint64_t seed = 0;
  std::string err;

  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0;

  Arena arena;
  CtrlState *d_st = nullptr;
  float *d_U = nullptr, *d_uinit = nullptr, *d_u0 = nullptr, *d_S = nullptr, *d_psum = nullptr, *d_dU = nullptr;
  BlockPartial *d_part = nullptr;
  StepDebug *d_dbg = nullptr;
  float *d_du = nullptr;       // plain-loop / debug noise [TM][K] (lazy)
  double *d_plain = nullptr;   // plain-loop reduction scratch, inside the d_du allocation
  uint32_t *d_ctr = nullptr;   // scratch counter for mppi_get_noise
  float *d_env = nullptr;      // cost map or forest (separate allocation)
  size_t env_bytes = 0;
  bool env_ok = false;
  unsigned char *d_mlp = nullptr;  // learned dynamics: MlpDev + tiles + biases
  bool mlp_ok = false;
  int mlp_precision = 0;
  int *d_mlp_err = nullptr;

  float *h_x0 = nullptr, *h_u0 = nullptr;    // pinned, mapped: the step graphs copy x0 from
  float *dh_x0 = nullptr, *dh_u0 = nullptr;  // h_x0 and write u0 into h_u0 directly
  unsigned int *h_ready = nullptr, *dh_ready = nullptr;  // pinned, mapped: set once u0 is in h_u0

  // The controls live in two buffers of T*m floats in d_U: half `ub` is current, and every
  // shift writes the shifted update into the other half and makes it current (host-side
  // bookkeeping: every shift is a call on this ctx, in stream order).  Each step graph is
  // therefore captured once per half.
  int ub = 0;
  float *U_cur() const { return d_U + static_cast<size_t>(ub) * T * m; }
  float *U_nxt() const { return d_U + static_cast<size_t>(ub ^ 1) * T * m; }

  cudaGraphExec_t graph[2] = {nullptr, nullptr};        // mppi_step: rollout -> merge
  cudaGraphExec_t graph_shift[2] = {nullptr, nullptr};  // mppi_step_shift: rollout -> merge + shift
  bool graph_dirty = true;
  cudaGraphExec_t iter_graph[2] = {nullptr, nullptr};  // mppi_iterate_async: rollout -> merge + shift
  bool iter_graph_dirty = true;
  const float *iter_x0 = nullptr;
  float *iter_u0 = nullptr;

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
  bool needs_env() const { return sys == MPPI_CAR || sys == MPPI_QUAD || sys == MPPI_CAR_MLP; }
};

#define MPPI_TRY(expr)             \
  do {                             \
    const int _rc = (expr);        \
    if (_rc != MPPI_OK) return _rc; \
  } while (0)

namespace {

int launch_rollout(mppi_ctx *c, const float *x0, cudaStream_t s) {
  if (c->sys == MPPI_CAR_MLP)
    return c->cuda(launch_rollout_mlp(c->p, x0, c->d_st, c->U_cur(), c->d_S, c->d_psum, c->d_part, c->mlp_precision, s),
                   "mlp rollout launch");
  if (c->weighting == MPPI_WEIGHT_TO_GO)
    return c->cuda(launch_rollout_to_go(c->sys, c->blk, c->p, x0, c->d_st, c->U_cur(), c->d_S, c->d_psum, c->d_part,
                                        c->d_prho, c->d_peta, s),
                   "cost-to-go rollout launch");
  return c->cuda(launch_rollout_fused(c->sys, c->blk, c->p, x0, c->d_st, c->U_cur(), c->d_S, c->d_psum, c->d_part, s),
                 "fused rollout launch");
}

// u0_ready: the path-weighting merge raises this mapped flag once u0 is in u0_out
int launch_update(mppi_ctx *c, float *u0_out, cudaStream_t s, unsigned int *u0_ready = nullptr) {
  if (c->weighting == MPPI_WEIGHT_TO_GO)
    return c->cuda(launch_merge_to_go(c->nblk, c->p, c->d_psum, c->d_prho, c->d_peta, c->d_part, c->U_cur(), u0_out,
                                      c->d_dU, c->d_dbg, s, false, nullptr, nullptr, nullptr, u0_ready),
                   "cost-to-go merge launch");
  return c->cuda(
      launch_merge_update(c->nblk, c->p, c->d_psum, c->d_part, c->U_cur(), u0_out, c->d_dU, c->d_dbg, s, u0_ready),
      "merge launch");
}

// The update and Algorithm 1's shift in one launch, from the current control buffer into the
// other one.  The caller makes the other buffer current once the launch (or the graph that
// holds it) is enqueued.
int launch_update_shift(mppi_ctx *c, float *u0_out, cudaStream_t s, unsigned int *u0_ready = nullptr) {
  if (c->weighting == MPPI_WEIGHT_PATH)
    return c->cuda(launch_merge_update_shift(c->nblk, c->p, c->d_psum, c->d_part, c->U_cur(), c->U_nxt(), u0_out,
                                             c->d_dU, c->d_dbg, c->d_uinit, c->d_st, s, u0_ready),
                   "merge + shift launch");
  return c->cuda(launch_merge_to_go(c->nblk, c->p, c->d_psum, c->d_prho, c->d_peta, c->d_part, c->U_cur(), u0_out,
                                    c->d_dU, c->d_dbg, s, true, c->d_uinit, c->d_st, c->U_nxt(), u0_ready),
                 "cost-to-go merge + shift launch");
}

// Algorithm 1's shift on its own (the shift kernel), then the other buffer is current.
int enqueue_shift(mppi_ctx *c, cudaStream_t s) {
  MPPI_TRY(c->cuda(launch_shift(c->p, c->U_cur(), c->U_nxt(), c->d_uinit, c->d_st, s), "shift launch"));
  c->ub ^= 1;
  return MPPI_OK;
}

// Blocks the rollout launches for this ctx's samples (all of K, or its shard).
int block_count(const mppi_ctx *c) {
  return (shard_samples(c->p) + fused_block_samples(c->blk) - 1) / fused_block_samples(c->blk);
}

int enqueue_fused(mppi_ctx *c, cudaStream_t s) {
  MPPI_TRY(launch_rollout(c, c->d_st->x0, s));
  return launch_update(c, c->d_u0, s);
}

// du [T*m][K] for the plain loop and the noise check hook, followed (256-byte aligned) by the
// plain loop's FP64 reduction scratch; allocated on first use.
int ensure_noise_buffer(mppi_ctx *c) {
  if (c->d_du) return MPPI_OK;
  const size_t du_bytes = (sizeof(float) * static_cast<size_t>(c->T) * c->m * c->K + 255) & ~static_cast<size_t>(255);
  MPPI_TRY(c->cuda(cudaMalloc(&c->d_du, du_bytes + sizeof(double) * plain_scratch_doubles(c->p)), "cudaMalloc(noise)"));
  c->d_plain = reinterpret_cast<double *>(reinterpret_cast<char *>(c->d_du) + du_bytes);
  return MPPI_OK;
}

int enqueue_plain(mppi_ctx *c, cudaStream_t s) {
  MPPI_TRY(ensure_noise_buffer(c));
  MPPI_TRY(c->cuda(launch_plain_noise(c->p, &c->d_st->counter, c->d_du, s), "plain noise"));
  MPPI_TRY(c->cuda(launch_plain_rollout(c->sys, c->p, c->d_st, c->U_cur(), c->d_du, c->d_S, s), "plain rollout"));
  return c->cuda(launch_plain_reduce_update(c->p, c->d_S, c->d_du, c->U_cur(), c->d_u0, c->d_dU, c->d_dbg, c->d_plain, s),
                 "plain reduce/update");
}

// Capture one step graph for the current control buffer: x0 copied from the pinned buffer
// (one DMA: cheaper than every CTA reading mapped host memory), the merge writes u0 straight
// into the mapped pinned buffer (no copy node) and then raises the mapped ready flag, and with
// `shift` the shift runs in the same launch.
int capture_step(mppi_ctx *c, bool shift, cudaGraphExec_t *out) {
  if (*out) {
    cudaGraphExecDestroy(*out);
    *out = nullptr;
  }
  cudaGraph_t g = nullptr;
  MPPI_TRY(c->cuda(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "begin capture"));
  int rc = c->cuda(cudaMemcpyAsync(c->d_st->x0, c->h_x0, sizeof(float) * c->n, cudaMemcpyHostToDevice, c->stream),
                   "x0 copy");
  if (rc == MPPI_OK) rc = launch_rollout(c, c->d_st->x0, c->stream);
  if (rc == MPPI_OK)
    rc = shift ? launch_update_shift(c, c->dh_u0, c->stream, c->dh_ready)
               : launch_update(c, c->dh_u0, c->stream, c->dh_ready);
  const int rc_end = c->cuda(cudaStreamEndCapture(c->stream, &g), "end capture");
  if (rc != MPPI_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  MPPI_TRY(rc_end);
  rc = c->cuda(cudaGraphInstantiate(out, g, 0), "graph instantiate");
  cudaGraphDestroy(g);
  return rc;
}

// Both step graphs for each control buffer.
int build_graph(mppi_ctx *c) {
  const int ub = c->ub;
  int rc = MPPI_OK;
  for (int q = 0; q < 2 && rc == MPPI_OK; ++q) {
    c->ub = q;
    rc = capture_step(c, false, &c->graph[q]);
    if (rc == MPPI_OK) rc = capture_step(c, true, &c->graph_shift[q]);
  }
  c->ub = ub;
  MPPI_TRY(rc);
  c->graph_dirty = false;
  return MPPI_OK;
}

int check_ready(mppi_ctx *c) {
  if (c->needs_env() && !c->env_ok) return c->fail(MPPI_ESTATE, "system needs an environment (mppi_set_env)");
  if (c->sys == MPPI_CAR_MLP && !c->mlp_ok) return c->fail(MPPI_ESTATE, "learned dynamics need MPPI_ENV_MLP weights");
  if (c->sys == MPPI_CAR_MLP && c->impl == MPPI_IMPL_PLAIN)
    return c->fail(MPPI_EINVAL, "the plain loop is not built for the learned dynamics");
  return MPPI_OK;
}

int check_mlp_error(mppi_ctx *c) {
  if (c->sys != MPPI_CAR_MLP) return MPPI_OK;
  int e = 0;
  MPPI_TRY(c->cuda(cudaMemcpyAsync(&e, c->d_mlp_err, sizeof e, cudaMemcpyDeviceToHost, c->stream), "err copy"));
  MPPI_TRY(c->cuda(cudaStreamSynchronize(c->stream), "sync"));
  return e ? c->fail(MPPI_ETIMEOUT, "a tensor-core wait of the learned-dynamics rollout ran out") : MPPI_OK;
}

// round-to-nearest-even float -> bfloat16 bits
uint16_t to_bf16_bits(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return static_cast<uint16_t>((u >> 16) | ((u & 0xffffu) ? 0x40u : 0u));
  u += 0x7fffu + ((u >> 16) & 1u);
  return static_cast<uint16_t>(u >> 16);
}

// round-to-nearest-even float -> E4M3 (1 sign, 4 exponent bits with bias 7, 3 fraction
// bits; largest finite 448, no infinities); out-of-range values saturate to +-448
uint8_t to_e4m3_bits(float f) {
  if (std::isnan(f)) return 0x7f;
  const uint8_t sign = std::signbit(f) ? 0x80 : 0x00;
  const float a = std::fabs(f);
  if (a >= 464.0f) return sign | 0x7e;
  if (a < 0.015625f) {  // subnormals: m * 2^-9, m = 0..7 (m = 8 is the smallest normal)
    const int m = static_cast<int>(std::nearbyint(a * 512.0f));
    return sign | static_cast<uint8_t>(m);
  }
  int e;
  const float fr = std::frexp(a, &e);  // a = fr * 2^e, fr in [0.5, 1)
  float q = std::nearbyint(fr * 16.0f);
  if (q >= 16.0f) {
    q = 8.0f;
    e += 1;
  }
  const int be = e - 1 + 7;
  if (be > 15 || (be == 15 && q - 8.0f > 6.0f)) return sign | 0x7e;
  return sign | static_cast<uint8_t>((be << 3) | static_cast<int>(q - 8.0f));
}

// weights W [rows][cols] -> K-major core-matrix tile (rows = output units, K = kpad >= cols)
// of BF16 (esize 2) or E4M3 (esize 1, values divided by `scale` first)
void to_tile(const float *W, int rows, int cols, int kpad, int esize, float scale, unsigned char *dst) {
  const int per = 16 / esize;
  for (int r = 0; r < rows; ++r)
    for (int k = 0; k < kpad; ++k) {
      const uint32_t off =
          static_cast<uint32_t>((((k / per) * (rows >> 3) + (r >> 3)) << 7) + ((r & 7) << 4) + (k % per) * esize);
      const float w = k < cols ? W[static_cast<size_t>(r) * cols + k] : 0.0f;
      if (esize == 2) {
        const uint16_t b = to_bf16_bits(w);
        std::memcpy(dst + off, &b, 2);
      } else {
        dst[off] = to_e4m3_bits(w / scale);
      }
    }
}

float max_abs(const float *a, size_t n) {
  float m = 0.0f;
  for (size_t i = 0; i < n; ++i) m = std::fmax(m, std::fabs(a[i]));
  return m;
}

int set_mlp_env(mppi_ctx *c, const void *blob, size_t bytes) {
  if (c->sys != MPPI_CAR_MLP) return c->fail(MPPI_EINVAL, "learned-dynamics weights for a system without them");
  if (bytes != sizeof(mppi_env_mlp) + sizeof(float) * mlp::kNumParams)
    return c->fail(MPPI_EINVAL, "MLP blob must hold the header and %d floats", static_cast<int>(mlp::kNumParams));
  mppi_env_mlp h;
  std::memcpy(&h, blob, sizeof h);
  if (h.precision != 0 && h.precision != 1) return c->fail(MPPI_EINVAL, "unsupported MLP precision %d", h.precision);
  const float *P = reinterpret_cast<const float *>(static_cast<const char *>(blob) + sizeof h);
  for (size_t i = 0; i < mlp::kNumParams; ++i)
    if (!std::isfinite(P[i])) return c->fail(MPPI_EINVAL, "non-finite MLP parameter");
  MPPI_TRY(c->cuda(cudaStreamSynchronize(c->stream), "sync"));  // no step of this ctx in flight
  const int E = h.precision == 0 ? 2 : 1, K1 = h.precision == 0 ? 16 : 32;
  float sc[3] = {1.0f, 1.0f, 1.0f};
  if (h.precision == 1) {  // per-tensor scales: the largest weight maps to the largest E4M3 value
    const float m1 = max_abs(P + mlp::kOffW1, 256 * 16), m2 = max_abs(P + mlp::kOffW2, 256 * 256),
                m3 = max_abs(P + mlp::kOffW3, 16 * 256);
    sc[0] = m1 > 0.0f ? m1 / 448.0f : 1.0f;
    sc[1] = m2 > 0.0f ? m2 / 448.0f : 1.0f;
    sc[2] = m3 > 0.0f ? m3 / 448.0f : 1.0f;
  }
  const size_t off_w1 = 256, off_w2 = off_w1 + 256 * K1 * E, off_w3 = off_w2 + 256 * 256 * E,
               off_b = off_w3 + 16 * 256 * E, total = off_b + sizeof(float) * (256 + 256 + 16);
  std::vector<unsigned char> host(total, 0);
  to_tile(P + mlp::kOffW1, 256, 16, K1, E, sc[0], host.data() + off_w1);
  to_tile(P + mlp::kOffW2, 256, 256, 256, E, sc[1], host.data() + off_w2);
  to_tile(P + mlp::kOffW3, 16, 256, 256, E, sc[2], host.data() + off_w3);
  std::memcpy(host.data() + off_b, P + mlp::kOffB1, sizeof(float) * 256);
  std::memcpy(host.data() + off_b + 1024, P + mlp::kOffB2, sizeof(float) * 256);
  std::memcpy(host.data() + off_b + 2048, P + mlp::kOffB3, sizeof(float) * 16);
  MPPI_TRY(c->cuda(cudaStreamSynchronize(c->stream), "sync"));
  if (c->d_mlp) {
    cudaFree(c->d_mlp);
    c->d_mlp = nullptr;
  }
  MPPI_TRY(c->cuda(cudaMalloc(&c->d_mlp, total), "cudaMalloc(mlp)"));
  MlpDev d{};
  d.w1 = c->d_mlp + off_w1;
  d.w2 = c->d_mlp + off_w2;
  d.w3 = c->d_mlp + off_w3;
  d.b1 = reinterpret_cast<const float *>(c->d_mlp + off_b);
  d.b2 = d.b1 + 256;
  d.b3 = d.b2 + 256;
  for (int i = 0; i < 7; ++i) d.out_scale[i] = h.out_scale[i];
  for (int i = 0; i < 3; ++i) d.w_scale[i] = sc[i];
  d.err = c->d_mlp_err;
  d.precision = h.precision;
  std::memcpy(host.data(), &d, sizeof d);
  c->mlp_precision = h.precision;
  MPPI_TRY(c->cuda(cudaMemcpy(c->d_mlp, host.data(), total, cudaMemcpyHostToDevice), "mlp copy"));
  MPPI_TRY(c->cuda(cudaMemset(c->d_mlp_err, 0, sizeof(int)), "err zero"));
  c->p.mlp = c->d_mlp;
  c->mlp_ok = true;
  c->graph_dirty = c->iter_graph_dirty = true;
  return MPPI_OK;
}

}  // namespace

extern "C" {

int mppi_debug_fail_allocations(int after_n) {
  g_alloc_fail_countdown.store(after_n < 0 ? -1 : after_n);
  return MPPI_OK;
}

const char *mppi_version(void) { return "mppi-b300 0.1 (sm_103a)"; }

const char *mppi_last_error(mppi_ctx *ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

int mppi_create(mppi_system sys, int K, int T, float dt, float nu, float lambda, const float *Sigma, const float *R,
                mppi_ctx **out) {
  if (!out) return MPPI_EINVAL;
  *out = nullptr;
  const int n = state_dim(sys), m = control_dim(sys);
  auto bad = [](const char *msg) {
    g_create_error = msg;
    return MPPI_EINVAL;
  };
  if (n == 0) return bad("unknown system");
  if (K < 1 || K > (1 << 20)) return bad("K out of range [1, 1048576]");
  if (T < 1 || T > 1024) return bad("T out of range [1, 1024]");
  float Lnu[kMaxM * kMaxM], Rf[kMaxM * kMaxM];
  if (const char *why = host::control_constants(m, dt, nu, lambda, Sigma, R, Lnu, Rf)) return bad(why);

  mppi_ctx *c = new (std::nothrow) mppi_ctx();
  if (!c) return MPPI_ENOMEM;
  c->sys = sys;
  c->K = K;
  c->T = T;
  c->m = m;
  c->n = n;
  CtrlParams &p = c->p;
  p.K = K;
  p.T = T;
  p.m = m;
  p.n = n;
  p.dt = dt;
  p.nu = nu;
  p.lambda = lambda;
  p.inv_lambda = 1.0f / lambda;
  p.is_du = 0.5f * static_cast<float>(1.0 - 1.0 / static_cast<double>(nu));
  for (int i = 0; i < m * m; ++i) {
    p.Lnu[i] = Lnu[i];
    p.R[i] = Rf[i];
  }
  p.key_lo = 0;
  p.key_hi = 0;
  p.gid = 0;
  p.map_w = p.map_h = 2;
  p.map_inv_cell = 1.0f;

  c->blk = fused_block_size(sys, p);
  if (sys == MPPI_CAR_MLP) {
    if (T > kMlpMaxT) {
      delete c;
      return bad("T out of range [1, 500] for the learned dynamics");
    }
    c->blk = kFusedBlockRegen;  // 128 samples per block, du regenerated
  }
  if (c->blk == 0) {
    delete c;
    return bad("T*m too large for the fused rollout's shared memory");
  }
  c->nblk = block_count(c);

  int rc = c->cuda(cudaGetDevice(&c->device), "cudaGetDevice");
  if (rc == MPPI_OK) rc = c->cuda(prepare_kernels(), "kernel attributes");
  if (rc == MPPI_OK && sys == MPPI_CAR_MLP) rc = c->cuda(prepare_mlp_kernel(), "mlp kernel attributes");
  if (rc == MPPI_OK) rc = c->cuda(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking), "stream");
  if (rc == MPPI_OK) c->own_stream = true;
  const size_t TM = static_cast<size_t>(T) * m;
  const size_t nb_max = (K + kMinBlockSamples - 1) / kMinBlockSamples;  // block partials of any shape fit
  c->nblk_cap = static_cast<int>(nb_max);
  c->arena.size = 256 * 16 + sizeof(CtrlState) + sizeof(float) * (3 * TM + 2 * kMaxM + K + nb_max * TM) +
                  sizeof(BlockPartial) * nb_max + sizeof(StepDebug) + 2 * sizeof(uint32_t);
  if (rc == MPPI_OK) rc = c->cuda(dev_malloc(&c->arena.base, c->arena.size), "cudaMalloc(arena)");
  if (rc == MPPI_OK) {
    c->d_st = c->arena.take<CtrlState>(1);
    c->d_U = c->arena.take<float>(2 * TM);  // two control buffers (shifts alternate them)
    c->d_dU = c->arena.take<float>(TM);
    c->d_uinit = c->arena.take<float>(kMaxM);
    c->d_u0 = c->arena.take<float>(kMaxM);
    c->d_S = c->arena.take<float>(K);
    c->d_psum = c->arena.take<float>(nb_max * TM);
    c->d_part = c->arena.take<BlockPartial>(nb_max);
    c->d_dbg = c->arena.take<StepDebug>(1);
    c->d_ctr = c->arena.take<uint32_t>(1);
    c->d_mlp_err = c->arena.take<int>(1);
    if (!c->d_mlp_err) rc = c->fail(MPPI_ENOMEM, "arena too small");
  }
  if (rc == MPPI_OK) rc = c->cuda(cudaMemsetAsync(c->arena.base, 0, c->arena.size, c->stream), "memset");
  if (rc == MPPI_OK)
    rc = c->cuda(host_alloc(&c->h_x0, sizeof(float) * kMaxN, cudaHostAllocMapped),
                 "cudaHostAlloc");
  if (rc == MPPI_OK)
    rc = c->cuda(host_alloc(&c->h_u0, sizeof(float) * kMaxM, cudaHostAllocMapped),
                 "cudaHostAlloc");
  if (rc == MPPI_OK)
    rc = c->cuda(cudaHostGetDevicePointer(reinterpret_cast<void **>(&c->dh_x0), c->h_x0, 0), "mapped x0");
  if (rc == MPPI_OK)
    rc = c->cuda(cudaHostGetDevicePointer(reinterpret_cast<void **>(&c->dh_u0), c->h_u0, 0), "mapped u0");
  if (rc == MPPI_OK)
    rc = c->cuda(host_alloc(&c->h_ready, sizeof(unsigned int), cudaHostAllocMapped),
                 "cudaHostAlloc");
  if (rc == MPPI_OK)
    rc = c->cuda(cudaHostGetDevicePointer(reinterpret_cast<void **>(&c->dh_ready), c->h_ready, 0), "mapped flag");
  if (rc == MPPI_OK) rc = c->cuda(cudaStreamSynchronize(c->stream), "sync");
  if (rc != MPPI_OK) {
    g_create_error = c->err;
    mppi_destroy(c);
    return rc;
  }
  *out = c;
  return MPPI_OK;
}

int mppi_debug_forest_nearest(const float *obs, int n_obs, int n_points, const float *px, const float *py,
                              float *d_grid, float *d_all, int *in_grid) {
  if (!obs || n_obs < 1 || n_obs > 256 || n_points < 0 || (n_points > 0 && (!px || !py || !d_grid || !d_all || !in_grid)))
    return MPPI_EINVAL;
  ForestGrid g;
  if (!build_forest_grid(obs, n_obs, g)) return MPPI_EINVAL;
  auto dist = [&](int j, float x, float y) {
    const float ax = x - obs[3 * j], ay = y - obs[3 * j + 1];
    return std::sqrt(std::fma(ax, ax, ay * ay)) - obs[3 * j + 2];
  };
  for (int i = 0; i < n_points; ++i) {
    float all = INFINITY;
    for (int j = 0; j < n_obs; ++j) all = std::fmin(all, dist(j, px[i], py[i]));
    d_all[i] = all;
    const float gx = (px[i] - g.ox) * g.inv_h, gy = (py[i] - g.oy) * g.inv_h;
    in_grid[i] = gx >= 0.0f && gy >= 0.0f && gx < static_cast<float>(g.nx) && gy < static_cast<float>(g.ny);
    if (!in_grid[i]) {
      d_grid[i] = all;
      continue;
    }
    const int cell = static_cast<int>(gy) * g.nx + static_cast<int>(gx);
    float d = INFINITY;
    for (int t = g.off[cell]; t < g.off[cell + 1]; ++t) d = std::fmin(d, dist(g.idx[t], px[i], py[i]));
    d_grid[i] = d;
  }
  return MPPI_OK;
}

int mppi_destroy(mppi_ctx *c) {
  if (!c) return MPPI_OK;
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (int q = 0; q < 2; ++q) {
    if (c->graph[q]) cudaGraphExecDestroy(c->graph[q]);
    if (c->graph_shift[q]) cudaGraphExecDestroy(c->graph_shift[q]);
    if (c->iter_graph[q]) cudaGraphExecDestroy(c->iter_graph[q]);
  }
  if (c->arena.base) cudaFree(c->arena.base);
  if (c->d_du) cudaFree(c->d_du);
  if (c->d_prho) cudaFree(c->d_prho);
  if (c->d_gen) cudaFree(c->d_gen);
  if (c->d_peta) cudaFree(c->d_peta);
  if (c->d_env) cudaFree(c->d_env);
  if (c->d_mlp) cudaFree(c->d_mlp);
  if (c->h_x0) cudaFreeHost(c->h_x0);
  if (c->h_u0) cudaFreeHost(c->h_u0);
  if (c->h_ready) cudaFreeHost(c->h_ready);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
  return MPPI_OK;
}

int mppi_set_stream(mppi_ctx *c, void *stream) {
  if (!c) return MPPI_EINVAL;
  MPPI_TRY(c->cuda(cudaStreamSynchronize(c->stream), "sync"));
  if (c->own_stream) cudaStreamDestroy(c->stream);
  c->own_stream = false;
  c->stream = static_cast<cudaStream_t>(stream);
  c->graph_dirty = c->iter_graph_dirty = true;
  return MPPI_OK;
}

int mppi_set_impl(mppi_ctx *c, mppi_impl impl) {
  if (!c || (impl != MPPI_IMPL_FUSED && impl != MPPI_IMPL_PLAIN)) return MPPI_EINVAL;
  if (impl == MPPI_IMPL_PLAIN && c->weighting == MPPI_WEIGHT_TO_GO)
    return c->fail(MPPI_EINVAL, "the plain loop is built for the path weighting only");
  if (impl == MPPI_IMPL_PLAIN && c->p.gen)
    return c->fail(MPPI_EINVAL, "the plain loop is built for the nu * Sigma sampling covariance only");
  if (impl == MPPI_IMPL_PLAIN && (c->p.k_begin != 0 || c->p.k_count != 0))
    return c->fail(MPPI_EINVAL, "the plain loop runs all K samples: clear the shard first");
  c->impl = impl;
  return MPPI_OK;
}

namespace {
// block shape for the ctx's system, environment and weighting (0 if nothing fits)
int block_shape(mppi_ctx *c, const CtrlParams &p) {
  if (c->sys == MPPI_CAR_MLP) return kFusedBlockRegen;
  return c->weighting == MPPI_WEIGHT_TO_GO ? fused_block_size_to_go(c->sys, p) : fused_block_size(c->sys, p);
}
}  // namespace

int mppi_set_sampling_covariance(mppi_ctx *c, const float *h_Sigma_E) {
  if (!c) return MPPI_EINVAL;
  if (!h_Sigma_E) {
    c->p.gen = nullptr;
  } else {
    if (c->sys == MPPI_CAR_MLP)
      return c->fail(MPPI_EINVAL, "the general sampling covariance is not built for the learned dynamics");
    if (c->impl == MPPI_IMPL_PLAIN)
      return c->fail(MPPI_EINVAL, "the plain loop is built for the nu * Sigma sampling covariance only");
    const int m = c->m, T = c->T, mm = m * m;
    std::vector<float> host(static_cast<size_t>(T) * 2 * mm);
    double Rd[kMaxM * kMaxM];
    for (int a = 0; a < mm; ++a) Rd[a] = c->p.R[a];
    for (int i = 0; i < T; ++i) {
      double S[kMaxM * kMaxM], L[kMaxM * kMaxM], Si[kMaxM * kMaxM];
      for (int a = 0; a < mm; ++a) S[a] = h_Sigma_E[static_cast<size_t>(i) * mm + a];
      if (!symmetric(S, m)) return c->fail(MPPI_EINVAL, "Sigma_E[%d] is not symmetric", i);
      if (!cholesky_psd(S, m, L) || !invert(S, m, Si))
        return c->fail(MPPI_EINVAL, "Sigma_E[%d] is not positive definite", i);
      for (int a = 0; a < m; ++a)
        if (!(L[a * m + a] > 0.0)) return c->fail(MPPI_EINVAL, "Sigma_E[%d] is not positive definite", i);
      float *dst = host.data() + static_cast<size_t>(i) * 2 * mm;
      for (int a = 0; a < mm; ++a) {
        dst[a] = static_cast<float>(L[a]);
        dst[mm + a] = static_cast<float>(Rd[a] - static_cast<double>(c->p.lambda) * Si[a]);
      }
    }
    MPPI_TRY(c->cuda(cudaStreamSynchronize(c->stream), "sync"));  // no step of this ctx in flight
    if (!c->d_gen) MPPI_TRY(c->cuda(cudaMalloc(&c->d_gen, sizeof(float) * host.size()), "cudaMalloc(covariances)"));
    MPPI_TRY(c->cuda(cudaMemcpy(c->d_gen, host.data(), sizeof(float) * host.size(), cudaMemcpyHostToDevice),
                     "covariance copy"));
    c->p.gen = c->d_gen;
  }
  const int blk = block_shape(c, c->p);
  if (blk == 0) {
    c->p.gen = nullptr;
    c->blk = block_shape(c, c->p);
    c->nblk = block_count(c);
    c->graph_dirty = c->iter_graph_dirty = true;
    return c->fail(MPPI_EINVAL, "horizon too long for the per-step covariances in shared memory");
  }
  c->blk = blk;
  c->nblk = block_count(c);
  c->graph_dirty = c->iter_graph_dirty = true;
  return MPPI_OK;
}

int mppi_set_weighting(mppi_ctx *c, int mode) {
  if (!c || (mode != MPPI_WEIGHT_PATH && mode != MPPI_WEIGHT_TO_GO)) return MPPI_EINVAL;
  if (mode == MPPI_WEIGHT_TO_GO) {
    if (c->sys == MPPI_CAR_MLP) return c->fail(MPPI_EINVAL, "the cost-to-go weighting is not built for the learned dynamics");
    if (c->p.k_begin != 0 || c->p.k_count != 0)
      return c->fail(MPPI_EINVAL, "the cost-to-go weighting is not built for K-sharding");
    if (c->impl == MPPI_IMPL_PLAIN) return c->fail(MPPI_EINVAL, "the plain loop is built for the path weighting only");
    if (fused_block_size_to_go(c->sys, c->p) == 0)
      return c->fail(MPPI_EINVAL, "horizon too long for the cost-to-go weighting's shared memory");
    if (!c->d_prho) {
      const size_t n = static_cast<size_t>(c->nblk_cap) * c->T;
      MPPI_TRY(c->cuda(cudaMalloc(&c->d_prho, sizeof(float) * n), "cudaMalloc(step minima)"));
      MPPI_TRY(c->cuda(cudaMalloc(&c->d_peta, sizeof(DF) * n), "cudaMalloc(step normalisers)"));
    }
  }
  c->weighting = mode;
  c->blk = block_shape(c, c->p);
  c->nblk = block_count(c);
  c->graph_dirty = c->iter_graph_dirty = true;
  return MPPI_OK;
}

int mppi_set_seed(mppi_ctx *c, uint64_t seed) {
  if (!c) return MPPI_EINVAL;
  c->seed = seed;
  c->p.key_lo = static_cast<uint32_t>(seed & 0xffffffffu);
  c->p.key_hi = static_cast<uint32_t>(seed >> 32);
  c->graph_dirty = c->iter_graph_dirty = true;
  return MPPI_OK;
}

int mppi_set_controller_id(mppi_ctx *c, uint32_t gid) {
  if (!c) return MPPI_EINVAL;
  c->p.gid = gid;
  c->graph_dirty = c->iter_graph_dirty = true;
  return MPPI_OK;
}

int mppi_set_iteration(mppi_ctx *c, uint32_t counter) {
  if (!c) return MPPI_EINVAL;
  MPPI_TRY(c->cuda(cudaMemcpyAsync(&c->d_st->counter, &counter, sizeof counter, cudaMemcpyHostToDevice, c->stream),
                   "counter copy"));
  return c->cuda(cudaStreamSynchronize(c->stream), "sync");
}

int mppi_get_iteration(mppi_ctx *c, uint32_t *counter) {
  if (!c || !counter) return MPPI_EINVAL;
  MPPI_TRY(c->cuda(cudaMemcpyAsync(counter, &c->d_st->counter, sizeof *counter, cudaMemcpyDeviceToHost, c->stream),
                   "counter copy"));
  return c->cuda(cudaStreamSynchronize(c->stream), "sync");
}

int mppi_set_controls(mppi_ctx *c, const float *U) {
  if (!c || !U) return MPPI_EINVAL;
  MPPI_TRY(c->cuda(cudaMemcpyAsync(c->U_cur(), U, sizeof(float) * c->T * c->m, cudaMemcpyHostToDevice, c->stream),
                   "U copy"));
  return c->cuda(cudaStreamSynchronize(c->stream), "sync");
}

int mppi_get_controls(mppi_ctx *c, float *U) {
  if (!c || !U) return MPPI_EINVAL;
  MPPI_TRY(c->cuda(cudaMemcpyAsync(U, c->U_cur(), sizeof(float) * c->T * c->m, cudaMemcpyDeviceToHost, c->stream),
                   "U copy"));
  return c->cuda(cudaStreamSynchronize(c->stream), "sync");
}

int mppi_set_u_init(mppi_ctx *c, const float *u) {
  if (!c || !u) return MPPI_EINVAL;
  MPPI_TRY(c->cuda(cudaMemcpyAsync(c->d_uinit, u, sizeof(float) * c->m, cudaMemcpyHostToDevice, c->stream),
                   "u_init copy"));
  return c->cuda(cudaStreamSynchronize(c->stream), "sync");
}

int mppi_set_env(mppi_ctx *c, const void *blob, size_t bytes) {
  if (!c || !blob || bytes < sizeof(uint32_t)) return MPPI_EINVAL;
  uint32_t kind;
  std::memcpy(&kind, blob, sizeof kind);
  const char *payload = nullptr;
  size_t payload_bytes = 0;
  CtrlParams np = c->p;
  ForestGrid grid;
  std::vector<char> forest;  // cylinders + grid, when there is a grid
  if (kind == MPPI_ENV_MLP) return set_mlp_env(c, blob, bytes);
  if (kind == MPPI_ENV_MAP) {
    if (c->sys != MPPI_CAR && c->sys != MPPI_CAR_MLP) return c->fail(MPPI_EINVAL, "map env for a non-car system");
    if (bytes < sizeof(mppi_env_map)) return c->fail(MPPI_EINVAL, "map header truncated");
    mppi_env_map h;
    std::memcpy(&h, blob, sizeof h);
    if (h.width < 2 || h.height < 2 || h.width > 16384 || h.height > 16384)
      return c->fail(MPPI_EINVAL, "map size out of range [2, 16384]");
    if (!(h.cell > 0.0f) || !std::isfinite(h.origin_x) || !std::isfinite(h.origin_y))
      return c->fail(MPPI_EINVAL, "bad map geometry");
    payload_bytes = sizeof(float) * static_cast<size_t>(h.width) * h.height;
    if (bytes != sizeof h + payload_bytes) return c->fail(MPPI_EINVAL, "map blob size mismatch");
    payload = static_cast<const char *>(blob) + sizeof h;
    np.map_w = h.width;
    np.map_h = h.height;
    np.map_ox = h.origin_x;
    np.map_oy = h.origin_y;
    np.map_inv_cell = 1.0f / h.cell;
    np.n_obs = 0;
    np.grid_nx = np.grid_ny = np.grid_nidx = 0;
  } else if (kind == MPPI_ENV_FOREST) {
    if (c->sys != MPPI_QUAD) return c->fail(MPPI_EINVAL, "forest env for a non-quadrotor system");
    if (bytes < sizeof(mppi_env_forest)) return c->fail(MPPI_EINVAL, "forest header truncated");
    mppi_env_forest h;
    std::memcpy(&h, blob, sizeof h);
    if (h.n_obstacles < 0 || h.n_obstacles > 256) return c->fail(MPPI_EINVAL, "n_obstacles out of range [0, 256]");
    payload_bytes = sizeof(float) * 3 * static_cast<size_t>(h.n_obstacles);
    if (bytes != sizeof h + payload_bytes) return c->fail(MPPI_EINVAL, "forest blob size mismatch");
    payload = static_cast<const char *>(blob) + sizeof h;
    np.n_obs = h.n_obstacles;
    for (int i = 0; i < 3; ++i) np.goal[i] = h.goal[i];
    // the cylinders, then the nearest-cylinder grid (offsets, indices) in one device buffer
    if (build_forest_grid(reinterpret_cast<const float *>(payload), h.n_obstacles, grid)) {
      np.grid_nx = grid.nx;
      np.grid_ny = grid.ny;
      np.grid_nidx = static_cast<int>(grid.idx.size());
      np.grid_ox = grid.ox;
      np.grid_oy = grid.oy;
      np.grid_inv_h = grid.inv_h;
      forest.assign(payload, payload + payload_bytes);
      const size_t at = forest.size();
      forest.resize(at + grid.bytes());
      std::memcpy(forest.data() + at, grid.off.data(), sizeof(uint16_t) * grid.off.size());
      std::memcpy(forest.data() + at + sizeof(uint16_t) * grid.off.size(), grid.idx.data(), grid.idx.size());
      payload = forest.data();
      payload_bytes = forest.size();
    } else {
      np.grid_nx = np.grid_ny = np.grid_nidx = 0;
    }
    if (block_shape(c, np) == 0) return c->fail(MPPI_EINVAL, "forest too large for shared memory");
  } else {
    return c->fail(MPPI_EINVAL, "unknown env kind 0x%08x", kind);
  }
  MPPI_TRY(c->cuda(cudaStreamSynchronize(c->stream), "sync"));
  if (c->d_env && c->env_bytes < payload_bytes) {
    cudaFree(c->d_env);
    c->d_env = nullptr;
    c->env_bytes = 0;
  }
  if (!c->d_env && payload_bytes > 0) {
    MPPI_TRY(c->cuda(cudaMalloc(&c->d_env, payload_bytes), "cudaMalloc(env)"));
    c->env_bytes = payload_bytes;
  }
  if (payload_bytes > 0)
    MPPI_TRY(c->cuda(cudaMemcpy(c->d_env, payload, payload_bytes, cudaMemcpyHostToDevice), "env copy"));
  if (kind == MPPI_ENV_MAP) {
    np.map = c->d_env;
    np.obs = nullptr;
  } else {
    np.obs = c->d_env;
    np.map = nullptr;
    const char *g = reinterpret_cast<const char *>(c->d_env) + sizeof(float) * 3 * static_cast<size_t>(np.n_obs);
    np.grid_off = np.grid_nx > 0 ? reinterpret_cast<const unsigned short *>(g) : nullptr;
    np.grid_idx = np.grid_nx > 0 ? reinterpret_cast<const unsigned char *>(g) + sizeof(uint16_t) *
                                                                                   (static_cast<size_t>(np.grid_nx) *
                                                                                        np.grid_ny + 1)
                                 : nullptr;
  }
  np.mlp = c->p.mlp;
  c->p = np;
  c->blk = block_shape(c, c->p);
  if (c->blk == 0) return c->fail(MPPI_EINVAL, "environment too large for the block's shared memory");
  c->nblk = block_count(c);
  if (c->nblk > c->nblk_cap) return c->fail(MPPI_EINVAL, "block shape needs more partials than allocated");
  c->env_ok = true;
  c->graph_dirty = c->iter_graph_dirty = true;
  return MPPI_OK;
}

namespace {
// Wait until the step graph's merge has put u0 into host memory (its mapped ready flag), or
// the stream has finished; the rest of the iteration (U, the shift, the counter) may still be
// running, and every later call on the ctx's stream is ordered after it.
int wait_u0(mppi_ctx *c) {
  for (unsigned long it = 1;; ++it) {
    if (*reinterpret_cast<volatile unsigned int *>(c->h_ready) != 0u) break;
    if ((it & 63u) == 0u) {
      const cudaError_t q = cudaStreamQuery(c->stream);
      if (q == cudaSuccess) break;
      if (q != cudaErrorNotReady) return c->cuda(q, "step");
    }
  }
  std::atomic_thread_fence(std::memory_order_acquire);
  return MPPI_OK;
}

int step_host(mppi_ctx *c, const float *state, float *u0_out, bool shift) {
  const NvtxRange range(shift ? "mppi_step_shift (rollout, merge + update + shift)" : "mppi_step (rollout, merge + update)");
  if (!c || !state || !u0_out) return MPPI_EINVAL;
  MPPI_TRY(check_ready(c));
  std::memcpy(c->h_x0, state, sizeof(float) * c->n);
  if (c->impl == MPPI_IMPL_PLAIN || c->stream == nullptr) {
    // the plain loop, or the legacy stream (which cannot be captured): launch directly
    MPPI_TRY(c->cuda(cudaMemcpyAsync(c->d_st->x0, c->h_x0, sizeof(float) * c->n, cudaMemcpyHostToDevice, c->stream),
                     "x0 copy"));
    MPPI_TRY(c->impl == MPPI_IMPL_PLAIN ? enqueue_plain(c, c->stream) : enqueue_fused(c, c->stream));
    MPPI_TRY(c->cuda(cudaMemcpyAsync(c->h_u0, c->d_u0, sizeof(float) * c->m, cudaMemcpyDeviceToHost, c->stream),
                     "u0 copy"));
    if (shift) MPPI_TRY(enqueue_shift(c, c->stream));
  } else {
    if (c->graph_dirty) MPPI_TRY(build_graph(c));
    // the merge raises the ready flag; the learned dynamics also need the kernel's own
    // status, read after the stream finishes
    const bool flag = c->sys != MPPI_CAR_MLP;
    if (flag) *reinterpret_cast<volatile unsigned int *>(c->h_ready) = 0u;
    MPPI_TRY(c->cuda(cudaGraphLaunch(shift ? c->graph_shift[c->ub] : c->graph[c->ub], c->stream), "graph launch"));
    if (shift) c->ub ^= 1;
    if (flag) {
      MPPI_TRY(wait_u0(c));
      std::memcpy(u0_out, c->h_u0, sizeof(float) * c->m);
      return MPPI_OK;
    }
  }
  MPPI_TRY(c->cuda(cudaStreamSynchronize(c->stream), "sync"));
  MPPI_TRY(check_mlp_error(c));
  std::memcpy(u0_out, c->h_u0, sizeof(float) * c->m);
  return MPPI_OK;
}
}  // namespace

int mppi_step(mppi_ctx *c, const float *state, float *u0_out) { return step_host(c, state, u0_out, false); }

int mppi_step_shift(mppi_ctx *c, const float *state, float *u0_out) { return step_host(c, state, u0_out, true); }

int mppi_rollout_async(mppi_ctx *c, const float *d_state) {
  if (!c || !d_state) return MPPI_EINVAL;
  MPPI_TRY(check_ready(c));
  if (c->impl == MPPI_IMPL_PLAIN) {
    MPPI_TRY(c->cuda(cudaMemcpyAsync(c->d_st->x0, d_state, sizeof(float) * c->n, cudaMemcpyDeviceToDevice, c->stream),
                     "x0 copy"));
    MPPI_TRY(ensure_noise_buffer(c));
    MPPI_TRY(c->cuda(launch_plain_noise(c->p, &c->d_st->counter, c->d_du, c->stream), "plain noise"));
    return c->cuda(launch_plain_rollout(c->sys, c->p, c->d_st, c->U_cur(), c->d_du, c->d_S, c->stream), "plain rollout");
  }
  return launch_rollout(c, d_state, c->stream);  // the kernel reads the caller's state directly
}

int mppi_update_async(mppi_ctx *c, float *d_u0_out) {
  if (!c) return MPPI_EINVAL;
  MPPI_TRY(check_ready(c));
  if (c->impl == MPPI_IMPL_PLAIN) {
    MPPI_TRY(c->cuda(launch_plain_reduce_update(c->p, c->d_S, c->d_du, c->U_cur(), c->d_u0, c->d_dU, c->d_dbg, c->d_plain, c->stream),
                     "plain reduce/update"));
    if (d_u0_out)
      MPPI_TRY(c->cuda(cudaMemcpyAsync(d_u0_out, c->d_u0, sizeof(float) * c->m, cudaMemcpyDeviceToDevice, c->stream),
                       "u0 copy"));
    return MPPI_OK;
  }
  return launch_update(c, d_u0_out ? d_u0_out : c->d_u0, c->stream);  // u0 written in place
}

int mppi_step_async(mppi_ctx *c, const float *d_state, float *d_u0_out) {
  const NvtxRange range("mppi_step_async (rollout, merge + update)");
  MPPI_TRY(mppi_rollout_async(c, d_state));
  return mppi_update_async(c, d_u0_out);
}

namespace {
// The iteration graph (rollout -> merge + update + shift) of control buffer q.
int capture_iterate(mppi_ctx *c, int q, const float *d_state, float *u0) {
  if (c->iter_graph[q]) cudaGraphExecDestroy(c->iter_graph[q]);
  c->iter_graph[q] = nullptr;
  const int ub = c->ub;
  c->ub = q;
  cudaGraph_t g = nullptr;
  int rc = c->cuda(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
  if (rc == MPPI_OK) {
    rc = launch_rollout(c, d_state, c->stream);
    if (rc == MPPI_OK) rc = launch_update_shift(c, u0, c->stream);
    const int rc_end = c->cuda(cudaStreamEndCapture(c->stream, &g), "end capture");
    if (rc == MPPI_OK) rc = rc_end;
    if (rc == MPPI_OK) rc = c->cuda(cudaGraphInstantiate(&c->iter_graph[q], g, 0), "graph instantiate");
    if (g) cudaGraphDestroy(g);
  }
  c->ub = ub;
  return rc;
}
}  // namespace

int mppi_iterate_async(mppi_ctx *c, const float *d_state, float *d_u0_out) {
  const NvtxRange range("mppi_iterate_async (graph: rollout, merge + update + shift)");
  if (!c || !d_state) return MPPI_EINVAL;
  MPPI_TRY(check_ready(c));
  if (c->impl == MPPI_IMPL_PLAIN || c->stream == nullptr) {
    MPPI_TRY(mppi_step_async(c, d_state, d_u0_out));
    return enqueue_shift(c, c->stream);
  }
  float *u0 = d_u0_out ? d_u0_out : c->d_u0;
  if (c->iter_graph_dirty || c->iter_graph[0] == nullptr || c->iter_graph[1] == nullptr || c->iter_x0 != d_state ||
      c->iter_u0 != u0) {
    c->iter_graph_dirty = true;
    for (int q = 0; q < 2; ++q) MPPI_TRY(capture_iterate(c, q, d_state, u0));
    c->iter_x0 = d_state;
    c->iter_u0 = u0;
    c->iter_graph_dirty = false;
  }
  MPPI_TRY(c->cuda(cudaGraphLaunch(c->iter_graph[c->ub], c->stream), "graph launch"));
  c->ub ^= 1;
  return MPPI_OK;
}

int mppi_shift(mppi_ctx *c) {
  if (!c) return MPPI_EINVAL;
  return enqueue_shift(c, c->stream);
}

int mppi_get_debug(mppi_ctx *c, float *S, int *argmin, double *eta, float *dU) {
  if (!c) return MPPI_EINVAL;
  StepDebug d;
  MPPI_TRY(c->cuda(cudaMemcpyAsync(&d, c->d_dbg, sizeof d, cudaMemcpyDeviceToHost, c->stream), "dbg copy"));
  if (S) MPPI_TRY(c->cuda(cudaMemcpyAsync(S, c->d_S, sizeof(float) * c->K, cudaMemcpyDeviceToHost, c->stream), "S"));
  if (dU)
    MPPI_TRY(c->cuda(cudaMemcpyAsync(dU, c->d_dU, sizeof(float) * c->T * c->m, cudaMemcpyDeviceToHost, c->stream),
                     "dU"));
  MPPI_TRY(c->cuda(cudaStreamSynchronize(c->stream), "sync"));
  if (argmin) *argmin = d.kstar;
  if (eta) *eta = d.eta;
  return MPPI_OK;
}

int mppi_get_noise(mppi_ctx *c, uint32_t counter, float *h_du) {
  if (!c || !h_du) return MPPI_EINVAL;
  if (c->p.gen) return c->fail(MPPI_EINVAL, "the noise check hook draws the nu * Sigma noise only");
  MPPI_TRY(ensure_noise_buffer(c));
  MPPI_TRY(c->cuda(cudaMemcpyAsync(c->d_ctr, &counter, sizeof counter, cudaMemcpyHostToDevice, c->stream), "ctr"));
  MPPI_TRY(c->cuda(launch_plain_noise(c->p, c->d_ctr, c->d_du, c->stream), "noise launch"));
  MPPI_TRY(c->cuda(cudaMemcpyAsync(h_du, c->d_du, sizeof(float) * static_cast<size_t>(c->T) * c->m * c->K,
                                   cudaMemcpyDeviceToHost, c->stream),
                   "noise copy"));
  return c->cuda(cudaStreamSynchronize(c->stream), "sync");
}

int mppi_philox_words(uint64_t seed, int K, int n_blocks, uint32_t counter, uint32_t gid, uint32_t *h_out) {
  if (K < 1 || n_blocks < 1 || n_blocks > 65535 || !h_out || static_cast<size_t>(K) * n_blocks > (1u << 26))
    return MPPI_EINVAL;
  const size_t bytes = sizeof(uint32_t) * 4 * static_cast<size_t>(K) * n_blocks;
  uint32_t *d = nullptr;
  if (cudaMalloc(&d, bytes) != cudaSuccess) {
    cudaGetLastError();
    return MPPI_ENOMEM;
  }
  cudaError_t e = launch_philox_words(static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32), K, n_blocks,
                                      counter, gid, d, nullptr);
  if (e == cudaSuccess) e = cudaMemcpy(h_out, d, bytes, cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) {
    g_create_error = cudaGetErrorString(e);
    cudaGetLastError();
    return MPPI_ECUDA;
  }
  return MPPI_OK;
}

// ---- K-sharding: one controller's samples over several ranks --------------------------
int mppi_set_shard(mppi_ctx *c, int k_begin, int k_count) {
  if (!c) return MPPI_EINVAL;
  const bool whole = k_begin == 0 && (k_count == 0 || k_count == c->K);
  if (!whole) {
    if (c->sys == MPPI_CAR_MLP) return c->fail(MPPI_EINVAL, "K-sharding is not built for the learned dynamics");
    if (c->impl == MPPI_IMPL_PLAIN) return c->fail(MPPI_EINVAL, "K-sharding runs on the fused path only");
    if (c->weighting != MPPI_WEIGHT_PATH) return c->fail(MPPI_EINVAL, "K-sharding is built for the path weighting only");
    if (k_begin < 0 || k_count < 1 || static_cast<int64_t>(k_begin) + k_count > c->K)
      return c->fail(MPPI_EINVAL, "shard [%d, %d + %d) is not inside [0, K = %d)", k_begin, k_begin, k_count, c->K);
    if (k_begin % kShardAlign != 0 || (k_begin + k_count != c->K && k_count % kShardAlign != 0))
      return c->fail(MPPI_EINVAL, "shard boundaries must be multiples of %d (except at K)", kShardAlign);
  }
  MPPI_TRY(c->cuda(cudaStreamSynchronize(c->stream), "sync"));  // no step of this ctx in flight
  c->p.k_begin = whole ? 0 : k_begin;
  c->p.k_count = whole ? 0 : k_count;
  c->nblk = block_count(c);
  c->graph_dirty = c->iter_graph_dirty = true;
  return MPPI_OK;
}

int mppi_shard_partial_async(mppi_ctx *c, const float *d_state, double *d_partial) {
  const NvtxRange range("mppi_shard_partial_async (rollout, shard partial)");
  if (!c || !d_state || !d_partial) return MPPI_EINVAL;
  MPPI_TRY(check_ready(c));
  if (c->sys == MPPI_CAR_MLP || c->impl == MPPI_IMPL_PLAIN || c->weighting != MPPI_WEIGHT_PATH)
    return c->fail(MPPI_EINVAL, "the shard partial is built for the fused path with the path weighting");
  MPPI_TRY(launch_rollout(c, d_state, c->stream));
  return c->cuda(launch_shard_partial(c->nblk, c->p, c->d_psum, c->d_part, d_partial, c->stream), "shard partial");
}

int mppi_shard_update_async(mppi_ctx *c, const double *d_partials, int n_ranks, float *d_u0_out) {
  const NvtxRange range("mppi_shard_update_async (shard merge + update)");
  if (!c || !d_partials || n_ranks < 1 || n_ranks > 4096) return MPPI_EINVAL;
  MPPI_TRY(check_ready(c));
  MPPI_TRY(c->cuda(launch_shard_update(c->p, d_partials, n_ranks, c->U_cur(), d_u0_out ? d_u0_out : c->d_u0, c->d_dU,
                                       c->d_dbg, c->stream),
                   "shard update"));
  return MPPI_OK;
}

}  // extern "C"
