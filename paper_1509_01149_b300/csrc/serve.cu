// Serving runtime: many MPPI controllers (different systems, K and T) stepped together.
//
// Device side
//   slot table   SlotDesc per admitted controller: constants, buffer pointers into the
//                arena, iteration counter (persistent between ticks).
//   k_serve_rollout<BLK>  persistent: each CTA takes work items (slot, block of BLK
//                samples) from an atomic queue, heaviest first, and runs the fused
//                rollout body.  du is never stored: the block's weighted sums regenerate
//                it from the counter-based generator once the path costs are known, so
//                the rollout writes only S~ and the block partials, and many CTAs share
//                an SM (no du in shared memory).  Items of different systems / K / T run
//                side by side.
//   k_serve_merge          persistent: one slot per CTA taken from a second queue; merge of
//                the slot's block partials (FP64 normaliser, double-FP32 weighted sums), U
//                update, u_0 out, shift, counter++.
// Host side
//   first-fit arena allocator (admission by memory), work-item builder, an autotuner over
//   (BLK, CTAs per SM), and two tick contexts, each a CUDA graph (memset queue counters ->
//   H2D tick buffer -> rollout -> merge -> D2H u_0) whose copy sizes are updated per tick.
//   Synchronous use: mppi_server_tick runs one tick and waits.  Asynchronous use (continuous
//   batching): a scheduler thread takes submitted step requests from a queue and launches
//   them, at most one per controller and tick, into whichever context is idle, so the next
//   tick is filled and enqueued behind the one on the GPU; finished ticks publish their u_0
//   to the request table (poll / wait / reap).  Admission and release work while ticks are
//   in flight: a new slot's uploads go on a separate copy stream, and a released slot's
//   memory returns to the arena when the last tick using it retires.
// No kernel waits on another block or on the host, so nothing here can hang on a flag.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/mppi.h"
#include "alloc_fault.h"
#include "forest_grid.h"
#include "host_params.h"
#include "nvtx_range.h"
#include "merge_common.cuh"
#include "kernels.cuh"
#include "rollout_body.cuh"

namespace mppi {

struct SlotDesc {
  CtrlParams p;
  int sys, tm, nblk, blk;  // nblk and blk adjacent: the host refreshes just these two
  float *U, *u_init, *S, *part_sums;
  BlockPartial *part;
  uint32_t counter;
  int kstar;
  float rho;
  float pad;
  double eta;
};

struct WorkItem {
  int slot, tick, block, pad;
};

struct TickHeader {
  int n_items, n_slots, pad0, pad1;
};

struct ServeArgs {
  SlotDesc *slots;
  const TickHeader *hdr;
  const int *tick_slots;   // [n_slots]
  const float *states;     // [n_slots][16]
  const WorkItem *items;   // [n_items]
  float *u0_out;           // [n_slots][4]
  int *counters;           // [0] rollout queue, [1] merge queue
};

constexpr int kServeMergeThreads = 256;
constexpr int kServeMaxK = 65536;
constexpr int kServeMaxT = 256;

template <int BLK, int MINB>
__global__ void __launch_bounds__(BLK, MINB) k_serve_rollout(const ServeArgs a) {
  extern __shared__ __align__(16) float smem[];
  __shared__ CtrlParams s_p;
  __shared__ int s_item;
  constexpr int kWords = static_cast<int>(sizeof(CtrlParams) / sizeof(int));
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(&a.counters[0], 1);
    __syncthreads();
    const int it = s_item;
    if (it >= a.hdr->n_items) return;
    const WorkItem w = a.items[it];
    const SlotDesc *d = a.slots + w.slot;
    for (int i = threadIdx.x; i < kWords; i += BLK)
      reinterpret_cast<int *>(&s_p)[i] = reinterpret_cast<const int *>(&d->p)[i];
    __syncthreads();
    const float *x0 = a.states + 16 * w.tick;
    float *ps = d->part_sums + static_cast<size_t>(w.block) * d->tm;
    switch (d->sys) {
      case MPPI_CARTPOLE:
        rollout_block<CartPole, BLK, true>(s_p, x0, d->counter, d->U, w.block * BLK, d->S, ps, d->part + w.block,
                                           smem);
        break;
      case MPPI_CAR:
        rollout_block<Car, BLK, true>(s_p, x0, d->counter, d->U, w.block * BLK, d->S, ps, d->part + w.block, smem);
        break;
      case MPPI_QUAD:
        rollout_block<Quad, BLK, true>(s_p, x0, d->counter, d->U, w.block * BLK, d->S, ps, d->part + w.block, smem);
        break;
      case MPPI_CARTPOLE_VEL:
        rollout_block<CartPoleVel, BLK, true>(s_p, x0, d->counter, d->U, w.block * BLK, d->S, ps, d->part + w.block,
                                              smem);
        break;
      default:
        break;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kServeMergeThreads) k_serve_merge(const ServeArgs a, int max_nblk) {
  constexpr int NW = kServeMergeThreads / 32;
  extern __shared__ __align__(16) unsigned char msm[];
  float *s_scale = reinterpret_cast<float *>(msm);  // [max_nblk]
  float *s_unew = s_scale + max_nblk;                // [T*m]
  __shared__ int s_slot;
  __shared__ float s_rho[NW];
  __shared__ int s_k[NW];
  __shared__ double s_e[NW];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (;;) {
    if (tid == 0) s_slot = atomicAdd(&a.counters[1], 1);
    __syncthreads();
    const int ts = s_slot;
    if (ts >= a.hdr->n_slots) return;
    SlotDesc *d = a.slots + a.tick_slots[ts];
    const int nblk = d->nblk, TM = d->tm, m = d->p.m;
    const float inv_lambda = d->p.inv_lambda;

    float v = INFINITY;
    int idx = INT_MAX;
    for (int b = tid; b < nblk; b += kServeMergeThreads) {
      const float r = d->part[b].rho;
      const int kk = d->part[b].kstar;
      if (r < v || (r == v && kk < idx)) {
        v = r;
        idx = kk;
      }
    }
    warp_argmin(v, idx);
    if (lane == 0) {
      s_rho[warp] = v;
      s_k[warp] = idx;
    }
    __syncthreads();
    if (warp == 0) {
      float vv = lane < NW ? s_rho[lane] : INFINITY;
      int ii = lane < NW ? s_k[lane] : INT_MAX;
      warp_argmin(vv, ii);
      if (lane == 0) {
        s_rho[0] = vv;
        s_k[0] = ii;
      }
    }
    __syncthreads();
    const float rho = s_rho[0];
    double e = 0.0;
    for (int b = tid; b < nblk; b += kServeMergeThreads) {
      const float sc = merge_scale(d->part[b].rho, rho, inv_lambda);
      s_scale[b] = sc;
      e += static_cast<double>(sc) * d->part[b].eta;
    }
    e = warp_sum_d(e);
    if (lane == 0) s_e[warp] = e;
    __syncthreads();
    double eta = 0.0;
#pragma unroll
    for (int q = 0; q < NW; ++q) eta += s_e[q];
    // per output: double-FP32 sums (exact products, TwoSum) over the blocks in four
    // interleaved chains (b mod 4), combined in order; du in FP64
    for (int o = tid; o < TM; o += kServeMergeThreads) {
      DF acc[4] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
      const float *ps = d->part_sums + o;
      int b = 0;
      for (; b + 3 < nblk; b += 4) {
        const float x0 = ps[static_cast<size_t>(b) * TM], x1 = ps[static_cast<size_t>(b + 1) * TM];
        const float x2 = ps[static_cast<size_t>(b + 2) * TM], x3 = ps[static_cast<size_t>(b + 3) * TM];
        df_add_prod(acc[0], s_scale[b], x0);
        df_add_prod(acc[1], s_scale[b + 1], x1);
        df_add_prod(acc[2], s_scale[b + 2], x2);
        df_add_prod(acc[3], s_scale[b + 3], x3);
      }
      for (; b < nblk; ++b) df_add_prod(acc[b & 3], s_scale[b], ps[static_cast<size_t>(b) * TM]);
      df_add(acc[0], acc[1]);
      df_add(acc[0], acc[2]);
      df_add(acc[0], acc[3]);
      const double du = eta > 0.0 ? merge_du(acc[0], 1.0 / eta) : 0.0;
      s_unew[o] = d->U[o] + static_cast<float>(du);
    }
    __syncthreads();
    if (tid < m) a.u0_out[4 * ts + tid] = s_unew[tid];
    for (int o = tid; o < TM; o += kServeMergeThreads) d->U[o] = (o + m < TM) ? s_unew[o + m] : d->u_init[o - (TM - m)];
    if (tid == 0) {
      d->counter += 1u;
      d->rho = rho;
      d->kstar = s_k[0];
      d->eta = eta;
    }
    __syncthreads();
  }
}

}  // namespace mppi

using namespace mppi;

namespace {

int dims_of(int sys, int *n, int *m) {
  switch (sys) {
    case MPPI_CARTPOLE: *n = 4; *m = 1; return MPPI_OK;
    case MPPI_CAR: *n = 7; *m = 2; return MPPI_OK;
    case MPPI_QUAD: *n = 12; *m = 4; return MPPI_OK;
    case MPPI_CARTPOLE_VEL: *n = 4; *m = 1; return MPPI_OK;
    default: return MPPI_EINVAL;
  }
}

// relative cost of one rollout-step of each system (for heaviest-first ordering)
double step_weight(int sys) { return sys == MPPI_QUAD ? 7.0 : (sys == MPPI_CAR ? 1.0 : 0.5); }

// First-fit allocator over [0, size) with coalescing frees (offsets, 256-byte granules).
struct FreeList {
  std::map<size_t, size_t> free_;  // offset -> size
  size_t size = 0, used = 0;
  void reset(size_t n) {
    free_.clear();
    free_[0] = n;
    size = n;
    used = 0;
  }
  bool alloc(size_t bytes, size_t *off) {
    bytes = (bytes + 255) & ~static_cast<size_t>(255);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t noff = it->first + bytes;
        free_.erase(it);
        if (rest) free_[noff] = rest;
        used += bytes;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) & ~static_cast<size_t>(255);
    used -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
};

struct HostSlot {
  bool active = false;     // holds arena memory and a descriptor
  bool releasing = false;  // released while a tick in flight still uses it: freed when that retires
  int inflight = 0;        // ticks in flight that include this slot
  int sys = 0, K = 0, T = 0, m = 0, n = 0;
  size_t off = 0, bytes = 0;
  SlotDesc desc{};
};

struct EnvSlot {
  bool set = false;
  uint32_t kind = 0;
  mppi_env_map map{};
  mppi_env_forest forest{};
  float *ptr = nullptr;  // map, or cylinders followed by the nearest-cylinder grid (offsets, indices)
  int grid_nx = 0, grid_ny = 0, grid_nidx = 0;
  float grid_ox = 0.0f, grid_oy = 0.0f, grid_inv_h = 0.0f;
};

// One step request of the asynchronous interface.
enum ReqStatus { kQueued = 0, kInFlight = 1, kDone = 2, kFailed = 3 };
struct Request {
  int slot = -1;
  int status = kQueued;
  int code = MPPI_OK;  // kFailed: the status the tick failed with
  float state[16];
  float u0[4];
  std::chrono::steady_clock::time_point t_submit, t_done;
};

// A tick's buffers and CUDA graph.  Two of them alternate on the server's stream: while one
// tick runs, the next batch is filled into the other and enqueued behind it.
struct TickCtx {
  // tick buffer: header | tick_slots[max_slots] | states[max_slots][16] | items[cap]
  size_t item_cap = 0, off_slots = 0, off_states = 0, off_items = 0, tick_bytes = 0;
  unsigned char *d_tick = nullptr, *h_tick = nullptr;
  float *d_u0 = nullptr, *h_u0 = nullptr;
  int *d_counters = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t n_memset = nullptr, n_h2d = nullptr, n_roll = nullptr, n_merge = nullptr, n_d2h = nullptr;
  ServeArgs args{};
  int max_nblk_arg = 1;
  int built_gen = -1;  // shape generation the graph was built for
  cudaEvent_t start = nullptr, done = nullptr;  // around the tick on the stream (timing events)
  std::chrono::steady_clock::time_point launched;
  bool busy = false;
  uint64_t seq = 0;                 // launch order
  double work = 0.0;                // sum over its controllers of K * T * step weight
  std::vector<uint64_t> req_ids;    // asynchronous requests of the tick in flight, in tick order
  std::vector<int> slot_ids;        // slot of each
};

thread_local std::string g_server_create_error;

constexpr int kMaxEnvs = 16;
constexpr int kMaxBlockShape = 64;  // smallest BLK the tuner may choose (items are sized for it)
constexpr int kNumTickCtx = 2;
constexpr size_t kMaxOutstanding = 1u << 20;  // queued + in flight + finished-but-unread requests

}  // namespace

struct mppi_server {
  int max_slots = 0;
  size_t arena_bytes = 0;
  std::string err;
  int device = 0, num_sms = 0;
  cudaStream_t stream = nullptr;       // every tick, in order
  cudaStream_t copy_stream = nullptr;  // admission uploads (not ordered behind ticks in flight)

  char *arena = nullptr;
  FreeList fl;
  SlotDesc *d_slots = nullptr;
  std::vector<HostSlot> slots;
  EnvSlot envs[kMaxEnvs];

  int max_tm = 1, max_nblk = 1, max_nobs = 0;
  size_t max_grid = 0;  // largest nearest-cylinder grid of an admitted slot (bytes in shared memory)
  int shape_gen = 0;    // bumped whenever the kernels' shared memory or launch shape must change

  int blk = 128, ctas_per_sm = 0, variant = 1;
  TickCtx tc[kNumTickCtx];
  uint64_t launches = 0;
  int ticks = 0;
  double last_tick_ms = 0.0;

  // asynchronous interface: one scheduler thread; every field below and every host-side
  // field above is guarded by mu while the scheduler runs
  std::mutex mu;
  std::condition_variable cv_work;  // scheduler: new requests, a finished tick, stop
  std::condition_variable cv_done;  // callers of wait / reap: a tick retired
  std::thread worker;
  bool running = false, stop_req = false;
  int max_batch = 0;
  // while a tick runs, the next one is formed when the running tick is predicted to end within
  // kLaunchSlackMs (from the recent ticks' GPU time per unit of work), or once min_batch
  // requests wait, or once the oldest has waited max_wait_ms (a tick is launched at once
  // whenever the GPU has none)
  int min_batch = 1024;
  double max_wait_ms = 4.0;
  double ms_per_work = 0.0;   // GPU milliseconds per unit of tick work (EMA over retired ticks)
  std::chrono::steady_clock::time_point last_retire;
  uint64_t next_id = 0;
  std::unordered_map<uint64_t, Request> reqs;
  std::deque<uint64_t> queue;       // submitted, not yet launched (lazy: cancelled ids are skipped)
  std::deque<uint64_t> done_queue;  // finished, in completion order, for reap
  std::atomic<uint64_t> wakeups{0};  // completion callbacks, submissions, stop
  uint64_t async_ticks = 0, async_requests_done = 0;

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

#define SRV_TRY(expr)               \
  do {                              \
    const int _rc = (expr);         \
    if (_rc != MPPI_OK) return _rc; \
  } while (0)

namespace {

size_t round256(size_t b) { return (b + 255) & ~static_cast<size_t>(255); }

size_t slot_bytes(int K, int T, int m) {
  const size_t TM = static_cast<size_t>(T) * m;
  const size_t nb = (K + kMaxBlockShape - 1) / kMaxBlockShape;
  return round256(sizeof(float) * TM) + round256(sizeof(float) * kMaxM) + round256(sizeof(float) * K) +
         round256(sizeof(float) * nb * TM) + round256(sizeof(BlockPartial) * nb);
}

size_t rollout_smem(const mppi_server *s, int blk) {
  return rollout_smem_bytes(s->max_tm, 1, s->max_nobs, blk, true, false, false, s->max_grid);
}
size_t merge_smem(const mppi_server *s) { return sizeof(float) * (s->max_nblk + s->max_tm); }

// Rollout kernel variants the autotuner chooses from: block size and the register cap
// implied by a minimum number of resident blocks per SM.
struct RolloutVariant {
  int blk, minb;
  const void *fn;
};
const RolloutVariant kVariants[] = {
    {64, 8, reinterpret_cast<const void *>(k_serve_rollout<64, 8>)},
    {128, 4, reinterpret_cast<const void *>(k_serve_rollout<128, 4>)},
    {128, 6, reinterpret_cast<const void *>(k_serve_rollout<128, 6>)},
    {256, 2, reinterpret_cast<const void *>(k_serve_rollout<256, 2>)},
    {256, 3, reinterpret_cast<const void *>(k_serve_rollout<256, 3>)},
};
constexpr int kNumVariants = static_cast<int>(sizeof(kVariants) / sizeof(kVariants[0]));

void free_tick_ctx(TickCtx &t) {
  if (t.exec) cudaGraphExecDestroy(t.exec);
  if (t.graph) cudaGraphDestroy(t.graph);
  if (t.d_tick) cudaFree(t.d_tick);
  if (t.h_tick) cudaFreeHost(t.h_tick);
  if (t.d_u0) cudaFree(t.d_u0);
  if (t.h_u0) cudaFreeHost(t.h_u0);
  if (t.d_counters) cudaFree(t.d_counters);
  if (t.done) cudaEventDestroy(t.done);
  if (t.start) cudaEventDestroy(t.start);
  t = TickCtx{};
}

int init_tick_ctx(mppi_server *s, TickCtx &t) {
  SRV_TRY(s->cuda(dev_malloc(&t.d_u0, sizeof(float) * 4 * s->max_slots), "cudaMalloc(u0)"));
  SRV_TRY(s->cuda(host_alloc(&t.h_u0, sizeof(float) * 4 * s->max_slots, cudaHostAllocDefault), "cudaMallocHost(u0)"));
  SRV_TRY(s->cuda(dev_malloc(&t.d_counters, sizeof(int) * 2), "cudaMalloc(counters)"));
  SRV_TRY(s->cuda(cudaEventCreate(&t.start), "event"));
  return s->cuda(cudaEventCreate(&t.done), "event");
}

// The context's tick buffer must hold `items` work items; reallocating needs the context idle.
int ensure_tick_capacity(mppi_server *s, TickCtx &t, size_t items) {
  if (items <= t.item_cap && t.d_tick) return MPPI_OK;
  size_t cap = std::max<size_t>(t.item_cap ? t.item_cap : 4096, 4096);
  while (cap < items) cap *= 2;
  if (t.d_tick) cudaFree(t.d_tick);
  if (t.h_tick) cudaFreeHost(t.h_tick);
  t.d_tick = nullptr;
  t.h_tick = nullptr;
  t.item_cap = 0;
  t.off_slots = round256(sizeof(TickHeader));
  t.off_states = t.off_slots + round256(sizeof(int) * s->max_slots);
  t.off_items = t.off_states + round256(sizeof(float) * 16 * s->max_slots);
  t.tick_bytes = t.off_items + sizeof(WorkItem) * cap;
  SRV_TRY(s->cuda(dev_malloc(&t.d_tick, t.tick_bytes), "cudaMalloc(tick)"));
  SRV_TRY(s->cuda(host_alloc(&t.h_tick, t.tick_bytes, cudaHostAllocDefault), "cudaMallocHost(tick)"));
  std::memset(t.h_tick, 0, t.tick_bytes);
  t.item_cap = cap;
  t.built_gen = -1;
  return MPPI_OK;
}

// (Re)build the context's graph: memset queue counters -> H2D tick buffer -> rollout ->
// merge -> D2H u_0.  Needs the context idle.
int build_graph(mppi_server *s, TickCtx &t) {
  if (t.exec) cudaGraphExecDestroy(t.exec);
  if (t.graph) cudaGraphDestroy(t.graph);
  t.exec = nullptr;
  t.graph = nullptr;
  if (s->variant < 0 || s->variant >= kNumVariants) return s->fail(MPPI_EINVAL, "bad kernel variant");
  const void *rfn = kVariants[s->variant].fn;
  s->blk = kVariants[s->variant].blk;
  const size_t rsm = rollout_smem(s, s->blk), msm = merge_smem(s);
  SRV_TRY(s->cuda(cudaFuncSetAttribute(rfn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(rsm)),
                  "rollout smem attribute"));
  SRV_TRY(s->cuda(cudaFuncSetAttribute(reinterpret_cast<const void *>(k_serve_merge),
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(msm)),
                  "merge smem attribute"));
  int occ = 0, mocc = 0;
  SRV_TRY(s->cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, rfn, s->blk, rsm), "occupancy"));
  SRV_TRY(s->cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&mocc, reinterpret_cast<const void *>(k_serve_merge),
                                                                kServeMergeThreads, msm),
                  "occupancy"));
  if (occ < 1 || mocc < 1) return s->fail(MPPI_EINVAL, "serving kernels do not fit on an SM");
  const int cps = s->ctas_per_sm > 0 ? std::min(s->ctas_per_sm, occ) : occ;

  ServeArgs &a = t.args;
  a.slots = s->d_slots;
  a.hdr = reinterpret_cast<const TickHeader *>(t.d_tick);
  a.tick_slots = reinterpret_cast<const int *>(t.d_tick + t.off_slots);
  a.states = reinterpret_cast<const float *>(t.d_tick + t.off_states);
  a.items = reinterpret_cast<const WorkItem *>(t.d_tick + t.off_items);
  a.u0_out = t.d_u0;
  a.counters = t.d_counters;
  t.max_nblk_arg = s->max_nblk;

  SRV_TRY(s->cuda(cudaGraphCreate(&t.graph, 0), "graph create"));
  cudaMemsetParams mp{};
  mp.dst = t.d_counters;
  mp.value = 0;
  mp.elementSize = 4;
  mp.width = 2;
  mp.height = 1;
  mp.pitch = 0;
  SRV_TRY(s->cuda(cudaGraphAddMemsetNode(&t.n_memset, t.graph, nullptr, 0, &mp), "memset node"));
  SRV_TRY(s->cuda(cudaGraphAddMemcpyNode1D(&t.n_h2d, t.graph, &t.n_memset, 1, t.d_tick, t.h_tick, t.off_items,
                                           cudaMemcpyHostToDevice),
                  "h2d node"));
  void *rargs[] = {&t.args};
  cudaKernelNodeParams kp{};
  kp.func = const_cast<void *>(rfn);
  kp.gridDim = dim3(s->num_sms * cps);
  kp.blockDim = dim3(s->blk);
  kp.sharedMemBytes = static_cast<unsigned>(rsm);
  kp.kernelParams = rargs;
  SRV_TRY(s->cuda(cudaGraphAddKernelNode(&t.n_roll, t.graph, &t.n_h2d, 1, &kp), "rollout node"));
  void *margs[] = {&t.args, &t.max_nblk_arg};
  cudaKernelNodeParams km{};
  km.func = reinterpret_cast<void *>(k_serve_merge);
  km.gridDim = dim3(s->num_sms * std::min(mocc, 4));
  km.blockDim = dim3(kServeMergeThreads);
  km.sharedMemBytes = static_cast<unsigned>(msm);
  km.kernelParams = margs;
  SRV_TRY(s->cuda(cudaGraphAddKernelNode(&t.n_merge, t.graph, &t.n_roll, 1, &km), "merge node"));
  SRV_TRY(s->cuda(cudaGraphAddMemcpyNode1D(&t.n_d2h, t.graph, &t.n_merge, 1, t.h_u0, t.d_u0, sizeof(float) * 4,
                                           cudaMemcpyDeviceToHost),
                  "d2h node"));
  SRV_TRY(s->cuda(cudaGraphInstantiate(&t.exec, t.graph, 0), "graph instantiate"));
  s->ctas_per_sm = cps;
  t.built_gen = s->shape_gen;
  return MPPI_OK;
}

// Fill an idle context with one tick of the n listed slots (states [n][16]) and launch it on
// the server stream, followed by the context's completion event.  No host synchronisation.
int launch_tick(mppi_server *s, TickCtx &t, int n, const int *slot_ids, const float *states) {
  // work items, heaviest slots first
  std::vector<int> order(n);
  size_t n_items = 0;
  for (int q = 0; q < n; ++q) {
    order[q] = q;
    const HostSlot &h = s->slots[slot_ids[q]];
    n_items += (h.K + s->blk - 1) / s->blk;
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    const HostSlot &x = s->slots[slot_ids[a]], &y = s->slots[slot_ids[b]];
    return step_weight(x.sys) * x.T > step_weight(y.sys) * y.T;
  });
  t.work = 0.0;
  for (int q = 0; q < n; ++q) {
    const HostSlot &h = s->slots[slot_ids[q]];
    t.work += step_weight(h.sys) * static_cast<double>(h.K) * h.T;
  }
  SRV_TRY(ensure_tick_capacity(s, t, n_items));
  if (t.built_gen != s->shape_gen) SRV_TRY(build_graph(s, t));

  TickHeader *hdr = reinterpret_cast<TickHeader *>(t.h_tick);
  int *ts = reinterpret_cast<int *>(t.h_tick + t.off_slots);
  float *st = reinterpret_cast<float *>(t.h_tick + t.off_states);
  WorkItem *it = reinterpret_cast<WorkItem *>(t.h_tick + t.off_items);
  size_t k = 0;
  for (int q = 0; q < n; ++q) {
    const int i = order[q];
    const HostSlot &h = s->slots[slot_ids[i]];
    const int nb = (h.K + s->blk - 1) / s->blk;
    for (int b = 0; b < nb; ++b) it[k++] = WorkItem{slot_ids[i], i, b, 0};
  }
  for (int q = 0; q < n; ++q) {
    ts[q] = slot_ids[q];
    std::memcpy(st + 16 * q, states + 16 * q, sizeof(float) * 16);
  }
  hdr->n_items = static_cast<int>(n_items);
  hdr->n_slots = n;
  SRV_TRY(s->cuda(cudaGraphExecMemcpyNodeSetParams1D(t.exec, t.n_h2d, t.d_tick, t.h_tick,
                                                     t.off_items + sizeof(WorkItem) * n_items, cudaMemcpyHostToDevice),
                  "h2d update"));
  SRV_TRY(s->cuda(cudaGraphExecMemcpyNodeSetParams1D(t.exec, t.n_d2h, t.h_u0, t.d_u0, sizeof(float) * 4 * n,
                                                     cudaMemcpyDeviceToHost),
                  "d2h update"));
  SRV_TRY(s->cuda(cudaEventRecord(t.start, s->stream), "event record"));
  SRV_TRY(s->cuda(cudaGraphLaunch(t.exec, s->stream), "graph launch"));
  SRV_TRY(s->cuda(cudaEventRecord(t.done, s->stream), "event record"));
  t.seq = ++s->launches;
  t.launched = std::chrono::steady_clock::now();
  return MPPI_OK;
}

// Block shape changed since admission (autotune): refresh (nblk, blk) of the listed slots.
int refresh_shapes(mppi_server *s, int n, const int *slot_ids) {
  for (int q = 0; q < n; ++q) {
    HostSlot &h = s->slots[slot_ids[q]];
    const int nb = (h.K + s->blk - 1) / s->blk;
    if (h.desc.nblk != nb || h.desc.blk != s->blk) {
      h.desc.nblk = nb;
      h.desc.blk = s->blk;
      // only these two fields: the rest of the device descriptor (e.g. the counter) is device-owned
      SRV_TRY(s->cuda(cudaMemcpyAsync(&s->d_slots[slot_ids[q]].nblk, &h.desc.nblk, 2 * sizeof(int),
                                      cudaMemcpyHostToDevice, s->stream),
                      "slot shape"));
      SRV_TRY(s->cuda(cudaStreamSynchronize(s->stream), "sync"));
    }
  }
  return MPPI_OK;
}

// Synchronous tick on context 0 (the scheduler is not running).
int run_tick(mppi_server *s, int n, const int *slot_ids, const float *states, float *u0_out) {
  const NvtxRange range("server tick (serve rollout, serve merge)");
  SRV_TRY(refresh_shapes(s, n, slot_ids));
  TickCtx &t = s->tc[0];
  const auto t0 = std::chrono::steady_clock::now();
  SRV_TRY(launch_tick(s, t, n, slot_ids, states));
  SRV_TRY(s->cuda(cudaStreamSynchronize(s->stream), "tick sync"));
  s->last_tick_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  s->ticks += 1;
  if (u0_out) std::memcpy(u0_out, t.h_u0, sizeof(float) * 4 * n);
  return MPPI_OK;
}

int check_slots(mppi_server *s, int n, const int *slot_ids) {
  if (n < 0 || n > s->max_slots || (n > 0 && !slot_ids)) return s->fail(MPPI_EINVAL, "bad slot list");
  std::vector<char> seen(s->max_slots, 0);
  for (int q = 0; q < n; ++q) {
    const int i = slot_ids[q];
    if (i < 0 || i >= s->max_slots || !s->slots[i].active || s->slots[i].releasing)
      return s->fail(MPPI_EINVAL, "slot %d is not active", i);
    if (seen[i]) return s->fail(MPPI_EINVAL, "slot %d listed twice", i);
    seen[i] = 1;
  }
  return MPPI_OK;
}

void free_slot(mppi_server *s, int slot) {
  HostSlot &h = s->slots[slot];
  s->fl.release(h.off, h.bytes);
  h.active = false;
  h.releasing = false;
  h.inflight = 0;
}

// ---- the scheduler (continuous batching) ----------------------------------------------

void CUDART_CB on_tick_done(void *p) {
  // runs on a CUDA driver thread: no CUDA calls and no lock (a caller holding the lock may be
  // waiting on this very stream); a counter and a wake-up only
  auto *s = static_cast<mppi_server *>(p);
  s->wakeups.fetch_add(1, std::memory_order_release);
  s->cv_work.notify_all();
}

// Publish the results of finished ticks, oldest first (caller holds mu).
void retire(mppi_server *s) {
  const NvtxRange range("server: retire finished ticks");
  for (;;) {
    TickCtx *oldest = nullptr;
    for (auto &t : s->tc)
      if (t.busy && (!oldest || t.seq < oldest->seq)) oldest = &t;
    if (!oldest) return;
    const cudaError_t q = cudaEventQuery(oldest->done);
    if (q == cudaErrorNotReady) return;
    int code = MPPI_OK;
    if (q != cudaSuccess) {
      code = s->cuda(q, "tick");
    }
    TickCtx &t = *oldest;
    float gpu_ms = 0.0f;
    if (code == MPPI_OK && cudaEventElapsedTime(&gpu_ms, t.start, t.done) == cudaSuccess && t.work > 0.0) {
      const double r = gpu_ms / t.work;
      s->ms_per_work = s->ms_per_work > 0.0 ? 0.8 * s->ms_per_work + 0.2 * r : r;
    }
    cudaGetLastError();
    s->last_retire = std::chrono::steady_clock::now();
    for (size_t i = 0; i < t.req_ids.size(); ++i) {
      HostSlot &h = s->slots[t.slot_ids[i]];
      h.inflight -= 1;
      if (h.releasing && h.inflight == 0) free_slot(s, t.slot_ids[i]);
      auto r = s->reqs.find(t.req_ids[i]);
      if (r == s->reqs.end()) continue;  // cancelled while in flight: the result is dropped
      r->second.t_done = s->last_retire;
      if (code == MPPI_OK) {
        std::memcpy(r->second.u0, t.h_u0 + 4 * i, sizeof(float) * 4);
        r->second.status = kDone;
      } else {
        r->second.status = kFailed;
        r->second.code = code;
      }
      s->done_queue.push_back(t.req_ids[i]);
      s->async_requests_done += 1;
    }
    t.req_ids.clear();
    t.slot_ids.clear();
    t.busy = false;
    s->async_ticks += 1;
    s->ticks += 1;
    s->cv_done.notify_all();
  }
}

constexpr double kLaunchSlackMs = 0.25;  // form the next tick this long before the running one ends

// Predicted milliseconds until the tick on the GPU finishes (caller holds mu): its work times
// the recent GPU time per unit of work, counted from when it can have started (its launch, or
// the retirement of the tick before it); 0 without a prediction.
double running_tick_remaining_ms(mppi_server *s) {
  const TickCtx *run = nullptr;
  for (const auto &t : s->tc)
    if (t.busy && (!run || t.seq < run->seq)) run = &t;
  if (!run || s->ms_per_work <= 0.0) return 0.0;
  const auto began = std::max(run->launched, s->last_retire);
  const double elapsed = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - began).count();
  return std::max(0.0, run->work * s->ms_per_work - elapsed);
}

// Drop cancelled requests from the front of the queue; the oldest live request's age in ms
// (caller holds mu), or -1 when nothing is queued.
double oldest_wait_ms(mppi_server *s) {
  while (!s->queue.empty()) {
    auto r = s->reqs.find(s->queue.front());
    if (r != s->reqs.end() && r->second.status == kQueued)
      return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - r->second.t_submit).count();
    s->queue.pop_front();
  }
  return -1.0;
}

// Launch the queued requests (at most one per slot, up to max_batch) on an idle context
// (caller holds mu).  With a tick already on the GPU the next one is only formed once
// min_batch requests wait or the oldest has waited max_wait_ms, so that it batches what
// arrives meanwhile.  Returns true when a tick was launched.
bool launch_queued(mppi_server *s) {
  const NvtxRange range("server: batch queued requests and launch a tick");
  TickCtx *idle = nullptr;
  bool busy = false;
  for (auto &t : s->tc) {
    if (!t.busy && !idle) idle = &t;
    busy = busy || t.busy;
  }
  if (!idle) return false;
  const double age = oldest_wait_ms(s);
  if (age < 0.0) return false;
  if (busy && static_cast<int>(s->queue.size()) < s->min_batch && age < s->max_wait_ms &&
      running_tick_remaining_ms(s) > kLaunchSlackMs)
    return false;
  std::vector<uint64_t> ids;
  std::vector<int> slot_ids;
  std::vector<float> states;
  std::vector<char> taken(s->max_slots, 0);
  std::deque<uint64_t> keep;
  const size_t cap = s->max_batch > 0 ? static_cast<size_t>(s->max_batch) : static_cast<size_t>(s->max_slots);
  while (!s->queue.empty()) {
    const uint64_t id = s->queue.front();
    s->queue.pop_front();
    auto r = s->reqs.find(id);
    if (r == s->reqs.end() || r->second.status != kQueued) continue;  // cancelled
    const int slot = r->second.slot;
    if (taken[slot] || ids.size() >= cap) {
      keep.push_back(id);  // one step per slot and tick: the next tick takes it
      continue;
    }
    taken[slot] = 1;
    ids.push_back(id);
    slot_ids.push_back(slot);
    states.insert(states.end(), r->second.state, r->second.state + 16);
  }
  s->queue.swap(keep);
  if (ids.empty()) return false;
  const int rc = launch_tick(s, *idle, static_cast<int>(ids.size()), slot_ids.data(), states.data());
  if (rc != MPPI_OK) {
    for (uint64_t id : ids) {
      Request &r = s->reqs[id];
      r.status = kFailed;
      r.code = rc;
      s->done_queue.push_back(id);
    }
    s->cv_done.notify_all();
    return false;
  }
  cudaLaunchHostFunc(s->stream, on_tick_done, s);
  for (size_t i = 0; i < ids.size(); ++i) {
    s->reqs[ids[i]].status = kInFlight;
    s->slots[slot_ids[i]].inflight += 1;
  }
  idle->req_ids = std::move(ids);
  idle->slot_ids = std::move(slot_ids);
  idle->busy = true;
  return true;
}

void scheduler(mppi_server *s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    retire(s);
    while (launch_queued(s)) {
    }
    bool busy = false;
    for (auto &t : s->tc) busy = busy || t.busy;
    if (s->stop_req && !busy && s->queue.empty()) break;
    if (busy) {
      // woken by the completion callback, a submission or the stop; the timeout bounds a
      // wake-up lost between the check above and the wait, and the batching delay
      const uint64_t seen = s->wakeups.load(std::memory_order_acquire);
      double wait_us = 500.0;
      const double age = oldest_wait_ms(s);
      if (age >= 0.0) {
        wait_us = std::min(wait_us, 1e3 * (s->max_wait_ms - age));
        const double rem = running_tick_remaining_ms(s);
        if (rem > kLaunchSlackMs) wait_us = std::min(wait_us, 1e3 * (rem - kLaunchSlackMs));
        wait_us = std::max(20.0, wait_us);
      }
      s->cv_work.wait_for(lk, std::chrono::microseconds(static_cast<int64_t>(wait_us)),
                          [&] { return s->wakeups.load(std::memory_order_acquire) != seen; });
    } else {
      s->cv_work.wait(lk, [&] { return s->stop_req || !s->queue.empty(); });
    }
  }
}

// Stop the scheduler after it has finished everything submitted (caller does not hold mu).
void stop_scheduler(mppi_server *s) {
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (!s->running) return;
    s->stop_req = true;
    s->wakeups.fetch_add(1, std::memory_order_release);
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  std::lock_guard<std::mutex> lk(s->mu);
  s->running = false;
  s->stop_req = false;
}

}  // namespace

extern "C" {

const char *mppi_server_last_error(mppi_server *s) { return s ? s->err.c_str() : g_server_create_error.c_str(); }

int mppi_server_create(int max_slots, size_t arena_bytes, mppi_server **out) {
  if (!out) return MPPI_EINVAL;
  *out = nullptr;
  if (max_slots < 1 || max_slots > 4096 || arena_bytes < 4096) return MPPI_EINVAL;
  mppi_server *s = new (std::nothrow) mppi_server();
  if (!s) return MPPI_ENOMEM;
  s->max_slots = max_slots;
  s->arena_bytes = arena_bytes;
  s->slots.resize(max_slots);
  int rc = s->cuda(cudaGetDevice(&s->device), "cudaGetDevice");
  if (rc == MPPI_OK) rc = s->cuda(cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device), "sms");
  if (rc == MPPI_OK) rc = s->cuda(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking), "stream");
  if (rc == MPPI_OK) rc = s->cuda(cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking), "copy stream");
  if (rc == MPPI_OK) rc = s->cuda(dev_malloc(&s->arena, arena_bytes), "cudaMalloc(arena)");
  if (rc == MPPI_OK) rc = s->cuda(dev_malloc(&s->d_slots, sizeof(SlotDesc) * max_slots), "cudaMalloc(slots)");
  if (rc == MPPI_OK) rc = s->cuda(cudaMemset(s->d_slots, 0, sizeof(SlotDesc) * max_slots), "memset(slots)");
  for (int i = 0; i < kNumTickCtx && rc == MPPI_OK; ++i) {
    rc = init_tick_ctx(s, s->tc[i]);
    if (rc == MPPI_OK) rc = ensure_tick_capacity(s, s->tc[i], 4096);
  }
  if (rc != MPPI_OK) {
    g_server_create_error = s->err;
    mppi_server_destroy(s);
    return rc;
  }
  s->fl.reset(arena_bytes);
  *out = s;
  return MPPI_OK;
}

int mppi_server_destroy(mppi_server *s) {
  if (!s) return MPPI_OK;
  stop_scheduler(s);
  if (s->stream) cudaStreamSynchronize(s->stream);
  for (auto &t : s->tc) free_tick_ctx(t);
  for (auto &e : s->envs)
    if (e.ptr) cudaFree(e.ptr);
  if (s->arena) cudaFree(s->arena);
  if (s->d_slots) cudaFree(s->d_slots);
  if (s->stream) cudaStreamDestroy(s->stream);
  if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
  delete s;
  return MPPI_OK;
}

int mppi_server_set_env(mppi_server *s, int env_id, const void *blob, size_t bytes) {
  if (!s || !blob || env_id < 0 || env_id >= kMaxEnvs || bytes < 8) return MPPI_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  for (const auto &h : s->slots)
    if (h.active && (h.desc.p.map || h.desc.p.obs) && s->envs[env_id].ptr &&
        (h.desc.p.map == s->envs[env_id].ptr || h.desc.p.obs == s->envs[env_id].ptr))
      return s->fail(MPPI_ESTATE, "env %d is in use by an active slot", env_id);
  EnvSlot e;
  std::memcpy(&e.kind, blob, 4);
  size_t payload = 0;
  if (e.kind == MPPI_ENV_MAP) {
    if (bytes < sizeof(mppi_env_map)) return s->fail(MPPI_EINVAL, "map header truncated");
    std::memcpy(&e.map, blob, sizeof e.map);
    if (e.map.width < 2 || e.map.height < 2 || e.map.width > 16384 || e.map.height > 16384 || !(e.map.cell > 0.0f))
      return s->fail(MPPI_EINVAL, "bad map header");
    payload = sizeof(float) * static_cast<size_t>(e.map.width) * e.map.height;
    if (bytes != sizeof e.map + payload) return s->fail(MPPI_EINVAL, "map blob size mismatch");
  } else if (e.kind == MPPI_ENV_FOREST) {
    if (bytes < sizeof(mppi_env_forest)) return s->fail(MPPI_EINVAL, "forest header truncated");
    std::memcpy(&e.forest, blob, sizeof e.forest);
    if (e.forest.n_obstacles < 0 || e.forest.n_obstacles > 256) return s->fail(MPPI_EINVAL, "bad forest header");
    payload = sizeof(float) * 3 * static_cast<size_t>(e.forest.n_obstacles);
    if (bytes != sizeof e.forest + payload) return s->fail(MPPI_EINVAL, "forest blob size mismatch");
  } else {
    return s->fail(MPPI_EINVAL, "unknown env kind");
  }
  const char *src = static_cast<const char *>(blob) + (e.kind == MPPI_ENV_MAP ? sizeof e.map : sizeof e.forest);
  std::vector<char> forest;  // cylinders + grid
  ForestGrid grid;
  if (e.kind == MPPI_ENV_FOREST &&
      build_forest_grid(reinterpret_cast<const float *>(src), e.forest.n_obstacles, grid)) {
    e.grid_nx = grid.nx;
    e.grid_ny = grid.ny;
    e.grid_nidx = static_cast<int>(grid.idx.size());
    e.grid_ox = grid.ox;
    e.grid_oy = grid.oy;
    e.grid_inv_h = grid.inv_h;
    forest.assign(src, src + payload);
    forest.resize(payload + grid.bytes());
    std::memcpy(forest.data() + payload, grid.off.data(), sizeof(uint16_t) * grid.off.size());
    std::memcpy(forest.data() + payload + sizeof(uint16_t) * grid.off.size(), grid.idx.data(), grid.idx.size());
    src = forest.data();
    payload = forest.size();
  }
  // no slot uses this env (checked above), so nothing in flight reads the old payload
  if (s->envs[env_id].ptr) cudaFree(s->envs[env_id].ptr);
  s->envs[env_id].ptr = nullptr;
  s->envs[env_id].set = false;
  SRV_TRY(s->cuda(cudaMalloc(&e.ptr, std::max<size_t>(payload, 16)), "cudaMalloc(env)"));
  if (payload) {
    int rc = s->cuda(cudaMemcpyAsync(e.ptr, src, payload, cudaMemcpyHostToDevice, s->copy_stream), "env copy");
    if (rc == MPPI_OK) rc = s->cuda(cudaStreamSynchronize(s->copy_stream), "env copy sync");
    if (rc != MPPI_OK) {
      cudaFree(e.ptr);
      return rc;
    }
  }
  e.set = true;
  s->envs[env_id] = e;
  return MPPI_OK;
}

int mppi_server_admit(mppi_server *s, const mppi_slot_config *c, int *slot_out) {
  if (!s || !c || !slot_out) return MPPI_EINVAL;
  *slot_out = -1;
  std::lock_guard<std::mutex> lk(s->mu);
  int n = 0, m = 0;
  if (dims_of(c->system, &n, &m) != MPPI_OK) return s->fail(MPPI_EINVAL, "unknown system %d", c->system);
  if (c->K < 1 || c->K > kServeMaxK || c->T < 1 || c->T > kServeMaxT)
    return s->fail(MPPI_EINVAL, "K in [1, %d] and T in [1, %d] for serving", kServeMaxK, kServeMaxT);
  float Lnu[kMaxM * kMaxM], Rf[kMaxM * kMaxM];
  if (const char *why = host::control_constants(m, c->dt, c->nu, c->lambda, c->Sigma, c->has_R ? c->R : nullptr, Lnu,
                                                Rf))
    return s->fail(MPPI_EINVAL, "%s", why);
  CtrlParams p{};
  p.K = c->K;
  p.T = c->T;
  p.m = m;
  p.n = n;
  p.dt = c->dt;
  p.nu = c->nu;
  p.lambda = c->lambda;
  p.inv_lambda = 1.0f / c->lambda;
  p.is_du = 0.5f * static_cast<float>(1.0 - 1.0 / static_cast<double>(c->nu));
  p.key_lo = static_cast<uint32_t>(c->seed & 0xffffffffu);
  p.key_hi = static_cast<uint32_t>(c->seed >> 32);
  p.gid = c->gid;
  p.map_w = p.map_h = 2;
  p.map_inv_cell = 1.0f;
  for (int i = 0; i < m * m; ++i) {
    p.Lnu[i] = Lnu[i];
    p.R[i] = Rf[i];
  }
  if (c->system == MPPI_CAR || c->system == MPPI_QUAD) {
    if (c->env_id < 0 || c->env_id >= kMaxEnvs || !s->envs[c->env_id].set)
      return s->fail(MPPI_EINVAL, "env %d is not set", c->env_id);
    const EnvSlot &e = s->envs[c->env_id];
    if (c->system == MPPI_CAR) {
      if (e.kind != MPPI_ENV_MAP) return s->fail(MPPI_EINVAL, "car needs a map env");
      p.map = e.ptr;
      p.map_w = e.map.width;
      p.map_h = e.map.height;
      p.map_ox = e.map.origin_x;
      p.map_oy = e.map.origin_y;
      p.map_inv_cell = 1.0f / e.map.cell;
    } else {
      if (e.kind != MPPI_ENV_FOREST) return s->fail(MPPI_EINVAL, "quadrotor needs a forest env");
      p.obs = e.ptr;
      p.n_obs = e.forest.n_obstacles;
      for (int i = 0; i < 3; ++i) p.goal[i] = e.forest.goal[i];
      p.grid_nx = e.grid_nx;
      p.grid_ny = e.grid_ny;
      p.grid_nidx = e.grid_nidx;
      p.grid_ox = e.grid_ox;
      p.grid_oy = e.grid_oy;
      p.grid_inv_h = e.grid_inv_h;
      if (e.grid_nx > 0) {
        p.grid_off = reinterpret_cast<const unsigned short *>(e.ptr + 3 * static_cast<size_t>(p.n_obs));
        p.grid_idx = reinterpret_cast<const unsigned char *>(p.grid_off + (static_cast<size_t>(e.grid_nx) * e.grid_ny + 1));
      }
    }
  }
  int slot = -1;
  for (int i = 0; i < s->max_slots; ++i)
    if (!s->slots[i].active) {
      slot = i;
      break;
    }
  if (slot < 0) return s->fail(MPPI_EBUSY, "no free slot");
  const size_t bytes = slot_bytes(c->K, c->T, m);
  size_t off = 0;
  if (!s->fl.alloc(bytes, &off)) return s->fail(MPPI_EBUSY, "arena full (%zu of %zu bytes used)", s->fl.used, s->fl.size);

  HostSlot &h = s->slots[slot];
  h.active = true;
  h.releasing = false;
  h.inflight = 0;
  h.sys = c->system;
  h.K = c->K;
  h.T = c->T;
  h.m = m;
  h.n = n;
  h.off = off;
  h.bytes = bytes;
  const size_t TM = static_cast<size_t>(c->T) * m;
  const size_t nb = (c->K + kMaxBlockShape - 1) / kMaxBlockShape;
  char *base = s->arena + off;
  SlotDesc d{};
  d.p = p;
  d.sys = c->system;
  d.tm = static_cast<int>(TM);
  d.blk = s->blk;
  d.nblk = (c->K + s->blk - 1) / s->blk;
  d.U = reinterpret_cast<float *>(base);
  base += round256(sizeof(float) * TM);
  d.u_init = reinterpret_cast<float *>(base);
  base += round256(sizeof(float) * kMaxM);
  d.S = reinterpret_cast<float *>(base);
  base += round256(sizeof(float) * c->K);
  d.part_sums = reinterpret_cast<float *>(base);
  base += round256(sizeof(float) * nb * TM);
  d.part = reinterpret_cast<BlockPartial *>(base);
  d.counter = c->counter;
  h.desc = d;

  // uploads on the copy stream: they touch only this slot's memory and descriptor, which no
  // tick in flight reads, so admission does not wait for the ticks on the server stream
  std::vector<float> U0(TM);
  for (size_t i = 0; i < TM; ++i) U0[i] = c->u_init[i % m];
  int rc = s->cuda(cudaMemcpyAsync(d.U, U0.data(), sizeof(float) * TM, cudaMemcpyHostToDevice, s->copy_stream), "U init");
  if (rc == MPPI_OK)
    rc = s->cuda(cudaMemcpyAsync(d.u_init, c->u_init, sizeof(float) * m, cudaMemcpyHostToDevice, s->copy_stream),
                 "u_init");
  if (rc == MPPI_OK)
    rc = s->cuda(cudaMemcpyAsync(s->d_slots + slot, &d, sizeof d, cudaMemcpyHostToDevice, s->copy_stream), "slot desc");
  if (rc == MPPI_OK) rc = s->cuda(cudaStreamSynchronize(s->copy_stream), "admission sync");
  if (rc != MPPI_OK) {
    s->fl.release(off, bytes);
    h.active = false;
    return rc;
  }
  // shapes the persistent kernels' shared memory must cover
  const int nblk_max = (c->K + kMaxBlockShape - 1) / kMaxBlockShape;
  if (static_cast<int>(TM) > s->max_tm || nblk_max > s->max_nblk || p.n_obs > s->max_nobs ||
      quad_grid_bytes(p) > s->max_grid) {
    s->max_tm = std::max(s->max_tm, static_cast<int>(TM));
    s->max_nblk = std::max(s->max_nblk, nblk_max);
    s->max_nobs = std::max(s->max_nobs, p.n_obs);
    s->max_grid = std::max(s->max_grid, quad_grid_bytes(p));
    s->shape_gen += 1;  // contexts rebuild their graphs when next idle
  }
  *slot_out = slot;
  return MPPI_OK;
}

int mppi_server_release(mppi_server *s, int slot) {
  if (!s) return MPPI_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (slot < 0 || slot >= s->max_slots || !s->slots[slot].active || s->slots[slot].releasing)
    return s->fail(MPPI_EINVAL, "slot %d is not active", slot);
  HostSlot &h = s->slots[slot];
  // queued requests of the slot are cancelled (forgotten); a tick in flight finishes first
  for (auto it = s->reqs.begin(); it != s->reqs.end();)
    it = (it->second.slot == slot && it->second.status == kQueued) ? s->reqs.erase(it) : std::next(it);
  if (h.inflight > 0) {
    h.releasing = true;  // the scheduler frees it when the last tick using it retires
    return MPPI_OK;
  }
  if (!s->running) SRV_TRY(s->cuda(cudaStreamSynchronize(s->stream), "sync"));
  free_slot(s, slot);
  return MPPI_OK;
}

// Controls and results of a slot: copied on the server stream (after every tick already
// enqueued; the scheduler cannot enqueue another while the lock is held) and waited for.
int mppi_server_set_controls(mppi_server *s, int slot, const float *U) {
  if (!s || !U) return MPPI_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (slot < 0 || slot >= s->max_slots || !s->slots[slot].active || s->slots[slot].releasing) return MPPI_EINVAL;
  const HostSlot &h = s->slots[slot];
  SRV_TRY(s->cuda(cudaMemcpyAsync(h.desc.U, U, sizeof(float) * h.T * h.m, cudaMemcpyHostToDevice, s->stream), "U copy"));
  return s->cuda(cudaStreamSynchronize(s->stream), "sync");
}

int mppi_server_get_controls(mppi_server *s, int slot, float *U) {
  if (!s || !U) return MPPI_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (slot < 0 || slot >= s->max_slots || !s->slots[slot].active || s->slots[slot].releasing) return MPPI_EINVAL;
  const HostSlot &h = s->slots[slot];
  SRV_TRY(s->cuda(cudaMemcpyAsync(U, h.desc.U, sizeof(float) * h.T * h.m, cudaMemcpyDeviceToHost, s->stream), "U copy"));
  return s->cuda(cudaStreamSynchronize(s->stream), "sync");
}

int mppi_server_get_debug(mppi_server *s, int slot, float *S, int *argmin, double *eta) {
  if (!s) return MPPI_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (slot < 0 || slot >= s->max_slots || !s->slots[slot].active || s->slots[slot].releasing) return MPPI_EINVAL;
  const HostSlot &h = s->slots[slot];
  SlotDesc d;
  SRV_TRY(s->cuda(cudaMemcpyAsync(&d, s->d_slots + slot, sizeof d, cudaMemcpyDeviceToHost, s->stream), "slot desc"));
  if (S) SRV_TRY(s->cuda(cudaMemcpyAsync(S, h.desc.S, sizeof(float) * h.K, cudaMemcpyDeviceToHost, s->stream), "S copy"));
  SRV_TRY(s->cuda(cudaStreamSynchronize(s->stream), "sync"));
  if (argmin) *argmin = d.kstar;
  if (eta) *eta = d.eta;
  return MPPI_OK;
}

int mppi_server_tick(mppi_server *s, int n, const int *slot_ids, const float *states, float *u0_out) {
  if (!s || (n > 0 && !states)) return MPPI_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->running) return s->fail(MPPI_ESTATE, "the scheduler is running: use submit / poll");
  SRV_TRY(check_slots(s, n, slot_ids));
  if (n == 0) return MPPI_OK;
  return run_tick(s, n, slot_ids, states, u0_out);
}

int mppi_server_autotune(mppi_server *s, int n, const int *slot_ids, const float *states) {
  if (!s || n < 1 || !states) return MPPI_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->running) return s->fail(MPPI_ESTATE, "the scheduler is running: autotune before mppi_server_start");
  SRV_TRY(check_slots(s, n, slot_ids));
  // snapshot the listed slots (controls + descriptors) so tuning leaves no trace
  std::vector<std::vector<float>> U(n);
  std::vector<SlotDesc> D(s->max_slots);
  SRV_TRY(s->cuda(cudaStreamSynchronize(s->stream), "sync"));
  SRV_TRY(s->cuda(cudaMemcpy(D.data(), s->d_slots, sizeof(SlotDesc) * s->max_slots, cudaMemcpyDeviceToHost), "snap"));
  for (int q = 0; q < n; ++q) {
    const HostSlot &h = s->slots[slot_ids[q]];
    U[q].resize(static_cast<size_t>(h.T) * h.m);
    SRV_TRY(s->cuda(cudaMemcpy(U[q].data(), h.desc.U, sizeof(float) * U[q].size(), cudaMemcpyDeviceToHost), "U snap"));
  }
  auto restore = [&]() -> int {
    for (int q = 0; q < n; ++q) {
      const HostSlot &h = s->slots[slot_ids[q]];
      SRV_TRY(s->cuda(cudaMemcpy(h.desc.U, U[q].data(), sizeof(float) * U[q].size(), cudaMemcpyHostToDevice), "U restore"));
    }
    return s->cuda(cudaMemcpy(s->d_slots, D.data(), sizeof(SlotDesc) * s->max_slots, cudaMemcpyHostToDevice),
                   "restore");
  };
  double best = 1e30;
  int best_var = s->variant, best_cps = 0;
  for (int bi = 0; bi < kNumVariants; ++bi) {
    for (int cps_try = 0; cps_try < 2; ++cps_try) {
      s->variant = bi;
      s->ctas_per_sm = 0;
      s->shape_gen += 1;
      SRV_TRY(build_graph(s, s->tc[0]));
      const int occ = s->ctas_per_sm;
      if (cps_try == 1) {
        if (occ < 2) continue;
        s->ctas_per_sm = occ / 2;
        s->shape_gen += 1;
        SRV_TRY(build_graph(s, s->tc[0]));
      }
      SRV_TRY(run_tick(s, n, slot_ids, states, nullptr));  // warm-up
      double t = 0.0;
      for (int r = 0; r < 3; ++r) {
        SRV_TRY(run_tick(s, n, slot_ids, states, nullptr));
        t += s->last_tick_ms;
      }
      SRV_TRY(restore());
      // the restored descriptors carry the admission-time block shape: refresh on the next tick
      for (int q = 0; q < n; ++q) s->slots[slot_ids[q]].desc.blk = -1;
      if (t < best) {
        best = t;
        best_var = s->variant;
        best_cps = s->ctas_per_sm;
      }
    }
  }
  s->variant = best_var;
  s->blk = kVariants[best_var].blk;
  s->ctas_per_sm = best_cps;
  s->shape_gen += 1;
  for (int i = 0; i < s->max_slots; ++i)
    if (s->slots[i].active) s->slots[i].desc.blk = -1;  // force the shape refresh on the next tick
  // every active slot takes the tuned block shape now, so that the scheduler (which never
  // changes shapes) can run them
  std::vector<int> act;
  for (int i = 0; i < s->max_slots; ++i)
    if (s->slots[i].active && !s->slots[i].releasing) act.push_back(i);
  SRV_TRY(refresh_shapes(s, static_cast<int>(act.size()), act.data()));
  s->ticks = 0;
  return MPPI_OK;
}

int mppi_server_get_info(mppi_server *s, mppi_server_info *out) {
  if (!s || !out) return MPPI_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  out->max_slots = s->max_slots;
  out->active_slots = 0;
  for (const auto &h : s->slots) out->active_slots += (h.active && !h.releasing) ? 1 : 0;
  out->arena_bytes = s->fl.size;
  out->arena_used = s->fl.used;
  out->rollout_block = s->blk;
  out->rollout_ctas_per_sm = s->ctas_per_sm;
  out->ticks = s->ticks;
  out->last_tick_ms = s->last_tick_ms;
  return MPPI_OK;
}

// ---- asynchronous interface ------------------------------------------------------------

int mppi_server_start(mppi_server *s, int max_batch) {
  if (!s || max_batch < 0) return MPPI_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->running) return s->fail(MPPI_ESTATE, "the scheduler is already running");
  // every active slot must carry the current block shape (the scheduler never refreshes it)
  std::vector<int> act;
  for (int i = 0; i < s->max_slots; ++i)
    if (s->slots[i].active && !s->slots[i].releasing) act.push_back(i);
  SRV_TRY(refresh_shapes(s, static_cast<int>(act.size()), act.data()));
  SRV_TRY(s->cuda(cudaStreamSynchronize(s->stream), "sync"));
  s->max_batch = max_batch;
  s->stop_req = false;
  try {
    s->worker = std::thread(scheduler, s);
  } catch (...) {
    return s->fail(MPPI_ENOMEM, "cannot start the scheduler thread");
  }
  s->running = true;
  return MPPI_OK;
}

int mppi_server_set_batching(mppi_server *s, int min_batch, double max_wait_ms) {
  if (!s || min_batch < 1 || !(max_wait_ms >= 0.0) || max_wait_ms > 1e4) return MPPI_EINVAL;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->min_batch = min_batch;
    s->max_wait_ms = max_wait_ms;
    s->wakeups.fetch_add(1, std::memory_order_release);
  }
  s->cv_work.notify_all();
  return MPPI_OK;
}

int mppi_server_stop(mppi_server *s) {
  if (!s) return MPPI_EINVAL;
  stop_scheduler(s);
  std::lock_guard<std::mutex> lk(s->mu);
  return s->cuda(cudaStreamSynchronize(s->stream), "sync");
}

int mppi_server_submit(mppi_server *s, int slot, const float *h_state, uint64_t *id_out) {
  if (!s || !h_state || !id_out) return MPPI_EINVAL;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (!s->running) return s->fail(MPPI_ESTATE, "the scheduler is not running (mppi_server_start)");
    if (slot < 0 || slot >= s->max_slots || !s->slots[slot].active || s->slots[slot].releasing)
      return s->fail(MPPI_EINVAL, "slot %d is not active", slot);
    if (s->reqs.size() >= kMaxOutstanding) return s->fail(MPPI_EBUSY, "too many outstanding requests");
    const uint64_t id = ++s->next_id;
    Request r;
    r.slot = slot;
    r.status = kQueued;
    std::memcpy(r.state, h_state, sizeof r.state);
    std::memset(r.u0, 0, sizeof r.u0);
    r.t_submit = std::chrono::steady_clock::now();
    if (s->slots[slot].desc.blk != s->blk) {
      // admitted before an autotune changed the block shape: refresh it (between ticks)
      SRV_TRY(refresh_shapes(s, 1, &slot));
    }
    s->reqs.emplace(id, r);
    s->queue.push_back(id);
    *id_out = id;
    s->wakeups.fetch_add(1, std::memory_order_release);
  }
  s->cv_work.notify_all();
  return MPPI_OK;
}

int mppi_server_submit_batch(mppi_server *s, int n, const int *slot_ids, const float *h_states, uint64_t *ids_out) {
  if (!s || n < 0 || (n > 0 && (!slot_ids || !h_states || !ids_out))) return MPPI_EINVAL;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (!s->running) return s->fail(MPPI_ESTATE, "the scheduler is not running (mppi_server_start)");
    for (int q = 0; q < n; ++q) {
      const int slot = slot_ids[q];
      if (slot < 0 || slot >= s->max_slots || !s->slots[slot].active || s->slots[slot].releasing)
        return s->fail(MPPI_EINVAL, "slot %d is not active", slot);
    }
    if (s->reqs.size() + static_cast<size_t>(n) > kMaxOutstanding)
      return s->fail(MPPI_EBUSY, "too many outstanding requests");
    for (int q = 0; q < n; ++q) {
      int slot = slot_ids[q];
      if (s->slots[slot].desc.blk != s->blk) SRV_TRY(refresh_shapes(s, 1, &slot));
      const uint64_t id = ++s->next_id;
      Request r;
      r.slot = slot;
      r.status = kQueued;
      std::memcpy(r.state, h_states + 16 * static_cast<size_t>(q), sizeof r.state);
      std::memset(r.u0, 0, sizeof r.u0);
      r.t_submit = std::chrono::steady_clock::now();
      s->reqs.emplace(id, r);
      s->queue.push_back(id);
      ids_out[q] = id;
    }
    s->wakeups.fetch_add(1, std::memory_order_release);
  }
  s->cv_work.notify_all();
  return MPPI_OK;
}

namespace {
// Take a finished request's result (caller holds mu); false if it is not finished.
int take_result(mppi_server *s, std::unordered_map<uint64_t, Request>::iterator r, float *u0) {
  if (r->second.status == kDone) {
    if (u0) std::memcpy(u0, r->second.u0, sizeof(float) * 4);
    s->reqs.erase(r);
    return MPPI_OK;
  }
  if (r->second.status == kFailed) {
    const int code = r->second.code;
    s->reqs.erase(r);
    return code;
  }
  return MPPI_EAGAIN;
}
}  // namespace

int mppi_server_poll(mppi_server *s, uint64_t id, float *h_u0) {
  if (!s) return MPPI_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto r = s->reqs.find(id);
  if (r == s->reqs.end()) return s->fail(MPPI_EINVAL, "unknown request %llu", static_cast<unsigned long long>(id));
  return take_result(s, r, h_u0);
}

int mppi_server_wait(mppi_server *s, uint64_t id, double timeout_ms, float *h_u0) {
  if (!s) return MPPI_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  const auto deadline = std::chrono::steady_clock::now() +
                        std::chrono::microseconds(static_cast<int64_t>(std::max(0.0, timeout_ms) * 1e3));
  for (;;) {
    auto r = s->reqs.find(id);
    if (r == s->reqs.end()) return s->fail(MPPI_EINVAL, "unknown request %llu", static_cast<unsigned long long>(id));
    const int rc = take_result(s, r, h_u0);
    if (rc != MPPI_EAGAIN) return rc;
    if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
      auto r2 = s->reqs.find(id);
      if (r2 != s->reqs.end()) {
        const int rc2 = take_result(s, r2, h_u0);
        if (rc2 != MPPI_EAGAIN) return rc2;
      }
      return MPPI_ETIMEOUT;
    }
  }
}

int mppi_server_reap(mppi_server *s, int max_n, uint64_t *ids, float *h_u0, int *status, double *latency_ms,
                     double timeout_ms, int *n_out) {
  if (!s || max_n < 0 || !n_out || (max_n > 0 && (!ids || !h_u0))) return MPPI_EINVAL;
  *n_out = 0;
  std::unique_lock<std::mutex> lk(s->mu);
  const auto deadline = std::chrono::steady_clock::now() +
                        std::chrono::microseconds(static_cast<int64_t>(std::max(0.0, timeout_ms) * 1e3));
  for (;;) {
    int k = 0;
    while (k < max_n && !s->done_queue.empty()) {
      const uint64_t id = s->done_queue.front();
      s->done_queue.pop_front();
      auto r = s->reqs.find(id);
      if (r == s->reqs.end()) continue;  // already taken by poll / wait, or cancelled
      ids[k] = id;
      if (latency_ms)
        latency_ms[k] = std::chrono::duration<double, std::milli>(r->second.t_done - r->second.t_submit).count();
      const int rc = take_result(s, r, h_u0 + 4 * k);
      if (status) status[k] = rc;
      ++k;
    }
    if (k > 0 || max_n == 0) {
      *n_out = k;
      return MPPI_OK;
    }
    if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) return MPPI_OK;
  }
}

int mppi_server_cancel(mppi_server *s, uint64_t id) {
  if (!s) return MPPI_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto r = s->reqs.find(id);
  if (r == s->reqs.end()) return s->fail(MPPI_EINVAL, "unknown request %llu", static_cast<unsigned long long>(id));
  // queued: it never runs (the slot's controls and counter are untouched); in flight: its tick
  // finishes (the slot's controls and counter advance) and the result is dropped; finished:
  // the result is dropped.  Either way the id is forgotten.
  s->reqs.erase(r);
  return MPPI_OK;
}

int mppi_server_get_stats(mppi_server *s, mppi_server_stats *out) {
  if (!s || !out) return MPPI_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  out->running = s->running ? 1 : 0;
  out->queued = static_cast<int64_t>(s->queue.size());
  int64_t inflight = 0;
  for (const auto &t : s->tc) inflight += t.busy ? static_cast<int64_t>(t.req_ids.size()) : 0;
  out->in_flight = inflight;
  out->ticks = static_cast<int64_t>(s->async_ticks);
  out->completed = static_cast<int64_t>(s->async_requests_done);
  return MPPI_OK;
}

}  // extern "C"
