// Serving runtime: many MPPI controllers (different systems, K and T) stepped together.
//
// Device side
//   slot table   SlotDesc per admitted controller: constants, buffer pointers into the
//                arena, iteration counter (persistent between ticks).
//   k_serve_rollout<BLK>  persistent: each CTA takes work items (slot, block of BLK
//                samples) from an atomic queue, heaviest first, and runs the fused
//                rollout body.  du goes to the CTA's own global-memory slab (written and
//                read back by the same CTA, so it stays in L2) rather than to shared
//                memory, so many CTAs share an SM.  Items of different systems / K / T
//                run side by side.
//   k_serve_merge          persistent: one slot per CTA taken from a second queue; merge of
//                the slot's block partials (FP64 normaliser, double-FP32 weighted sums), U
//                update, u_0 out, shift, counter++.
// Host side
//   first-fit arena allocator (admission by memory), work-item builder, one CUDA graph
//   (memset queue counters -> H2D tick buffer -> rollout -> merge -> D2H u_0) whose copy
//   sizes are updated per tick, and an autotuner over (BLK, CTAs per SM).
// No kernel waits on another block or on the host, so nothing here can hang on a flag.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "../../include/mppi.h"
#include "forest_grid.h"
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
  float *du_slab;          // per persistent CTA: [max_tm][BLK] perturbations (global, L2-resident)
  int slab_floats;         // floats per CTA slab
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
    float *slab = a.du_slab + static_cast<size_t>(blockIdx.x) * a.slab_floats;
    switch (d->sys) {
      case MPPI_CARTPOLE:
        rollout_block<CartPole, BLK, false>(s_p, x0, d->counter, d->U, w.block * BLK, d->S, ps, d->part + w.block,
                                            smem, slab);
        break;
      case MPPI_CAR:
        rollout_block<Car, BLK, false>(s_p, x0, d->counter, d->U, w.block * BLK, d->S, ps, d->part + w.block, smem,
                                       slab);
        break;
      case MPPI_QUAD:
        rollout_block<Quad, BLK, false>(s_p, x0, d->counter, d->U, w.block * BLK, d->S, ps, d->part + w.block, smem,
                                        slab);
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
    default: return MPPI_EINVAL;
  }
}

// relative cost of one rollout-step of each system (for heaviest-first ordering)
double step_weight(int sys) { return sys == MPPI_QUAD ? 7.0 : (sys == MPPI_CAR ? 1.0 : 0.5); }

bool chol_psd(const double *S, int m, double *L) {
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

void spd_inv(const double *L, int m, double *Ai) {
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
  bool active = false;
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

constexpr int kMaxEnvs = 16;
constexpr int kMaxBlockShape = 64;  // smallest BLK the tuner may choose (items are sized for it)

}  // namespace

struct mppi_server {
  int max_slots = 0;
  size_t arena_bytes = 0;
  std::string err;
  int device = 0, num_sms = 0;
  cudaStream_t stream = nullptr;

  char *arena = nullptr;
  FreeList fl;
  SlotDesc *d_slots = nullptr;
  std::vector<HostSlot> slots;
  EnvSlot envs[kMaxEnvs];

  // tick buffer: header | tick_slots[max_slots] | states[max_slots][16] | items[cap]
  size_t item_cap = 0, off_slots = 0, off_states = 0, off_items = 0, tick_bytes = 0;
  unsigned char *d_tick = nullptr, *h_tick = nullptr;
  float *d_u0 = nullptr, *h_u0 = nullptr;
  int *d_counters = nullptr;
  float *d_slab = nullptr;
  size_t slab_cap = 0;
  int max_tm = 1, max_nblk = 1, max_nobs = 0;
  size_t max_grid = 0;  // largest nearest-cylinder grid of an admitted slot (bytes in shared memory)

  int blk = 128, ctas_per_sm = 0, variant = 1;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t n_memset = nullptr, n_h2d = nullptr, n_roll = nullptr, n_merge = nullptr, n_d2h = nullptr;
  bool graph_dirty = true;
  ServeArgs args{};
  int ticks = 0;
  double last_tick_ms = 0.0;

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

int ensure_tick_capacity(mppi_server *s, size_t items) {
  if (items <= s->item_cap && s->d_tick) return MPPI_OK;
  size_t cap = std::max<size_t>(s->item_cap ? s->item_cap : 4096, 4096);
  while (cap < items) cap *= 2;
  SRV_TRY(s->cuda(cudaStreamSynchronize(s->stream), "sync"));
  if (s->d_tick) cudaFree(s->d_tick);
  if (s->h_tick) cudaFreeHost(s->h_tick);
  s->d_tick = nullptr;
  s->h_tick = nullptr;
  s->off_slots = round256(sizeof(TickHeader));
  s->off_states = s->off_slots + round256(sizeof(int) * s->max_slots);
  s->off_items = s->off_states + round256(sizeof(float) * 16 * s->max_slots);
  s->tick_bytes = s->off_items + sizeof(WorkItem) * cap;
  SRV_TRY(s->cuda(cudaMalloc(&s->d_tick, s->tick_bytes), "cudaMalloc(tick)"));
  SRV_TRY(s->cuda(cudaMallocHost(&s->h_tick, s->tick_bytes), "cudaMallocHost(tick)"));
  std::memset(s->h_tick, 0, s->tick_bytes);
  s->item_cap = cap;
  s->graph_dirty = true;
  return MPPI_OK;
}

int build_graph(mppi_server *s) {
  if (s->exec) cudaGraphExecDestroy(s->exec);
  if (s->graph) cudaGraphDestroy(s->graph);
  s->exec = nullptr;
  s->graph = nullptr;
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

  // per-CTA du slabs
  const size_t grid_ctas = static_cast<size_t>(s->num_sms) * cps;
  const size_t slab = static_cast<size_t>(s->max_tm) * s->blk;
  if (grid_ctas * slab > s->slab_cap) {
    if (s->d_slab) cudaFree(s->d_slab);
    s->d_slab = nullptr;
    s->slab_cap = 0;
    SRV_TRY(s->cuda(cudaMalloc(&s->d_slab, sizeof(float) * grid_ctas * slab), "cudaMalloc(du slabs)"));
    s->slab_cap = grid_ctas * slab;
  }
  ServeArgs &a = s->args;
  a.du_slab = s->d_slab;
  a.slab_floats = static_cast<int>(slab);
  a.slots = s->d_slots;
  a.hdr = reinterpret_cast<const TickHeader *>(s->d_tick);
  a.tick_slots = reinterpret_cast<const int *>(s->d_tick + s->off_slots);
  a.states = reinterpret_cast<const float *>(s->d_tick + s->off_states);
  a.items = reinterpret_cast<const WorkItem *>(s->d_tick + s->off_items);
  a.u0_out = s->d_u0;
  a.counters = s->d_counters;

  SRV_TRY(s->cuda(cudaGraphCreate(&s->graph, 0), "graph create"));
  cudaMemsetParams mp{};
  mp.dst = s->d_counters;
  mp.value = 0;
  mp.elementSize = 4;
  mp.width = 2;
  mp.height = 1;
  mp.pitch = 0;
  SRV_TRY(s->cuda(cudaGraphAddMemsetNode(&s->n_memset, s->graph, nullptr, 0, &mp), "memset node"));
  SRV_TRY(s->cuda(cudaGraphAddMemcpyNode1D(&s->n_h2d, s->graph, &s->n_memset, 1, s->d_tick, s->h_tick, s->off_items,
                                           cudaMemcpyHostToDevice),
                  "h2d node"));
  void *rargs[] = {&s->args};
  cudaKernelNodeParams kp{};
  kp.func = const_cast<void *>(rfn);
  kp.gridDim = dim3(s->num_sms * cps);
  kp.blockDim = dim3(s->blk);
  kp.sharedMemBytes = static_cast<unsigned>(rsm);
  kp.kernelParams = rargs;
  SRV_TRY(s->cuda(cudaGraphAddKernelNode(&s->n_roll, s->graph, &s->n_h2d, 1, &kp), "rollout node"));
  int max_nblk = s->max_nblk;
  void *margs[] = {&s->args, &max_nblk};
  cudaKernelNodeParams km{};
  km.func = reinterpret_cast<void *>(k_serve_merge);
  km.gridDim = dim3(s->num_sms * std::min(mocc, 4));
  km.blockDim = dim3(kServeMergeThreads);
  km.sharedMemBytes = static_cast<unsigned>(msm);
  km.kernelParams = margs;
  SRV_TRY(s->cuda(cudaGraphAddKernelNode(&s->n_merge, s->graph, &s->n_roll, 1, &km), "merge node"));
  SRV_TRY(s->cuda(cudaGraphAddMemcpyNode1D(&s->n_d2h, s->graph, &s->n_merge, 1, s->h_u0, s->d_u0, sizeof(float) * 4,
                                           cudaMemcpyDeviceToHost),
                  "d2h node"));
  SRV_TRY(s->cuda(cudaGraphInstantiate(&s->exec, s->graph, 0), "graph instantiate"));
  s->ctas_per_sm = cps;
  s->graph_dirty = false;
  return MPPI_OK;
}

int run_tick(mppi_server *s, int n, const int *slot_ids, const float *states, float *u0_out) {
  // work items, heaviest slots first
  std::vector<int> order(n);
  size_t n_items = 0;
  for (int t = 0; t < n; ++t) {
    order[t] = t;
    const HostSlot &h = s->slots[slot_ids[t]];
    n_items += (h.K + s->blk - 1) / s->blk;
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    const HostSlot &x = s->slots[slot_ids[a]], &y = s->slots[slot_ids[b]];
    return step_weight(x.sys) * x.T > step_weight(y.sys) * y.T;
  });
  SRV_TRY(ensure_tick_capacity(s, n_items));
  bool resized = false;
  for (int t = 0; t < n; ++t) {
    HostSlot &h = s->slots[slot_ids[t]];
    const int nb = (h.K + s->blk - 1) / s->blk;
    if (h.desc.nblk != nb || h.desc.blk != s->blk) {
      h.desc.nblk = nb;
      h.desc.blk = s->blk;
      resized = true;
    }
  }
  if (resized) {
    // block shape changed since admission: refresh (nblk, blk) of the listed slots only
    // (the rest of the device descriptor, e.g. the iteration counter, is device-owned)
    for (int t = 0; t < n; ++t) {
      const int i = slot_ids[t];
      SRV_TRY(s->cuda(cudaMemcpyAsync(&s->d_slots[i].nblk, &s->slots[i].desc.nblk, 2 * sizeof(int),
                                      cudaMemcpyHostToDevice, s->stream),
                      "slot shape"));
    }
  }
  if (s->graph_dirty) SRV_TRY(build_graph(s));

  TickHeader *hdr = reinterpret_cast<TickHeader *>(s->h_tick);
  int *ts = reinterpret_cast<int *>(s->h_tick + s->off_slots);
  float *st = reinterpret_cast<float *>(s->h_tick + s->off_states);
  WorkItem *it = reinterpret_cast<WorkItem *>(s->h_tick + s->off_items);
  size_t k = 0;
  for (int q = 0; q < n; ++q) {
    const int t = order[q];
    const HostSlot &h = s->slots[slot_ids[t]];
    const int nb = (h.K + s->blk - 1) / s->blk;
    for (int b = 0; b < nb; ++b) it[k++] = WorkItem{slot_ids[t], t, b, 0};
  }
  for (int t = 0; t < n; ++t) {
    ts[t] = slot_ids[t];
    std::memcpy(st + 16 * t, states + 16 * t, sizeof(float) * 16);
  }
  hdr->n_items = static_cast<int>(n_items);
  hdr->n_slots = n;
  SRV_TRY(s->cuda(cudaGraphExecMemcpyNodeSetParams1D(s->exec, s->n_h2d, s->d_tick, s->h_tick,
                                                     s->off_items + sizeof(WorkItem) * n_items, cudaMemcpyHostToDevice),
                  "h2d update"));
  SRV_TRY(s->cuda(cudaGraphExecMemcpyNodeSetParams1D(s->exec, s->n_d2h, s->h_u0, s->d_u0, sizeof(float) * 4 * n,
                                                     cudaMemcpyDeviceToHost),
                  "d2h update"));
  const auto t0 = std::chrono::steady_clock::now();
  SRV_TRY(s->cuda(cudaGraphLaunch(s->exec, s->stream), "graph launch"));
  SRV_TRY(s->cuda(cudaStreamSynchronize(s->stream), "tick sync"));
  s->last_tick_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  s->ticks += 1;
  if (u0_out) std::memcpy(u0_out, s->h_u0, sizeof(float) * 4 * n);
  return MPPI_OK;
}

int check_slots(mppi_server *s, int n, const int *slot_ids) {
  if (n < 0 || n > s->max_slots || (n > 0 && !slot_ids)) return s->fail(MPPI_EINVAL, "bad slot list");
  std::vector<char> seen(s->max_slots, 0);
  for (int t = 0; t < n; ++t) {
    const int i = slot_ids[t];
    if (i < 0 || i >= s->max_slots || !s->slots[i].active) return s->fail(MPPI_EINVAL, "slot %d is not active", i);
    if (seen[i]) return s->fail(MPPI_EINVAL, "slot %d listed twice", i);
    seen[i] = 1;
  }
  return MPPI_OK;
}

}  // namespace

extern "C" {

const char *mppi_server_last_error(mppi_server *s) { return s ? s->err.c_str() : "null server"; }

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
  if (rc == MPPI_OK) rc = s->cuda(cudaMalloc(&s->arena, arena_bytes), "cudaMalloc(arena)");
  if (rc == MPPI_OK) rc = s->cuda(cudaMalloc(&s->d_slots, sizeof(SlotDesc) * max_slots), "cudaMalloc(slots)");
  if (rc == MPPI_OK) rc = s->cuda(cudaMemset(s->d_slots, 0, sizeof(SlotDesc) * max_slots), "memset(slots)");
  if (rc == MPPI_OK) rc = s->cuda(cudaMalloc(&s->d_u0, sizeof(float) * 4 * max_slots), "cudaMalloc(u0)");
  if (rc == MPPI_OK) rc = s->cuda(cudaMallocHost(&s->h_u0, sizeof(float) * 4 * max_slots), "cudaMallocHost(u0)");
  if (rc == MPPI_OK) rc = s->cuda(cudaMalloc(&s->d_counters, sizeof(int) * 2), "cudaMalloc(counters)");
  if (rc == MPPI_OK) rc = ensure_tick_capacity(s, 4096);
  if (rc != MPPI_OK) {
    mppi_server_destroy(s);
    return rc;
  }
  s->fl.reset(arena_bytes);
  *out = s;
  return MPPI_OK;
}

int mppi_server_destroy(mppi_server *s) {
  if (!s) return MPPI_OK;
  if (s->stream) cudaStreamSynchronize(s->stream);
  if (s->exec) cudaGraphExecDestroy(s->exec);
  if (s->graph) cudaGraphDestroy(s->graph);
  for (auto &e : s->envs)
    if (e.ptr) cudaFree(e.ptr);
  if (s->arena) cudaFree(s->arena);
  if (s->d_slots) cudaFree(s->d_slots);
  if (s->d_u0) cudaFree(s->d_u0);
  if (s->h_u0) cudaFreeHost(s->h_u0);
  if (s->d_counters) cudaFree(s->d_counters);
  if (s->d_slab) cudaFree(s->d_slab);
  if (s->d_tick) cudaFree(s->d_tick);
  if (s->h_tick) cudaFreeHost(s->h_tick);
  if (s->stream) cudaStreamDestroy(s->stream);
  delete s;
  return MPPI_OK;
}

int mppi_server_set_env(mppi_server *s, int env_id, const void *blob, size_t bytes) {
  if (!s || !blob || env_id < 0 || env_id >= kMaxEnvs || bytes < 8) return MPPI_EINVAL;
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
  SRV_TRY(s->cuda(cudaStreamSynchronize(s->stream), "sync"));
  if (s->envs[env_id].ptr) cudaFree(s->envs[env_id].ptr);
  s->envs[env_id].ptr = nullptr;
  SRV_TRY(s->cuda(cudaMalloc(&e.ptr, std::max<size_t>(payload, 16)), "cudaMalloc(env)"));
  if (payload) SRV_TRY(s->cuda(cudaMemcpy(e.ptr, src, payload, cudaMemcpyHostToDevice), "env copy"));
  e.set = true;
  s->envs[env_id] = e;
  return MPPI_OK;
}

int mppi_server_admit(mppi_server *s, const mppi_slot_config *c, int *slot_out) {
  if (!s || !c || !slot_out) return MPPI_EINVAL;
  *slot_out = -1;
  int n = 0, m = 0;
  if (dims_of(c->system, &n, &m) != MPPI_OK) return s->fail(MPPI_EINVAL, "unknown system %d", c->system);
  if (c->K < 1 || c->K > kServeMaxK || c->T < 1 || c->T > kServeMaxT)
    return s->fail(MPPI_EINVAL, "K in [1, %d] and T in [1, %d] for serving", kServeMaxK, kServeMaxT);
  if (!(c->dt > 0.0f) || !(c->nu > 0.0f) || !(c->lambda > 0.0f)) return s->fail(MPPI_EINVAL, "dt, nu, lambda > 0");
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
  double S[kMaxM * kMaxM], L[kMaxM * kMaxM], Rd[kMaxM * kMaxM];
  for (int i = 0; i < m * m; ++i) S[i] = c->Sigma[i];
  if (!chol_psd(S, m, L)) return s->fail(MPPI_EINVAL, "Sigma is not positive semi-definite");
  if (c->has_R) {
    double LR[kMaxM * kMaxM];
    for (int i = 0; i < m * m; ++i) Rd[i] = c->R[i];
    if (!chol_psd(Rd, m, LR)) return s->fail(MPPI_EINVAL, "R is not positive definite");
    for (int j = 0; j < m; ++j)
      if (!(LR[j * m + j] > 0.0)) return s->fail(MPPI_EINVAL, "R is not positive definite");
  } else {
    for (int j = 0; j < m; ++j)
      if (!(L[j * m + j] > 0.0)) return s->fail(MPPI_EINVAL, "R = lambda Sigma^-1 needs Sigma positive definite");
    double Si[kMaxM * kMaxM];
    spd_inv(L, m, Si);
    for (int i = 0; i < m * m; ++i) Rd[i] = c->lambda * Si[i];
  }
  const double snu = std::sqrt(static_cast<double>(c->nu));
  for (int i = 0; i < m * m; ++i) {
    p.Lnu[i] = static_cast<float>(snu * L[i]);
    p.R[i] = static_cast<float>(Rd[i]);
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

  std::vector<float> U0(TM);
  for (size_t i = 0; i < TM; ++i) U0[i] = c->u_init[i % m];
  int rc = s->cuda(cudaMemcpy(d.U, U0.data(), sizeof(float) * TM, cudaMemcpyHostToDevice), "U init");
  if (rc == MPPI_OK) rc = s->cuda(cudaMemcpy(d.u_init, c->u_init, sizeof(float) * m, cudaMemcpyHostToDevice), "u_init");
  if (rc == MPPI_OK) rc = s->cuda(cudaMemcpy(s->d_slots + slot, &d, sizeof d, cudaMemcpyHostToDevice), "slot desc");
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
    s->graph_dirty = true;
  }
  *slot_out = slot;
  return MPPI_OK;
}

int mppi_server_release(mppi_server *s, int slot) {
  if (!s || slot < 0 || slot >= s->max_slots || !s->slots[slot].active) return MPPI_EINVAL;
  SRV_TRY(s->cuda(cudaStreamSynchronize(s->stream), "sync"));
  HostSlot &h = s->slots[slot];
  s->fl.release(h.off, h.bytes);
  h.active = false;
  return MPPI_OK;
}

int mppi_server_set_controls(mppi_server *s, int slot, const float *U) {
  if (!s || !U || slot < 0 || slot >= s->max_slots || !s->slots[slot].active) return MPPI_EINVAL;
  const HostSlot &h = s->slots[slot];
  SRV_TRY(s->cuda(cudaStreamSynchronize(s->stream), "sync"));
  return s->cuda(cudaMemcpy(h.desc.U, U, sizeof(float) * h.T * h.m, cudaMemcpyHostToDevice), "U copy");
}

int mppi_server_get_controls(mppi_server *s, int slot, float *U) {
  if (!s || !U || slot < 0 || slot >= s->max_slots || !s->slots[slot].active) return MPPI_EINVAL;
  const HostSlot &h = s->slots[slot];
  SRV_TRY(s->cuda(cudaStreamSynchronize(s->stream), "sync"));
  return s->cuda(cudaMemcpy(U, h.desc.U, sizeof(float) * h.T * h.m, cudaMemcpyDeviceToHost), "U copy");
}

int mppi_server_tick(mppi_server *s, int n, const int *slot_ids, const float *states, float *u0_out) {
  if (!s || (n > 0 && !states)) return MPPI_EINVAL;
  SRV_TRY(check_slots(s, n, slot_ids));
  if (n == 0) return MPPI_OK;
  return run_tick(s, n, slot_ids, states, u0_out);
}

int mppi_server_autotune(mppi_server *s, int n, const int *slot_ids, const float *states) {
  if (!s || n < 1 || !states) return MPPI_EINVAL;
  SRV_TRY(check_slots(s, n, slot_ids));
  // snapshot the listed slots (controls + descriptors) so tuning leaves no trace
  std::vector<std::vector<float>> U(n);
  std::vector<SlotDesc> D(s->max_slots);
  SRV_TRY(s->cuda(cudaStreamSynchronize(s->stream), "sync"));
  SRV_TRY(s->cuda(cudaMemcpy(D.data(), s->d_slots, sizeof(SlotDesc) * s->max_slots, cudaMemcpyDeviceToHost), "snap"));
  for (int t = 0; t < n; ++t) {
    const HostSlot &h = s->slots[slot_ids[t]];
    U[t].resize(static_cast<size_t>(h.T) * h.m);
    SRV_TRY(mppi_server_get_controls(s, slot_ids[t], U[t].data()));
  }
  auto restore = [&]() -> int {
    for (int t = 0; t < n; ++t) SRV_TRY(mppi_server_set_controls(s, slot_ids[t], U[t].data()));
    return s->cuda(cudaMemcpy(s->d_slots, D.data(), sizeof(SlotDesc) * s->max_slots, cudaMemcpyHostToDevice),
                   "restore");
  };
  double best = 1e30;
  int best_var = s->variant, best_cps = 0;
  for (int bi = 0; bi < kNumVariants; ++bi) {
    for (int cps_try = 0; cps_try < 2; ++cps_try) {
      s->variant = bi;
      s->ctas_per_sm = 0;
      s->graph_dirty = true;
      SRV_TRY(build_graph(s));
      const int occ = s->ctas_per_sm;
      if (cps_try == 1) {
        if (occ < 2) continue;
        s->ctas_per_sm = occ / 2;
        SRV_TRY(build_graph(s));
      }
      SRV_TRY(run_tick(s, n, slot_ids, states, nullptr));  // warm-up
      double t = 0.0;
      for (int r = 0; r < 3; ++r) {
        SRV_TRY(run_tick(s, n, slot_ids, states, nullptr));
        t += s->last_tick_ms;
      }
      SRV_TRY(restore());
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
  s->graph_dirty = true;
  for (int i = 0; i < s->max_slots; ++i)
    if (s->slots[i].active) {
      s->slots[i].desc.blk = -1;  // force the shape refresh on the next tick
    }
  s->ticks = 0;
  return MPPI_OK;
}

int mppi_server_get_info(mppi_server *s, mppi_server_info *out) {
  if (!s || !out) return MPPI_EINVAL;
  out->max_slots = s->max_slots;
  out->active_slots = 0;
  for (const auto &h : s->slots) out->active_slots += h.active ? 1 : 0;
  out->arena_bytes = s->fl.size;
  out->arena_used = s->fl.used;
  out->rollout_block = s->blk;
  out->rollout_ctas_per_sm = s->ctas_per_sm;
  out->ticks = s->ticks;
  out->last_tick_ms = s->last_tick_ms;
  return MPPI_OK;
}

}  // extern "C"
