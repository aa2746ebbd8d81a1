// NVTX ranges around the library's host calls (each names the kernels it launches), so that
// a profiler's timeline shows where each iteration, tick and training step begins and ends.
// Header-only NVTX v3: with no tool attached a range costs a few nanoseconds.
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace mppi {

struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

}  // namespace mppi
