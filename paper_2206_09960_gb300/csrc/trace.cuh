// trace.cuh -- NVTX ranges for the library's phases (header-only NVTX v3: a no-op unless a
// profiler is attached).
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace psi {

// NVTX range for the scope.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Consecutive phases of one function: next() closes the open range and opens another.
struct NvtxPhases {
  bool open = false;
  void next(const char* name) {
    if (open) nvtxRangePop();
    nvtxRangePushA(name);
    open = true;
  }
  ~NvtxPhases() {
    if (open) nvtxRangePop();
  }
  NvtxPhases() = default;
  NvtxPhases(const NvtxPhases&) = delete;
  NvtxPhases& operator=(const NvtxPhases&) = delete;
};

}  // namespace psi
