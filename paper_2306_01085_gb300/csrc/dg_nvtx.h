// NVTX range around a host-side phase (entry points, DIRK stages, Krylov solves, preconditioner
// builds), visible to timeline tools; with no tool attached it costs a pointer test.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace dg {
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
}  // namespace dg
