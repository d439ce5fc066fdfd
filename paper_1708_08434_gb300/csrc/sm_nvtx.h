// sm_nvtx.h -- NVTX ranges named after the C-ABI entry points, so that a
// profiler's timeline shows which call issued which kernels.  NVTX3 is
// header-only: nothing to link, and a range costs a few nanoseconds unless
// a tool attaches to it.
#pragma once

#include <nvtx3/nvToolsExt.h>

struct SmRange {
  explicit SmRange(const char *name) { nvtxRangePushA(name); }
  ~SmRange() { nvtxRangePop(); }
  SmRange(const SmRange &) = delete;
  SmRange &operator=(const SmRange &) = delete;
};

// a range over the rest of the enclosing scope, named after the function
#define SM_RANGE() SmRange sm_range_(__func__)
