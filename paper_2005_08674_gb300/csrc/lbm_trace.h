// lbm_trace.h -- NVTX ranges around the library's host entry points
// (lbm_init, lbm_step, lbm_get_macros, lbm_reduce, the autotuners and the
// batched step), so that a profiler attached to the process can attribute
// kernels and copies to the call that issued them (for example
// `ncu --nvtx --nvtx-include "lbm_step/"`).  NVTX 3 is header-only; with no
// tool attached a range costs one branch.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace lbmk {

struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

}  // namespace lbmk

#define LBM_TRACE(name) const lbmk::TraceRange lbm_trace_range_(name)
