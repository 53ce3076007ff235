// trace.cuh -- NVTX ranges around the host-side phases of the library
// (pic_step, each outer iteration, each map evaluation, the tangent solve,
// the commit, pic_start, the batch step, checkpoint save/load), so that a
// profiler's timeline groups the kernels by the phase of Algorithm 1 that
// launched them.  NVTX is header-only: with no profiler attached a range
// costs one indirect call.
#pragma once
#include <nvtx3/nvToolsExt.h>

struct TraceRange {
  explicit TraceRange(const char *name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange &) = delete;
  TraceRange &operator=(const TraceRange &) = delete;
};
