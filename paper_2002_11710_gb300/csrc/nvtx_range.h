// Host-side NVTX ranges around the library's entry points, for timeline tools. NVTX v3 is
// header-only: nothing is linked, and a range costs a few nanoseconds when no tool is
// attached. The calls are asynchronous, so a range covers the host's checks and the
// enqueueing of the work, not its execution on the device.
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace asched_nvtx {
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};
}  // namespace asched_nvtx
