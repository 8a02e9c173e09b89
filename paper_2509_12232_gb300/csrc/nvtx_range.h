// Named host-side ranges around the library's calls (grid build, ligand
// upload, search enqueue, result wait, scoring, local search, surrogate
// training and prediction) for timeline tools (NVIDIA Nsight Systems and
// others that read NVTX). The NVTX 3 header is self-contained: without a
// tool attached a range costs a check of a function pointer.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace dk {

struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

}  // namespace dk
