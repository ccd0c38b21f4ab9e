// nvtx_range.h -- NVTX range over one library call (visible in Nsight
// Systems / Compute timelines; a no-op without a tool attached).
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace lsm {

struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

}  // namespace lsm
