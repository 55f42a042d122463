// nvtx_range.cuh -- NVTX ranges around the C ABI calls.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace chs {

// An NVTX range spanning one ABI call, named after the entry point, so that the
// calls show up on profiler timelines (Nsight Systems, ncu --nvtx).  NVTX is
// header-only here: without an attached tool the push and pop cost a branch each.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace chs

#define CHS_NVTX_RANGE() const chs::NvtxRange chs_nvtx_range_(__func__)
