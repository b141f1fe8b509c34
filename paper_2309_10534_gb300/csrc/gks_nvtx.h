// gks_nvtx.h -- NVTX ranges over the library's host entry points (stages,
// steps, batch launches, adjoint passes and segments), for timeline tools and
// ncu's --nvtx-include filters; free when no tool is attached.
#pragma once

#include <nvtx3/nvToolsExt.h>

struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
