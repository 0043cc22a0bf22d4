// NVTX ranges around the C entry points, so that a timeline (Nsight Systems, or
// ncu's --nvtx filters) shows which library call each kernel launch belongs to.
// NVTX v3 is header-only: without a tool attached a range costs a few
// nanoseconds.  Compile with -DLABFM_NO_NVTX to leave them out.
#pragma once

#ifndef LABFM_NO_NVTX
#include <nvtx3/nvToolsExt.h>
#endif

namespace labfm {

struct NvtxRange {
    explicit NvtxRange(const char* name) {
#ifndef LABFM_NO_NVTX
        nvtxRangePushA(name);
#else
        (void)name;
#endif
    }
    ~NvtxRange() {
#ifndef LABFM_NO_NVTX
        nvtxRangePop();
#endif
    }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace labfm

#define LABFM_NVTX(name) ::labfm::NvtxRange labfm_nvtx_range_(name)
