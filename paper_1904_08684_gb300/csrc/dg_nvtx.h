// dg_nvtx.h -- NVTX ranges around the host entry points, so that timeline
// tools attribute device work to dg_init / dg_run / dg_rhs / batch calls.
// NVTX v3 is header-only: without an attached tool a range costs a branch.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace dgswe {

struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace dgswe
