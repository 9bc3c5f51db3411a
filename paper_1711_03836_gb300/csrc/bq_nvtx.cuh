// bq_nvtx.cuh -- NVTX ranges around the library's solver phases, so that a
// timeline profiler shows where each solve spends its time (header-only NVTX3;
// the ranges cost nothing when no tool is attached).
#pragma once

#include <nvtx3/nvToolsExt.h>

struct BqRange {
    explicit BqRange(const char *name) { nvtxRangePushA(name); }
    ~BqRange() { nvtxRangePop(); }
    BqRange(const BqRange &) = delete;
    BqRange &operator=(const BqRange &) = delete;
};
