// Host-side tracing and test hooks shared by the library's host files.
#pragma once

#include <cstddef>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

namespace pt2d {

// NVTX range for the duration of a scope (visible in Nsight timelines; costs
// nothing when no tool is attached).
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

// cudaMalloc for the library's context workspaces and batch pools; fails as
// if out of memory while a test has asked for injected allocation failures.
cudaError_t device_alloc(void **ptr, size_t bytes);

// PT2D_OK when the current device is an sm_103 GPU, else PT2D_ERR_UNSUPPORTED.
int check_device();

}  // namespace pt2d
