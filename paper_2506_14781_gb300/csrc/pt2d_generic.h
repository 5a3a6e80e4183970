// Runtime-degree sweep kernels of the plain contexts (pt2d_generic.cu).
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include "pt2d_internal.h"

namespace pt2d {

// One sweep block (nsweeps sweeps, then f and g) of an instance with wide
// records (pt2d_wide.cuh): the int8 slab in shared memory when the tiling
// says so, else in global memory.
cudaError_t launch_generic_sweeps(const Layout &L, const Walkers &wk, const SweepTiling &tl,
                                  int32_t quads_per_run, uint64_t seed, uint32_t sweep0, int32_t nsweeps,
                                  cudaStream_t st);

}  // namespace pt2d
