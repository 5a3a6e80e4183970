// Penalty-specialised shared-memory sweep kernel (pt2d_penalty.cu).
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include "pt2d_internal.h"

namespace pt2d {

// Degree layouts (coupling width DC, link width DL) the specialised kernel is
// instantiated for; records of instances with penalty terms are padded up to
// one of them when their degrees allow.
bool penalty_kernel_degrees(int DC, int DL);

// One sweep block (nsweeps sweeps, then f and g) of an instance with penalty
// terms whose records have a supported degree layout and whose tiling holds
// the slab in shared memory: int8 with four walkers per thread, or bit-packed
// with a byte (eight walkers) or a nibble (four) per thread.
cudaError_t launch_penalty_sweeps(const Layout &L, const Walkers &wk, const SweepTiling &tl,
                                  int32_t quads_per_run, uint64_t seed, uint32_t sweep0, int32_t nsweeps,
                                  cudaStream_t st);

}  // namespace pt2d
