// Instance preparation shared by the plain contexts and the batch: validation,
// greedy colouring, colour-sorted positions and packed neighbour records.
#pragma once

#include <cstdint>
#include <vector>

#include "../../include/pt2d.h"
#include "pt2d_internal.h"

namespace pt2d {

struct Prep {
    int32_t n = 0, I = 0, J = 0, R = 0, Rp = 0, runs = 0, C = 0, DC = 0, DL = 0;
    int64_t Wc = 0;
    int32_t trace_cap = 0;
    pt2d::SweepTiling tiling{};
    int32_t rec_vec = 0, pad_ref = 0;
    bool penalty = false;  // link weights other than 1 or penalty fields (records carry K and k)
    bool pen_kernel = false;  // penalty records swept by the degree-specialised shared-memory kernel
    bool wide = false;        // wide records (pt2d_wide.cuh) for the runtime-degree kernels
    int32_t dcmax = 0;        // largest coupling degree before padding
    int32_t g0 = 0;        // constant term of g
    std::vector<int32_t> color, pid, pos_of, cofs, rec;
};

// Validates the instance and ladders (beta / P may be NULL for size queries),
// colours it, orders spins by colour and packs the neighbour records; with
// force_dc > 0 the records use that coupling width (links 2) or the call fails;
// with force_dc < 0 they use the wide layout of the runtime-degree kernels.
// Also chooses the plain-context sweep tiling from `opt` and `runs`.  With
// records = false it stops before packing the records (the sizes, colours and
// tiling are set; pp.rec stays empty), for callers that only need sizes.
int prepare(const pt2d_instance *inst, int32_t I, const float *beta, int32_t J, const int32_t *P,
            int32_t runs, const pt2d_options *opt, Prep &pp, int force_dc = 0, bool records = true);

}  // namespace pt2d
