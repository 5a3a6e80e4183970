// One-shot 2D-PT entry point that allocates no device memory.
//
// Everything the sweep and swap kernels need beyond the caller's inputs and
// outputs (spin state, neighbour lists, per-walker beta/P, f/g, swap
// bookkeeping) is carved from one file-scope device array instead of
// cudaMalloc.  The array exists once per device for the life of the process and
// is shared by every call: a call clears the part it uses before starting, and
// two calls whose GPU work overlaps (other streams, other host threads) race on
// it.
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/pt2d.h"
#include "pt2d_trace.h"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[PT2D_NOALLOC_SCRATCH_BYTES];

// Device address of the scratch array on the current device.  In host code the
// array's name is only a host-side stand-in, so its address is looked up with
// the device current.  The look-up is repeated on every call rather than
// cached: after cudaDeviceReset, or under another context of the same device,
// the library's device code is loaded again at another address, and a cached
// pointer would then point at freed memory.
int scratch_address(void **out) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return PT2D_ERR_CUDA;
    }
    *out = p;
    return PT2D_OK;
}

}  // namespace

extern "C" int pt2d_run_noalloc(const pt2d_instance *inst, int32_t I, const float *beta,
                                int32_t J, const int32_t *P, int32_t runs, int64_t sweeps,
                                int32_t swap_interval, uint64_t seed, void *stream,
                                int8_t *states, int32_t *walker_at, int64_t *f, int64_t *g) {
    if (!inst || !beta || !P || runs < 1) return PT2D_ERR_INVALID_ARG;
    pt2d_options opt;
    pt2d_default_options(&opt);
    opt.stream = stream;
    opt.trace_capacity = 0;
    size_t need = 0;
    int st = pt2d_workspace_size(inst, I, J, runs, &opt, &need);
    if (st) return st;
    if (need > PT2D_NOALLOC_SCRATCH_BYTES) return PT2D_ERR_INVALID_ARG;
    st = pt2d::check_device();  // before the look-up, which fails on other devices
    if (st) return st;
    void *scratch = nullptr;
    st = scratch_address(&scratch);
    if (st) return st;
    opt.workspace = scratch;
    opt.workspace_bytes = PT2D_NOALLOC_SCRATCH_BYTES;
    pt2d_ctx *ctx = nullptr;
    st = pt2d_create(&ctx, inst, I, beta, J, P, runs, &opt);  // clears the carved scratch
    if (st) return st;
    st = pt2d_run(ctx, sweeps, swap_interval, seed);
    if (!st && states) st = pt2d_read(ctx, PT2D_STATES, states, pt2d_array_bytes(ctx, PT2D_STATES));
    if (!st && walker_at)
        st = pt2d_read(ctx, PT2D_WALKER_AT, walker_at, pt2d_array_bytes(ctx, PT2D_WALKER_AT));
    if (!st && f) st = pt2d_read(ctx, PT2D_F, f, pt2d_array_bytes(ctx, PT2D_F));
    if (!st && g) st = pt2d_read(ctx, PT2D_G, g, pt2d_array_bytes(ctx, PT2D_G));
    if (!st) st = pt2d_sync(ctx);
    pt2d_destroy(ctx);
    return st;
}
