// Internal interface between the C-ABI host layer and the CUDA kernels.
#pragma once

#include <atomic>
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace pt2d {

// Raise a kernel's dynamic shared memory limit to the most the current device
// allows next to the kernel's static shared memory, once per device.  The
// limit belongs to the kernel and is shared by every host thread, so it is
// never set to one launch's own size: contexts on other threads, whose slabs
// differ in size, would lower it under each other's launches (which then fail
// with cudaErrorInvalidValue).  Concurrent first calls set the same value.
// The kernel is a template argument, so each kernel has its own record of the
// devices it was set on.
template <auto kernel>
cudaError_t allow_max_dynamic_smem() {
    static std::atomic<uint64_t> done_mask{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = dev < 64 ? (uint64_t{1} << dev) : 0;
    if (bit && (done_mask.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    int optin = 0;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin - static_cast<int>(fa.sharedSizeBytes));
    if (e == cudaSuccess && bit) done_mask.fetch_or(bit, std::memory_order_acq_rel);
    return e;
}

// Device layout of one instance and its replica grid.
//  * Spins: int8 S[n + 1][Wc], one row per spin in colour-sorted position
//    order, columns = walkers (walker-fastest, so a warp's neighbour loads are
//    contiguous); row n is all zeros and serves as the padding neighbour.
//  * Columns: run r owns columns [r * Rp, r * Rp + R); Rp = R rounded up to 4
//    so that every group of 4 columns (one Philox call) lies in one run; Wc is
//    the total rounded up to the sweep tile.
//  * One packed record per position, rec_vec int4s: [nb_0..nb_{DC-1} (coupling
//    neighbours, padding -> zero row), lk_0..lk_{DL-1} (link neighbours, padding
//    -> zero row), spin id, 2h, 2J_0..2J_{DC-1}, zero padding], with link
//    weights K and the penalty field k after 2J when penalty is set; records of
//    the runtime-degree kernels use the wide layout of pt2d_wide.cuh (the spin
//    id is at DC + DL in every layout).  Neighbour references are row indices
//    for the global-memory kernels and byte offsets row * SW into the slab for
//    the shared-memory kernels.
struct Layout {
    int8_t *S;
    int64_t Wc;
    int32_t n;
    int32_t C;
    int32_t DC;
    int32_t DL;
    int32_t rec_vec;      // int4s per record
    int32_t pad_ref;      // neighbour reference of the zero row (n, or n * SW when scaled)
    const int4 *rec;      // [n][rec_vec]
    const int32_t *cofs;  // [C + 1] colour class offsets (positions)
    int32_t penalty;      // records carry link weights K and the penalty field k
    int32_t g0;           // constant term of g
};

struct Walkers {
    float *wbeta;   // [Wc] beta of each column's current slot
    int32_t *wP;    // [Wc] P of each column's current slot
    int64_t *f;     // [Wc] cost after the last sweep of an event
    int32_t *g;     // [Wc] constraint after the last sweep of an event
};

struct RunState {
    int32_t runs, I, J, R, Rp;
    const float *beta;      // [I]
    const int32_t *P;       // [J]
    int32_t *walker_at;     // [runs][R]
    int64_t *acc_P;         // [runs][R]
    int64_t *acc_B;         // [runs][R]
    int64_t *sum_f;         // [runs][R]
    int64_t *sum_g;         // [runs][R]
    int64_t *n_feasible;    // [runs][R]
    int64_t *trace_f;       // [runs][trace_cap]
    int64_t *trace_g;       // [runs][trace_cap]
    int64_t trace_cap;
    int64_t *best_f;        // [runs]
    int64_t *best_event;    // [runs]
    int8_t *best_state;     // [runs][n]
    const int64_t *target;  // [runs]
    int64_t *solved_event;  // [runs]
    int32_t swap_mode;      // PT2D_SWAP_2D or PT2D_SWAP_JCOLUMN
};

struct SweepTiling {
    int lanes_per_spin;  // quads (4 walkers) per spin row segment of a CTA
    int threads;         // threads per CTA
    bool smem;           // slab in shared memory (k_sweep_smem) or global (k_sweep_global)
    int walkers_per_thread;  // 4, or 8 in the int8 and bit-packed shared-memory kernels
    bool bits;           // slab bit-packed in shared memory (k_sweep_bits)
};

// Most threads per CTA of the byte-per-thread bit-packed sweep kernels: the
// launch bounds the kernels are compiled with and the host's tiling limit.
constexpr int kBits8Threads = 896;         // k_sweep_bits8: 72 registers, 28 warps
constexpr int kPenaltyBits8Threads = 512;  // k_sweep_penalty_bits8

// Dynamic shared memory of k_sweep_smem for n spins and a slab of W walkers.
size_t smem_sweep_bytes(int32_t n, int walkers_per_cta);
// Dynamic shared memory of k_sweep_bits (slab of bits plus the nibble table).
size_t bits_sweep_bytes(int32_t n, int walkers_per_cta);
constexpr size_t kSweepStaticSmem = 2048;  // epilogue reduction arrays and slack

cudaError_t launch_init(const Layout &L, const RunState &rs, const Walkers &wk, uint64_t seed,
                        cudaStream_t st);
cudaError_t launch_sweeps(const Layout &L, const Walkers &wk, const SweepTiling &tl,
                          int32_t quads_per_run, uint64_t seed, uint32_t sweep0, int32_t nsweeps,
                          cudaStream_t st);
cudaError_t launch_swap_event(const Layout &L, const RunState &rs, const Walkers &wk,
                              uint64_t seed, int64_t event, cudaStream_t st);

// diagnostics
cudaError_t diag_philox(const uint32_t *ctr, const uint32_t *key, uint32_t *out, int64_t count);
cudaError_t diag_pt_exp(const float *x, float *y, int64_t count);
cudaError_t diag_heatbath(const float *beta, const int32_t *H, const uint32_t *r, int8_t *spin,
                          int64_t count);
cudaError_t diag_swap_accept(const float *x, const uint32_t *r, int8_t *acc, int64_t count);

}  // namespace pt2d
