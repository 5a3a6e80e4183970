// Internal interface of the batched persistent kernel.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/pt2d.h"

namespace pt2d {

constexpr int kBatchMaxReplicas = 128;  // I * J of one run, padded to a power of two

// Per-run scalars (int64) in the pool.
enum BatchScalar : int {
    kScBestF = 0,
    kScBestEvent = 1,
    kScSolvedEvent = 2,
    kScTarget = 3,
    kScSweeps = 4,
    kScEvents = 5,
    kScInited = 6,
    kScCount = 8,
};

// One run of one instance.  Offsets are bytes from the pool base.
struct BatchRun {
    int64_t state;       // int8 [(n + 1) * Rp], row-major by colour-sorted position
    int64_t rec;         // int4 [n * rec_vec] packed neighbour records (row indices)
    int64_t cofs;        // int32 [C + 1]
    int64_t beta;        // float [I]
    int64_t P;           // int32 [J]
    int64_t walker_at;   // int32 [R] slot -> walker
    int64_t wparam;      // float beta [Rp], then int32 P [Rp]: each walker's current slot values
    int64_t fg;          // int64 f [Rp], then int32 g [Rp] (last event)
    int64_t stats;       // int64 acc_P, acc_B, sum_f, sum_g, n_feasible [R] each
    int64_t trace;       // int64 trace_f [trace_cap], then trace_g [trace_cap]
    int64_t best_state;  // int8 [n] by spin id
    int64_t scalars;     // int64 [kScCount]
    int64_t counter;     // int32: slabs of this run finished in the current launch
    uint32_t k0, k1;     // seed
    int32_t n, C, I, J, R, Rp, run, trace_cap, rec_vec;
    int32_t sw;          // walkers per slab (power of two, 8..Rp)
    int32_t nslab;       // Rp / sw
    int32_t mode;        // slab spins: 0 int8 in global memory, 1 int8 in shared memory,
                         // 2 bit-packed in shared memory
    int32_t swap_mode;   // PT2D_SWAP_2D or PT2D_SWAP_JCOLUMN
    int32_t dc, dl;      // record degrees (used by the runtime-degree kernel)
    int32_t penalty;     // records carry link weights K and the penalty field k
    int32_t g0;          // constant term of g
    int32_t pad2;
    int64_t work;        // n * Rp, for ordering
};

// One slab of one run: the unit a CTA takes from the work list.
struct BatchItem {
    int32_t run;   // index into the run array
    int32_t slab;  // walkers [slab * sw, (slab + 1) * sw) of the run
};

struct BatchArgs {
    uint8_t *pool;
    const BatchRun *runs;    // [n_runs]
    const BatchItem *items;  // [n_items], largest runs first
    int32_t n_runs;
    int32_t n_items;
    int32_t *queue;          // work counter, zero at launch
    int32_t interval;        // sweeps per event
    int32_t smem_state;      // dynamic shared memory available for one slab's spins
    int64_t *status;         // [n_runs][2]: solved event (-1 none), events done
};

size_t batch_small_smem_bytes();
// Shared memory of a bit-packed slab: (n + 1) rows of sw / 8 bytes, then the
// byte table of k_batch_bits8 (256 x 8 bytes; the runtime-degree kernel's
// nibble table takes the first 64 of them).
inline int64_t batch_bits_bytes(int32_t n, int32_t sw) {
    return ((static_cast<int64_t>(n + 1) * (sw / 8) + 15) & ~int64_t{15}) + 2048;
}
// DC = 0 selects the runtime-degree kernel (degrees and penalty terms read
// from each run's descriptor).
cudaError_t batch_kernel_attributes(int DC, int DL, int smem_state);
cudaError_t launch_batch(const BatchArgs &a, int DC, int DL, int grid, int threads, cudaStream_t st);
// CTAs of k_batch (bits8 false) or k_batch_bits8 that fit on one SM at `threads`
// threads with `smem_state` bytes of slab shared memory (at least 1).
int batch_blocks_per_sm(int DC, int DL, bool bits8, int threads, int smem_state);
// Bit-packed slabs of runs with specialised records (DC = 3, 4 or 6): k_batch_bits8,
// at most kBatchBits8Threads threads per CTA.
cudaError_t launch_batch_bits8(const BatchArgs &a, int DC, int DL, int grid, int threads, cudaStream_t st);
constexpr int kBatchBits8Threads = 896;
// Most threads per CTA of the runtime-degree batch kernel.
constexpr int kBatchGenericThreads = 768;
// Most threads per CTA of the specialised int8 batch kernel (8 walkers a thread).
constexpr int kBatchInt8Threads = 768;

// Bounds on pt2d_batch_instance_bytes from the degrees alone (no colouring and
// no check of the CSR, so O(n) plus a scan of the penalty terms): the sizes
// with 1 and with max degree + 1 colours, equal unless the colour offsets
// outgrow their 256-byte block.  Errors: INVALID_ARG (arguments, or a problem
// the batch cannot hold: degrees, penalty terms).
int batch_instance_bytes_bounds(const pt2d_batch *b, const pt2d_instance *inst, int32_t I, int32_t J,
                                int32_t runs, size_t *lo, size_t *hi);

}  // namespace pt2d
