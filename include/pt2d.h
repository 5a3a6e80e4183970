/*
 * pt2d.h — C ABI of the GB300 (sm_103a) two-dimensional parallel tempering
 * library (arxiv 2506.14781, "Two-dimensional Parallel Tempering for
 * Constrained Optimization").
 *
 * The library runs 2D-PT (Algorithm 1) on an I x J grid of replicas of a
 * constrained Ising problem with penalised energy E_j = f + P_j g (Eq. 1):
 * row i has inverse temperature beta_i, column j penalty P_j.  Heat-bath
 * Gibbs sweeps are interleaved with P-swaps inside rows (Eq. 2) and
 * beta-swaps inside columns (Eq. 3).  Many independent runs ("runs", each its
 * own I x J grid, all on the same instance) are simulated together.
 *
 * Conventions for every entry point:
 *  - returns PT2D_OK (0) or a negative PT2D_ERR_* code; pt2d_strerror() names it;
 *  - host pointers are read during the call only (inputs are copied); the
 *    caller keeps ownership of every buffer it passes;
 *  - device work is queued on the context's stream; pt2d_read/pt2d_write and
 *    pt2d_sync synchronise that stream;
 *  - no global state, with one documented exception: pt2d_run_noalloc
 *    carves its buffers from one file-scope device array that every call of
 *    that entry point shares (see its comment).  Otherwise one context per
 *    thread at a time (contexts are independent and may live on different
 *    streams).
 *
 * Numerical contract (identical on the CPU oracle and the GPU):
 *  - couplings are int16, fields and penalties integers, so f, g, E and the
 *    local field H_a = E(s_a=-1) - E(s_a=+1)
 *        = 2 sum_b J_ab s_b + 2 h_a + P_j (sum_{links l of a} K_al s_l + k_a)
 *    are exact integers (|H_a| < 2^24 is required);
 *  - g = g0 + sum_{links a<b} K_ab [s_a != s_b] + sum_a k_a [s_a = -1]; for copy
 *    constraints (K = 1, k = 0, g0 = 0) the number of copy links with
 *    s_a != s_b, normalised so that a broken link counts 1 (see pt2d_instance);
 *  - swap_mode selects Algorithm 1 (default) or the J-column PT baseline;
 *  - random words: Philox4x32-10 keyed by the 64-bit seed; counter
 *    (c0, c1, c2, (run << 4) | tag) with
 *      sweep: c0 = spin id, c1 = global sweep index, c2 = walker / 4, word walker % 4
 *      init:  c0 = spin id, c1 = 0,                 c2 = walker / 4, word walker % 4
 *      swap:  c0 = lower slot index of the pair, c1 = event index n (1-based), c2 = 0, word 0
 *    and u = ((word >> 9) + 1) * 2^-23, a uniform on the grid of (0, 1];
 *  - heat bath: t = beta (x) float(H); e = pt_exp(-t); d = 1 (+) e; v = u (x) d;
 *    new spin +1 iff v < 1 (single-precision, round-to-nearest, no fused ops);
 *  - swaps: x = beta_i (x) float(dP dg) for P-swaps, x = (beta_{i+1} (-) beta_i)
 *    (x) float(E_{i+1} - E_i) for beta-swaps; accept iff x >= 0 or u <= pt_exp(x);
 *  - pt_exp: Cody-Waite reduction by ln 2 split in two floats, degree-7 Taylor
 *    polynomial in Horner form, scaling by 2^k in two steps; +inf above 88.75,
 *    0 below -104.
 *  Spins of one colour of the greedy colouring (ascending ids, smallest colour
 *  free among coupling and link neighbours) are updated together; colours in
 *  ascending order make one sweep.
 */
#ifndef PT2D_H
#define PT2D_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define PT2D_OK 0
#define PT2D_ERR_INVALID_ARG (-1) /* malformed instance, ladder or size      */
#define PT2D_ERR_OOM (-2)         /* device or host allocation failed        */
#define PT2D_ERR_CUDA (-3)        /* a CUDA call failed (see pt2d_cuda_error) */
#define PT2D_ERR_TIMEOUT (-4)     /* a bounded device wait expired           */
#define PT2D_ERR_STATE (-5)       /* call not valid in the context's state   */
#define PT2D_ERR_UNSUPPORTED (-6) /* no sm_103a device or feature missing    */

/* ---- readable / writable context arrays (pt2d_read, pt2d_write) --------- */
/* R = I*J slots per run; slot index s = i*J + j; walker ids 0..R-1 per run. */
#define PT2D_STATES 1       /* int8  [runs][R][n]  spins of each walker (+1/-1)    */
#define PT2D_WALKER_AT 2    /* int32 [runs][R]     slot -> walker                  */
#define PT2D_F 3            /* int64 [runs][R]     cost f of each walker, last event */
#define PT2D_G 4            /* int64 [runs][R]     constraint g of each walker       */
#define PT2D_COUNTERS 5     /* int64 [4] sweeps done, events done, direction, inited */
#define PT2D_TRACE_F 6      /* int64 [runs][trace_capacity] bottom-right f after event n */
#define PT2D_TRACE_G 7      /* int64 [runs][trace_capacity] bottom-right g            */
#define PT2D_BEST_F 8       /* int64 [runs] lowest bottom-right f with g == 0         */
#define PT2D_BEST_EVENT 9   /* int64 [runs] event of BEST_F, -1 if none               */
#define PT2D_BEST_STATE 10  /* int8  [runs][n] spins of BEST_F                        */
#define PT2D_SOLVED_EVENT 11 /* int64 [runs] first event with g == 0 and f <= target, -1 */
#define PT2D_ACC_P 12       /* int64 [runs][R] accepted P-swaps, by lower slot        */
#define PT2D_ACC_B 13       /* int64 [runs][R] accepted beta-swaps, by lower slot     */
#define PT2D_SUM_F 14       /* int64 [runs][R] per slot: sum of f after each event    */
#define PT2D_SUM_G 15       /* int64 [runs][R] per slot: sum of g                     */
#define PT2D_N_FEASIBLE 16  /* int64 [runs][R] per slot: events with g == 0           */
#define PT2D_COLORS 17      /* int32 [n] colour of each spin (read only)              */
#define PT2D_TARGET 18      /* int64 [runs] solved threshold (write to set)           */

/* ---- problem description ---------------------------------------------- */
/* Physical (sparsified) instance.  Host pointers; copied at create time.
 * Couplings: symmetric CSR without self loops, J in int16, f = -sum_{a<b}
 * J_ab s_a s_b - sum_a h_a s_a.  Links: symmetric CSR of penalty terms,
 *   g = g0 + sum_{links a<b} K_ab [s_a != s_b] + sum_a k_a [s_a = -1],
 * the constraint function of Eq. 1 (any quadratic penalty of binary
 * variables, e.g. one-hot groups, has this form; pt2d_onehot_penalty builds
 * it).  Copy constraints are K = 1, k = 0, g0 = 0: g = #{links with s_a != s_b}
 * (lk_w = hk = NULL).  The local field of a spin is then
 *   H_a = E(s_a=-1) - E(s_a=+1) = 2 sum_b J_ab s_b + 2 h_a + P (sum_l K_al s_l + k_a).
 * Instances with weights other than K = 1 or any k != 0 run on the generic
 * sweep kernel of a context (not in batches or servers).  The caller keeps g
 * >= 0 for every state; g is an int32 per walker (|g0| + sum |K| + sum |k| <
 * 2^31 is checked).  Column indices need not be sorted. */
typedef struct {
    int32_t n;              /* physical spins, >= 1                          */
    const int32_t *cp_ptr;  /* [n+1] coupling row pointers                   */
    const int32_t *cp_col;  /* [cp_ptr[n]] coupling neighbours                */
    const int16_t *cp_J;    /* [cp_ptr[n]] coupling values                    */
    const int32_t *lk_ptr;  /* [n+1] link row pointers                        */
    const int32_t *lk_col;  /* [lk_ptr[n]] link neighbours                    */
    const int32_t *h;       /* [n] integer field, or NULL for zero            */
    const int32_t *color;   /* [n] proper colouring, or NULL: greedy (above)  */
    const int16_t *lk_w;    /* [lk_ptr[n]] penalty weight K of each link entry (equal
                               both ways), or NULL for all 1                   */
    const int32_t *hk;      /* [n] penalty field k, or NULL for zero          */
    int64_t g0;             /* constant term of g                             */
} pt2d_instance;

typedef struct {
    void *stream;            /* cudaStream_t for all work; NULL = default stream   */
    void *workspace;         /* caller-owned device memory, or NULL: library allocates */
    size_t workspace_bytes;  /* size of `workspace` (see pt2d_workspace_size)      */
    int32_t trace_capacity;  /* events kept in the bottom-right trace (default 1024) */
    int32_t walkers_per_cta; /* sweep tiling: 4..128 (16..128 int8 in shared memory,
                                8..128 bit-packed), power of two; 0 = automatic      */
    int32_t threads_per_cta; /* multiple of 32, >= walkers_per_cta/walkers_per_thread,
                                <= 256 (global slab), 1024 (shared slab, 4 walkers
                                a thread), 768 (int8 slab, 8 walkers a thread), 896
                                (bit-packed slab of a specialised layout, 8 walkers
                                a thread) or 512 (other bit-packed slabs, 8 walkers
                                a thread); 0 = automatic                          */
    int32_t device;          /* CUDA device ordinal; -1 = current device            */
    int32_t profile;         /* nonzero: time every kernel launch with CUDA events  */
    int32_t sweep_kernel;    /* 0 automatic, 1 slab in global memory, 2 int8 slab in
                                shared memory (also for generic degree layouts and
                                penalty terms), 3 bit-packed slab in shared memory
                                (specialised layouts and penalty terms with coupling
                                degree <= 6 and link degree <= 3 only, else
                                INVALID_ARG; 2, 3: INVALID_ARG if it does not fit)   */
    int32_t walkers_per_thread; /* 4 or 8 for the int8 shared-memory kernel of the
                                   specialised layouts and for the bit-packed
                                   kernels, others: 4; 0 = automatic: 8, or 4 when
                                   more threads are asked for than 8 walkers a
                                   thread allow                                    */
    int32_t swap_mode;       /* PT2D_SWAP_2D (0): Algorithm 1.  PT2D_SWAP_JCOLUMN (1):
                                the paper's J-column PT baseline -- every event is a
                                beta-swap event (pairs starting at the first row on
                                odd events, the second on even ones), so replicas
                                never change column (standard PT per column), and
                                each event records the last row's replica of lowest
                                g, then lowest f, then lowest column, instead of the
                                bottom-right one (trace, best, solved)             */
} pt2d_options;

#define PT2D_SWAP_2D 0
#define PT2D_SWAP_JCOLUMN 1

typedef struct pt2d_ctx pt2d_ctx;

/* Fill `opt` with defaults (stream NULL, no workspace, trace 1024, automatic tiling). */
void pt2d_default_options(pt2d_options *opt);

/* Device bytes a context needs (for a caller-provided workspace).
 * Errors: INVALID_ARG for a malformed instance or sizes. */
int pt2d_workspace_size(const pt2d_instance *inst, int32_t I, int32_t J, int32_t runs,
                        const pt2d_options *opt, size_t *bytes);

/* Create a context: validates and copies the instance (the inputs of
 * Algorithm 1: couplings and fields, the constraint given by the copy links,
 * and the two ordered ladders), colours it if no colouring is given, and lays
 * it out on the device.
 * beta: [I] float32, ascending, in the units of the integer couplings.
 * P:    [J] int32, ascending, >= 0.  I * J <= 8192.  runs >= 1 independent grids.
 * Errors: INVALID_ARG (bad CSR, asymmetric, self loop, improper colouring,
 * non-ascending ladder, |H| bound exceeded, workspace too small), OOM, CUDA,
 * UNSUPPORTED (device is not sm_103). */
int pt2d_create(pt2d_ctx **out, const pt2d_instance *inst, int32_t I, const float *beta,
                int32_t J, const int32_t *P, int32_t runs, const pt2d_options *opt);

/* Run floor(sweeps / swap_interval) swap events of Algorithm 1: each event is
 * swap_interval sweeps of every walker, then f and g of the final sweep, then
 * one round of P-swaps (direction +1) or beta-swaps (direction -1) on odd
 * (odd n) or even (even n) pairs, then the bottom-right record; the direction
 * flips after every even event.  The first call initialises the spins from the
 * seeded init stream.  Counters persist, so run(a); run(b) equals run(a + b)
 * when both are multiples of the interval.  Asynchronous on the context stream.
 * Errors: INVALID_ARG (interval < 1, sweeps < 0, seed differs from the first
 * call's seed, sweep counter would pass 2^32), CUDA. */
int pt2d_run(pt2d_ctx *ctx, int64_t sweeps, int32_t swap_interval, uint64_t seed);

/* Copy one context array (PT2D_* above) to host memory; synchronises the
 * stream.  `bytes` must equal the array size.  Errors: INVALID_ARG, STATE
 * (reading spins before the first run), CUDA. */
int pt2d_read(pt2d_ctx *ctx, int32_t what, void *host_dst, size_t bytes);

/* Copy the spins of one walker (run, walker id) to host_dst[n] in spin-id
 * order; synchronises the stream.  Used to read a single replica (for example
 * the one in the bottom-right slot, whose spins Algorithm 1 stores) without
 * copying every walker.  Errors: INVALID_ARG, STATE (before the first run), CUDA. */
int pt2d_read_walker(pt2d_ctx *ctx, int32_t run, int32_t walker, int8_t *host_dst);

/* Overwrite one context array from host memory (checkpoint restore):
 * STATES, WALKER_AT, COUNTERS, BEST_F, BEST_EVENT, BEST_STATE, SOLVED_EVENT,
 * ACC_P, ACC_B, SUM_F, SUM_G, N_FEASIBLE, TARGET, TRACE_F, TRACE_G.  Writing
 * COUNTERS with inited = 1 marks the context initialised (the seed of the next
 * run is then adopted).  Errors: INVALID_ARG (size, permutation not valid),
 * CUDA. */
int pt2d_write(pt2d_ctx *ctx, int32_t what, const void *host_src, size_t bytes);

/* Size in bytes of array `what` for this context (0 if unknown). */
size_t pt2d_array_bytes(const pt2d_ctx *ctx, int32_t what);

/* Block until the context's queued work is done.  Errors: CUDA, TIMEOUT. */
int pt2d_sync(pt2d_ctx *ctx);

/* Number of colours of the context's colouring, and kernel launches queued so far. */
int pt2d_num_colors(const pt2d_ctx *ctx);
int64_t pt2d_launch_count(const pt2d_ctx *ctx);

/* Sweep tiling the context chose: out[0] = kernel (1 slab in global memory, 2
 * int8 slab in shared memory, 3 bit-packed slab in shared memory, 4 generic
 * degree layout in global memory, 5 generic degree layout with the int8 slab in
 * shared memory, 6 penalty terms with coupling width 3, 4 or 6 and link width
 * 2 or 3, int8 slab in shared memory, 7 the same with a bit-packed slab),
 * out[1] = walkers per CTA, out[2] = threads per CTA,
 * out[3] = walkers per thread.  Host only.  Errors: INVALID_ARG (NULL). */
int pt2d_tiling(const pt2d_ctx *ctx, int32_t out[4]);

/* The sweep tiling pt2d_create would choose for this problem (out as for
 * pt2d_tiling), without creating a context or touching the GPU; with no GPU
 * visible it plans for 152 SMs and 227 KB of shared memory per CTA.  Host
 * only.  Errors: INVALID_ARG (as pt2d_workspace_size). */
int pt2d_plan_tiling(const pt2d_instance *inst, int32_t I, int32_t J, int32_t runs,
                     const pt2d_options *opt, int32_t out[4]);

/* Kernel timing of a context created with opt.profile != 0: total device
 * milliseconds and launch count of the sweep kernel (kind 0) or the swap-event
 * kernel (kind 1) since creation, from CUDA events recorded on the context
 * stream around each launch.  Synchronises the stream.
 * Errors: INVALID_ARG (bad kind), STATE (profiling off), CUDA. */
#define PT2D_KERNEL_SWEEP 0
#define PT2D_KERNEL_SWAP 1
int pt2d_kernel_time(pt2d_ctx *ctx, int32_t kind, double *ms, int64_t *launches);

/* Release everything the context owns (not a caller-provided workspace). */
void pt2d_destroy(pt2d_ctx *ctx);

/* Static description of a status code. */
const char *pt2d_strerror(int status);

/* Last CUDA error code (cudaError_t) recorded by the context, 0 if none. */
int pt2d_cuda_error(const pt2d_ctx *ctx);

/* ---- batched persistent form ------------------------------------------------ */
/* Many independent 2D-PT problems of uneven size (each an instance with its own
 * ladders, runs and seed) simulated by one persistent kernel (Algorithm 1 for
 * each run, I * J <= 128 replicas per run).  Each launch advances every run by
 * one event: a run's replicas are split into slabs, CTAs take slabs from a
 * work list sorted by decreasing run size and perform the sweeps and f and g
 * (a slab's spins in shared memory when they fit), and the CTA finishing a
 * run's last slab performs its swap event and bottom-right record.  Events are
 * launches replayed from a CUDA graph.  Each run follows exactly the
 * trajectory of a context created with pt2d_create on the same instance and
 * ladders, run with the same seed (run r of an instance uses run index r).
 *
 * Memory: the batch owns a device pool (or uses opt->workspace); instances are
 * added and removed at any time between launches (continuous batching), and
 * pt2d_batch_add fails with PT2D_ERR_OOM, leaving the batch unchanged, when
 * the pool has no room.  All calls are on the batch stream (opt->stream, or a
 * stream the batch creates). */
typedef struct pt2d_batch pt2d_batch;

/* pool_bytes: device bytes for instances (ignored with opt->workspace, whose
 * size then includes the batch's bookkeeping); max_coupling_degree: largest
 * number of coupling neighbours of any spin that will be added: <= 6 (with at
 * most 2 links per spin, copy constraints only) uses kernels specialised for
 * that degree; larger values use a kernel that reads each problem's degrees at
 * run time and also takes any number of links and general penalty terms
 * (pt2d_instance lk_w, hk, g0); max_runs: most runs alive at once.  opt: stream, workspace,
 * trace_capacity, and the initial launch shape (pt2d_batch_shape below):
 * threads_per_cta (0 = 1024), sweep_kernel (= storage), walkers_per_cta
 * (= global_width, 0 = 32); balance starts at 2.  device.
 * Errors: INVALID_ARG, OOM, CUDA, UNSUPPORTED. */
int pt2d_batch_create(pt2d_batch **out, size_t pool_bytes, int32_t max_coupling_degree,
                      int32_t max_runs, const pt2d_options *opt);

/* Device bytes pt2d_batch_add would take for this problem (0 if invalid). */
size_t pt2d_batch_instance_bytes(const pt2d_batch *b, const pt2d_instance *inst, int32_t I,
                                 int32_t J, int32_t runs);

/* Add a problem: instance, ladders (as for pt2d_create), `runs` runs seeded by
 * `seed`, target[runs] (solved iff bottom-right g == 0 and f <= target) or
 * NULL.  Its spins are initialised at its first event.  *id receives the
 * problem's id.  Errors: INVALID_ARG (also I * J > 128 or a degree above the
 * batch's), OOM (pool full), CUDA. */
int pt2d_batch_add(pt2d_batch *b, const pt2d_instance *inst, int32_t I, const float *beta,
                   int32_t J, const int32_t *P, int32_t runs, uint64_t seed,
                   const int64_t *target, int64_t *id);

/* Remove a problem and return its memory to the pool.  Errors: INVALID_ARG. */
int pt2d_batch_remove(pt2d_batch *b, int64_t id);

/* Advance every run of every problem by `events` swap events of
 * `swap_interval` sweeps (one launch).  Asynchronous.  Errors: INVALID_ARG,
 * OOM (more runs than max_runs), CUDA. */
int pt2d_batch_run(pt2d_batch *b, int32_t events, int32_t swap_interval);

/* Launch shape of a batch.  Every shape computes the same trajectories.
 *   threads_per_cta  128..1024, multiple of 32; the kernels run at most 768
 *                    (int8 slabs of specialised records, 8 walkers a thread),
 *                    896 (bit-packed slabs of specialised records) or 768
 *                    (every slab of the runtime-degree kernel) of them
 *   storage          where a run's slab of spins lives during an event: 0 =
 *                    int8 in shared memory where it fits, else bit-packed in
 *                    shared memory where that fits, else int8 in global
 *                    memory; 1 = always global; 2 = no bit-packed slabs; 3 = no
 *                    int8 shared-memory slabs
 *   global_width     walkers per slab of runs kept in global memory (16..128,
 *                    power of two)
 *   balance          0, or k >= 1: a run is split into slabs of at most
 *                    (total spins x replicas) / (k x CTAs) spin-walkers each,
 *                    down to the narrowest slab its storage allows, so that
 *                    large runs do not leave other CTAs idle at the event's end */
typedef struct pt2d_batch_shape {
    int32_t threads_per_cta;
    int32_t storage;
    int32_t global_width;
    int32_t balance;
} pt2d_batch_shape;

/* Read / set the launch shape (host only; applies from the next launch).
 * Errors: INVALID_ARG. */
int pt2d_batch_get_shape(const pt2d_batch *b, pt2d_batch_shape *shape);
int pt2d_batch_set_shape(pt2d_batch *b, const pt2d_batch_shape *shape);

/* Time candidate launch shapes (storage 0, 1 or 2 x balance 0, 2, 4 or 8 at
 * 1024 threads, then the best of those at 512, 256 and 128 threads) on two
 * launches of `events` events each and keep the fastest, returned in *chosen
 * (may be NULL).  The trial launches advance the chains like pt2d_batch_run.
 * Errors as pt2d_batch_run. */
int pt2d_batch_autotune(pt2d_batch *b, int32_t events, int32_t swap_interval,
                        pt2d_batch_shape *chosen);

/* Copy array `what` (the PT2D_* arrays of pt2d_read, for this problem's runs)
 * to host memory; synchronises.  Errors: INVALID_ARG, STATE, CUDA. */
int pt2d_batch_read(pt2d_batch *b, int64_t id, int32_t what, void *host_dst, size_t bytes);
size_t pt2d_batch_array_bytes(const pt2d_batch *b, int64_t id, int32_t what);

/* Status of every problem after the last launch (synchronises): ids[k],
 * solved_event[k] (earliest event at which one of its runs was solved, -1 if
 * none) and events_done[k], for at most `capacity` problems; *count = number
 * of problems.  Problems added since the last launch are not listed.
 * Errors: INVALID_ARG, CUDA. */
int pt2d_batch_poll(pt2d_batch *b, int64_t *ids, int64_t *solved_event, int64_t *events_done,
                    int32_t capacity, int32_t *count);

int pt2d_batch_sync(pt2d_batch *b);
size_t pt2d_batch_free_bytes(const pt2d_batch *b);   /* largest free block of the pool */
int64_t pt2d_batch_launch_count(const pt2d_batch *b);
int pt2d_batch_cuda_error(const pt2d_batch *b);
void pt2d_batch_destroy(pt2d_batch *b);

/* ---- continuous-batching server ------------------------------------------- */
/* A request loop over the batched form: requests (one constrained Ising
 * problem each, with its ladders, seed, target energy and sweep limit) wait in
 * a FIFO queue; pt2d_server_step admits queued requests in order while the
 * device pool has room, advances every resident request by `events_per_step`
 * swap events in one batched launch, and evicts those that are solved (the
 * bottom-right replica has g == 0 and f <= target) or have used max_sweeps,
 * keeping each one's lowest-energy feasible state.  A request's result does
 * not depend on the other requests resident with it. */
typedef struct pt2d_server pt2d_server;

#define PT2D_REQUEST_QUEUED 0
#define PT2D_REQUEST_RUNNING 1
#define PT2D_REQUEST_DONE 2
#define PT2D_REQUEST_CANCELLED 3
#define PT2D_REQUEST_FAILED 4

typedef struct {
    int32_t state;         /* PT2D_REQUEST_*                                     */
    int32_t error;         /* status code when FAILED                            */
    int32_t n;             /* physical spins                                      */
    int64_t best_f;        /* lowest bottom-right f with g == 0 (INT64_MAX: none) */
    int64_t best_event;    /* event of best_f, -1 if none                         */
    int64_t solved_event;  /* first event with g == 0 and f <= target, -1 if none */
    int64_t sweeps_done;
    double t_submit, t_admit, t_done;  /* seconds since the server was created    */
} pt2d_request_status;

/* pool_bytes: device bytes for resident problems; max_requests: most resident
 * at once; swap_interval: sweeps per event; events_per_step: events per
 * launch.  opt as for pt2d_batch_create.  Errors: those of pt2d_batch_create. */
int pt2d_server_create(pt2d_server **out, size_t pool_bytes, int32_t max_coupling_degree,
                       int32_t max_requests, int32_t swap_interval, int32_t events_per_step,
                       const pt2d_options *opt);

/* Queue a request (the problem is copied).  Errors: INVALID_ARG (bad
 * arguments, or a problem a batch cannot hold: general penalty terms,
 * I * J > 128, a coupling degree above the server's), OOM (larger than the
 * whole pool, so it could never be admitted).  The rest of the problem's
 * validation (a symmetric CSR without self loops or duplicates, the local-field
 * bound) happens at admission: a problem that fails it ends FAILED with
 * INVALID_ARG in its status.  Submission costs O(n) plus a copy of the arrays. */
int pt2d_server_submit(pt2d_server *s, const pt2d_instance *inst, int32_t I, const float *beta,
                       int32_t J, const int32_t *P, uint64_t seed, int64_t target,
                       int64_t max_sweeps, int64_t *request_id);

/* Admit, run one launch, evict finished requests; reports resident, queued
 * and just-finished counts (outputs may be NULL).  Synchronises.  Errors: CUDA. */
int pt2d_server_step(pt2d_server *s, int32_t *active, int32_t *queued, int32_t *finished);

/* State and results of a request; best_state[n] (spins by id) is filled for a
 * finished request when not NULL.  Errors: INVALID_ARG. */
int pt2d_server_status(pt2d_server *s, int64_t request_id, pt2d_request_status *status,
                       int8_t *best_state);

/* Cancel a queued or resident request (its memory returns to the pool). */
int pt2d_server_cancel(pt2d_server *s, int64_t request_id);

/* Drop a finished, cancelled or failed request's record.  Errors: STATE. */
int pt2d_server_forget(pt2d_server *s, int64_t request_id);

size_t pt2d_server_free_bytes(const pt2d_server *s);
void pt2d_server_destroy(pt2d_server *s);

/* ---- adaptive ladder schedule (Algorithm 2) ------------------------------- */
/* Builds the beta and P ladders of a problem with the paper's adaptive schedule
 * (Appendix, Algorithm 2), so that adjacent replicas swap at similar rates:
 *   - the first column (penalty P0) adds rows from beta0, each one step
 *     alpha_beta / sigma_E above the last, until a row's energy spread sigma_E
 *     is <= sigma_min or max_rows rows exist; each row that steps proposes the
 *     next penalty P0 + alpha_P / (beta sigma_g), and the next column takes the
 *     median proposal rounded to an integer;
 *   - every further column repeats the row walk from beta0 at its own penalty
 *     (sigma_E floored at sigma_min), and the schedule stops after the column
 *     whose coldest row has mean g < 1/2, at max_cols columns, or when no row
 *     proposes a penalty (every population had sigma_g = 0);
 *   - beta_i is the median over the columns of row i's beta.
 * A population sample at (beta, P) is n_chain runs of a 1 x 1 context: mcs
 * heat-bath sweeps from the INIT state (one event, no swap), then E = f + P g
 * and g of each chain; sigma_E, sigma_g (divide by n_chain) and mean g come from
 * exact integer sums rounded once to double.  Sample k (in drawing order) uses
 * seed + k.  Every sample is a context on opt's stream and device (opt may be
 * NULL), so the result is bit-reproducible and equal to a CPU restatement.
 * Outputs: beta_out[max_rows] (I_out used), P_out[max_cols] (J_out used),
 * samples_out (may be NULL): the number of population samples drawn.
 * Errors: INVALID_ARG (parameters out of range: beta0, sigma_min, the alphas
 * > 0 and finite, P0 >= 0, caps >= 1, n_chain >= 2, mcs >= 1; a penalty beyond
 * int32), and any error of pt2d_create / pt2d_run / pt2d_read. */
typedef struct pt2d_schedule_params {
    double beta0;        /* first inverse temperature, in 1 / coupling units          */
    int32_t P0;          /* penalty of the first column, coupling units              */
    int32_t max_rows;    /* cap on I                                                 */
    int32_t max_cols;    /* cap on J                                                 */
    int32_t n_chain;     /* chains per population sample                             */
    double sigma_min;    /* energy spread at which the first column stops adding rows */
    double alpha_beta;   /* learning rate of the beta steps                          */
    double alpha_P;      /* learning rate of the penalty steps                       */
    int32_t mcs;         /* sweeps per population sample                             */
    uint64_t seed;       /* sample k uses seed + k                                   */
} pt2d_schedule_params;

int pt2d_adaptive_schedule(const pt2d_instance *inst, const pt2d_schedule_params *prm,
                           const pt2d_options *opt, float *beta_out, int32_t *I_out,
                           int32_t *P_out, int32_t *J_out, int64_t *samples_out);

/* ---- one-shot run without device allocation ------------------------------ */
/* The paper has no counterpart to this entry point; it exists for callers that
 * cannot call cudaMalloc, for example a host program whose device memory is
 * already fully reserved by its own pool or allocator (a serving process that
 * claims the GPU's memory up front), or a loop that must not pay for the
 * implicit synchronisation and latency of a device allocation.
 *
 * It runs create + run + read + destroy of the context API in one call, with
 * every device buffer carved from a file-scope device array of
 * PT2D_NOALLOC_SCRATCH_BYTES bytes that the library holds on each GPU it is
 * used on until the process exits.  It calls no cudaMalloc or cudaFree.
 *  - Every call checks that the current device is an sm_103 GPU
 *    (PT2D_ERR_UNSUPPORTED otherwise) and then looks up the array's device
 *    address on that device.  The look-up is repeated on every call, so the
 *    address stays right after cudaDeviceReset or under another context of
 *    the same device; the first call on a device (and the first after a
 *    reset) also loads the library's device code there, so make it before any
 *    stream capture.
 *  - All calls share the array and it keeps the previous call's contents; each
 *    call clears the part it uses before starting.  Calls whose GPU work
 *    overlaps (several streams or host threads at once) race on the array and
 *    give undefined results: serialise them.
 *  - Problems whose context would need more than PT2D_NOALLOC_SCRATCH_BYTES of
 *    device memory (see pt2d_workspace_size with trace_capacity 0) are
 *    rejected with PT2D_ERR_INVALID_ARG before any device work.
 * Arguments are those of pt2d_create and pt2d_run (trace off); outputs are
 * host buffers or NULL: states int8 [runs][I*J][n], walker_at int32
 * [runs][I*J], f and g int64 [runs][I*J], as from pt2d_read.  Synchronous on
 * `stream` (NULL = default stream).  Errors: those of pt2d_create, pt2d_run
 * and pt2d_read. */
#define PT2D_NOALLOC_SCRATCH_BYTES (8u << 20)
int pt2d_run_noalloc(const pt2d_instance *inst, int32_t I, const float *beta, int32_t J,
                     const int32_t *P, int32_t runs, int64_t sweeps, int32_t swap_interval,
                     uint64_t seed, void *stream, int8_t *states, int32_t *walker_at, int64_t *f,
                     int64_t *g);

/* ---- host-side compiler helpers (section "Graph sparsification") ------- */
/* Copy-chain sparsification of a dense symmetric int16 logical coupling
 * matrix Jq[N*N] (zero diagonal).  Logical node i with K_i copies owns
 * physical ids offset_i..offset_i+K_i-1 chained by links; its nonzero
 * neighbours in ascending order are dealt round-robin over its copies,
 * skipping full copies; logical edge (i,j) becomes one coupling between the
 * copy of i that received j and the copy of j that received i.
 * rule: PT2D_SPARSIFY_FIXED (K = param), PT2D_SPARSIFY_MAX_EDGES (at most
 * param original edges per copy), PT2D_SPARSIFY_MAX_DEGREE (physical degree
 * including links <= param).
 * Call once with all output pointers NULL to get n, nnz_cp, nnz_lk; then again
 * with arrays of those sizes: cp_ptr[n+1], cp_col[nnz_cp], cp_J[nnz_cp],
 * lk_ptr[n+1], lk_col[nnz_lk], copy_of[n] (rows sorted by column).
 * Errors: INVALID_ARG (asymmetric matrix, bad rule). */
#define PT2D_SPARSIFY_FIXED 0
#define PT2D_SPARSIFY_MAX_EDGES 1
#define PT2D_SPARSIFY_MAX_DEGREE 2
int pt2d_sparsify(int32_t N, const int16_t *Jq, int32_t rule, int32_t param, int32_t *n,
                  int64_t *nnz_cp, int64_t *nnz_lk, int32_t *cp_ptr, int32_t *cp_col,
                  int16_t *cp_J, int32_t *lk_ptr, int32_t *lk_col, int32_t *copy_of);

/* Greedy colouring of a physical instance (the rule described above).
 * color: [n] output; *n_colors: number of colours.  Errors: INVALID_ARG. */
int pt2d_greedy_color(const pt2d_instance *inst, int32_t *color, int32_t *n_colors);

/* Penalty terms of one-hot constraints: for groups c of spins (binary x_a =
 * [s_a = +1]), g = sum_c (sum_{a in c} x_a - 1)^2, written in the links form
 * of pt2d_instance: each group adds (m - 1)^2 to g0, 2 - m to k_a of each of
 * its m members and -1 to K of each pair of members (pairs in several groups
 * add up; pairs that sum to 0 are dropped).  Groups: CSR grp_ptr[n_groups+1],
 * grp_col (spin ids in [0, n), no repeats within a group).  Outputs lk_ptr[n+1],
 * lk_col / lk_w [cap] (sorted by column per row), *nnz, hk[n], *g0.
 * Errors: INVALID_ARG (bad groups, NULL outputs, cap too small: *nnz still
 * receives the size needed). */
int pt2d_onehot_penalty(int32_t n, int32_t n_groups, const int32_t *grp_ptr, const int32_t *grp_col,
                        int32_t *lk_ptr, int32_t *lk_col, int16_t *lk_w, int32_t cap, int32_t *nnz,
                        int32_t *hk, int64_t *g0);

/* Penalty terms of linear equality constraints (the general g >= 0 of Eq. 1
 * beyond copy links): for constraints c over spins a with integer
 * coefficients A_a and right-hand side b_c (binary x_a = [s_a = +1]),
 *   g = sum_c (sum_{a in c} A_a x_a - b_c)^2,
 * zero exactly on the feasible states.  Written in the links form of
 * pt2d_instance with S = sum_{a in c} A_a: each constraint adds (S - b_c)^2 to
 * g0, A_a (2 b_c - S) to k_a of each member and -A_a A_b to K of each pair of
 * members (pairs in several constraints add up; pairs that sum to 0 are
 * dropped).  One-hot groups are A = 1, b = 1 (pt2d_onehot_penalty).  An
 * inequality sum A_a x_a <= b (b >= 0) takes slack spins z_t with
 * coefficients 1, 2, 4, ..., 2^(T-1) and b + 1 - 2^T, T = floor(log2(b + 1)),
 * whose sum takes every value 0..b, and becomes the equality
 * sum A_a x_a + sum c_t z_t = b over the spins and the slacks.
 * Constraints: CSR con_ptr[n_cons+1], con_col (spin ids in [0, n), no repeats
 * within a constraint), coef (int32, parallel to con_col), rhs[n_cons] (int64).
 * Outputs as pt2d_onehot_penalty.  Errors: INVALID_ARG (bad constraints, NULL
 * inputs or outputs, cap too small: *nnz still receives the size needed; a
 * weight K outside int16, a field k outside int32, |b| or g0 above 2^62). */
int pt2d_equality_penalty(int32_t n, int32_t n_cons, const int32_t *con_ptr, const int32_t *con_col,
                          const int32_t *coef, const int64_t *rhs, int32_t *lk_ptr, int32_t *lk_col,
                          int16_t *lk_w, int32_t cap, int32_t *nnz, int32_t *hk, int64_t *g0);

/* ---- test hook ------------------------------------------------------------ */
/* Host-side fault injection for failure-handling tests: the next `count`
 * device allocations of context workspaces and batch pools fail as if the
 * device were out of memory (pt2d_create / pt2d_batch_create return
 * PT2D_ERR_OOM and leave nothing allocated).  count <= 0 clears it.
 * Process-wide; returns the count that was pending. */
int32_t pt2d_debug_fail_allocations(int32_t count);

/* ---- diagnostics: the device arithmetic, element-wise -------------------- */
/* Each runs the same device functions the sweep and swap kernels use, on
 * `count` elements given in host memory, and copies results back (synchronous,
 * default device, legacy stream).  Errors: INVALID_ARG, CUDA, UNSUPPORTED. */
int pt2d_diag_philox(const uint32_t *ctr /*[count][4]*/, const uint32_t *key /*[count][2]*/,
                     uint32_t *out /*[count][4]*/, int64_t count);
int pt2d_diag_pt_exp(const float *x, float *y, int64_t count);
int pt2d_diag_heatbath(const float *beta, const int32_t *H, const uint32_t *r, int8_t *spin,
                       int64_t count);
int pt2d_diag_swap_accept(const float *x, const uint32_t *r, int8_t *accept, int64_t count);

/* Read-bandwidth probe: `iters` passes of 16-byte loads (cached in L2 only)
 * over `bytes` of device memory at device_buf (16-byte aligned, bytes a
 * multiple of 16), on the legacy default stream; *ms receives the time of all
 * passes from CUDA events.  device_out: 4 bytes of device memory the probe may
 * write (it keeps the loads alive; the value is meaningless).  A buffer well
 * below the L2 size measures the L2 read ceiling after a warm-up call, one well
 * above it the HBM read ceiling.  Errors: INVALID_ARG, UNSUPPORTED (no
 * device), CUDA. */
int pt2d_diag_read_bandwidth(const void *device_buf, size_t bytes, int32_t iters, void *device_out, float *ms);

#ifdef __cplusplus
}
#endif

#endif /* PT2D_H */
