// Batched persistent 2D-PT kernel: many independent runs of many instances of
// uneven size, each with its own ladders and seed.
//
// One launch advances every run by one swap event of Algorithm 1.  A run's
// replicas are split into slabs (a power-of-two number of walkers, the whole
// run when it fits in shared memory); a slab of one run is the unit of work.
// Persistent CTAs (as many as fit on the SMs at the launch's shared memory)
// take slabs from an atomic counter over a list sorted by decreasing run
// size and, for their slab, perform the sweep block of the event (colour
// classes separated by __syncthreads, the slab's spins in shared memory when
// they fit) and f and g of the final sweep.  The CTA that completes the last
// slab of a run, found with a fence and an atomic counter so that nothing ever
// waits, performs the run's swap event and bottom-right record.  The arithmetic
// (keys, decisions, swaps) is that of the plain kernels, so every run follows
// exactly the trajectory of a plain context with the same instance, ladders,
// seed and run index.  Events are chained by replaying launches from a CUDA
// graph.
#include <cstdint>

#include "pt2d_batch.h"
#include "pt2d_device.cuh"
#include "pt2d_internal.h"
#include "pt2d_sweep.cuh"
#include "pt2d_wide.cuh"

namespace pt2d {
namespace {

constexpr int kMaxR = kBatchMaxReplicas;

// The swap event and record of one run, by the CTA that finished its last slab.
// Reads other CTAs' writes of this launch through L2 (ld.global.cg).
template <int DC, int DL>
__device__ void run_swap(const BatchArgs &a, const BatchRun &d, int run_index, uint8_t *small) {
    uint8_t *pool = a.pool;
    const int n = d.n, Rp = d.Rp, R = d.R, I = d.I, J = d.J;
    int *s_at = reinterpret_cast<int *>(small);                      // [kMaxR]
    long long *s_f = reinterpret_cast<long long *>(s_at + kMaxR);    // [kMaxR]
    int *s_g = reinterpret_cast<int *>(s_f + kMaxR);                 // [kMaxR]
    float *s_beta = reinterpret_cast<float *>(s_g + kMaxR);          // [kMaxR]
    int *s_P = reinterpret_cast<int *>(s_beta + kMaxR);              // [kMaxR]
    __shared__ int s_copy;
    int64_t *sc = reinterpret_cast<int64_t *>(pool + d.scalars);
    int32_t *g_at = reinterpret_cast<int32_t *>(pool + d.walker_at);
    const long long *g_f = reinterpret_cast<const long long *>(pool + d.fg);
    const int *g_g = reinterpret_cast<const int *>(pool + d.fg + 8 * Rp);
    float *w_beta = reinterpret_cast<float *>(pool + d.wparam);
    int32_t *w_P = reinterpret_cast<int32_t *>(pool + d.wparam + 4 * Rp);
    int64_t *acc_P = reinterpret_cast<int64_t *>(pool + d.stats);
    int64_t *acc_B = acc_P + R;
    int64_t *sum_f = acc_B + R;
    int64_t *sum_g = sum_f + R;
    int64_t *n_feas = sum_g + R;
    int64_t *trace_f = reinterpret_cast<int64_t *>(pool + d.trace);
    int64_t *trace_g = trace_f + d.trace_cap;
    int8_t *best_state = reinterpret_cast<int8_t *>(pool + d.best_state);
    const int8_t *S = reinterpret_cast<const int8_t *>(pool + d.state);
    const int *recs = reinterpret_cast<const int *>(pool + d.rec);
    const int pid_at = DC == 0 ? d.dc + d.dl : DC + DL;

    const bool inited = sc[kScInited] != 0;
    const int64_t nev = sc[kScEvents] + 1;
    for (int i = threadIdx.x; i < I; i += blockDim.x) s_beta[i] = reinterpret_cast<const float *>(pool + d.beta)[i];
    for (int j = threadIdx.x; j < J; j += blockDim.x) s_P[j] = reinterpret_cast<const int32_t *>(pool + d.P)[j];
    for (int s = threadIdx.x; s < R; s += blockDim.x) s_at[s] = inited ? __ldcg(g_at + s) : s;
    for (int w = threadIdx.x; w < Rp; w += blockDim.x) {
        s_f[w] = __ldcg(g_f + w);
        s_g[w] = __ldcg(g_g + w);
    }
    __syncthreads();
    swap_pairs(s_at, [&](int w) { return s_f[w]; }, [&](int w) { return s_g[w]; }, s_beta, s_P, I, J,
               static_cast<uint32_t>(d.run), nev, event_dir_p(nev, d.swap_mode), d.k0, d.k1, acc_P, acc_B);
    __syncthreads();
    for (int w = threadIdx.x; w < Rp; w += blockDim.x) {  // pad walkers keep beta = 0, P = 0
        w_beta[w] = 0.0f;
        w_P[w] = 0;
    }
    __syncthreads();
    for (int s = threadIdx.x; s < R; s += blockDim.x) {
        const int w = s_at[s];
        g_at[s] = w;
        w_beta[w] = s_beta[s / J];
        w_P[w] = s_P[s % J];
        sum_f[s] += s_f[w];
        sum_g[s] += s_g[w];
        n_feas[s] += (s_g[w] == 0);
    }
    if (threadIdx.x == 0) {
        if (!inited) {
            sc[kScBestF] = INT64_MAX;
            sc[kScBestEvent] = -1;
            sc[kScSolvedEvent] = -1;
        }
        const int wl = s_at[record_slot(s_at, [&](int w) { return s_f[w]; }, [&](int w) { return s_g[w]; },
                                        I, J, d.swap_mode)];
        const long long fl = s_f[wl];
        const int gl = s_g[wl];
        if (nev - 1 < d.trace_cap) {
            trace_f[nev - 1] = fl;
            trace_g[nev - 1] = gl;
        }
        int copy = -1;
        if (gl == 0 && fl < sc[kScBestF]) {
            sc[kScBestF] = fl;
            sc[kScBestEvent] = nev;
            copy = wl;
        }
        if (sc[kScSolvedEvent] < 0 && gl == 0 && fl <= sc[kScTarget]) sc[kScSolvedEvent] = nev;
        sc[kScSweeps] += a.interval;
        sc[kScEvents] = nev;
        sc[kScInited] = 1;
        a.status[2 * run_index] = sc[kScSolvedEvent];
        a.status[2 * run_index + 1] = nev;
        *reinterpret_cast<int32_t *>(pool + d.counter) = 0;
        s_copy = copy;
    }
    __syncthreads();
    if (s_copy >= 0) {
        const int wc = s_copy;
        for (int pos = threadIdx.x; pos < n; pos += blockDim.x)
            best_state[recs[static_cast<int64_t>(pos) * d.rec_vec * 4 + pid_at]] =
                __ldcg(S + static_cast<int64_t>(pos) * Rp + wc);
    }
}

// The sweep block of one event for one slab of a runtime-degree run (wide
// records, optional penalty terms; colour classes separated by __syncthreads).
// fetch(row) / fetch_link(row) give the quad's spin word of a neighbour /
// copy-link row, store(pos, word) writes the new word.  The run's ten Philox
// round keys are read from shared memory, two rounds per 16-byte load: the
// wide records already need more registers than the CTA allows, and holding
// the keys too made the kernel spill (22 % slower).
template <int DC, int DL, typename Fetch, typename FetchLink, typename Store>
__device__ __forceinline__ void slab_sweeps(const BatchArgs &a, const BatchRun &d, const int4 *rec,
                                            const int32_t *cofs, const Quad &q, Fetch fetch,
                                            FetchLink fetch_link, Store store, int grp, int G,
                                            uint32_t lq, int64_t sweeps_done, const uint4 *round_keys) {
    static_assert(DC == 0, "specialised records take slab_sweeps8 or slab_event_bits8");
    const KeysShared keys{round_keys};
    const uint32_t c3 = (static_cast<uint32_t>(d.run) << 4) | kTagSweep;
    for (int t = 0; t < a.interval; ++t) {
        const uint32_t sweep = static_cast<uint32_t>(sweeps_done + t);
        for (int c = 0; c < d.C; ++c) {
            const int beg = __ldg(cofs + c), end = __ldg(cofs + c + 1);
            for (int pos = beg + grp; pos < end; pos += G) {
                const int dc = d.dc, dl = d.dl;
                const int jo = wide_jpack_offset(dc, dl), ko = jo + dc / 2;
                const int *rc = reinterpret_cast<const int *>(rec) + static_cast<int64_t>(pos) * d.rec_vec * 4;
                int j0, j1, j2, j3;  // sum_k J_k s_k per walker
                wide_coupling_sums<true>(rc, dc, jo, fetch, j0, j1, j2, j3);
                const int h2 = __ldg(rc + dc + dl + 1);
                const int kk = d.penalty ? __ldg(rc + ko + dl) : 0;
                int l0 = kk, l1 = kk, l2 = kk, l3 = kk;
                for (int k = 0; k < dl; ++k) {
                    const uint32_t y = fetch_link(__ldg(rc + dc + k));
                    const int w = d.penalty ? __ldg(rc + ko + k) : 1;
                    l0 += w * sbyte<0>(y);
                    l1 += w * sbyte<1>(y);
                    l2 += w * sbyte<2>(y);
                    l3 += w * sbyte<3>(y);
                }
                const uint4 r = keys(make_uint4(static_cast<uint32_t>(__ldg(rc + dc + dl)), sweep, lq, c3));
                store(pos, decide_fields(q, h2 + 2 * j0 + q.p0 * l0, h2 + 2 * j1 + q.p1 * l1,
                                         h2 + 2 * j2 + q.p2 * l2, h2 + 2 * j3 + q.p3 * l3, r));
            }
            __syncthreads();
        }
    }
}

// The sweep block of one event for one int8 slab of a run with specialised
// records, 8 walkers (two quads) per thread: one 8-byte fetch per neighbour and
// two Philox calls per position that share each shared-memory load of the
// run's round keys (the scheme of k_sweep_smem with 8 walkers a thread; 5 %
// faster than 4 walkers a thread with the keys held in registers, which took
// 20 of the 64 registers 1024 threads allow and spilled).  A missing link
// points at the slab's zero row.
template <int DC, int DL, typename Fetch8, typename Store8>
__device__ __forceinline__ void slab_sweeps8(const BatchArgs &a, const BatchRun &d, const int4 *rec,
                                             const int32_t *cofs, const Quad &qa, const Quad &qb,
                                             Fetch8 fetch8, Store8 store8, int grp, int G, uint32_t lq,
                                             int64_t sweeps_done, const uint4 *round_keys) {
    const uint32_t c3 = (static_cast<uint32_t>(d.run) << 4) | kTagSweep;
    for (int t = 0; t < a.interval; ++t) {
        const uint32_t sweep = static_cast<uint32_t>(sweeps_done + t);
        for (int c = 0; c < d.C; ++c) {
            const int beg = __ldg(cofs + c), end = __ldg(cofs + c + 1);
            for (int pos = beg + grp; pos < end; pos += G) {
                Rec<DC, DL> rc;
                rc.load(rec, pos);
                uint32_t xa[DC], xb[DC], ya[DL], yb[DL];
#pragma unroll
                for (int k = 0; k < DC; ++k) {
                    const uint2 w = fetch8(rc.nb(k));
                    xa[k] = w.x;
                    xb[k] = w.y;
                }
#pragma unroll
                for (int l = 0; l < DL; ++l) {
                    const uint2 w = fetch8(rc.lk(l));
                    ya[l] = w.x;
                    yb[l] = w.y;
                }
                const uint32_t id = static_cast<uint32_t>(rc.pid());
                uint4 ra = make_uint4(id, sweep, lq, c3), rb = make_uint4(id, sweep, lq + 1, c3);
                philox_pair_shared(round_keys, ra, rb);
                store8(pos, make_uint2(decide4<DC, DL>(rc, qa, xa, ya, ra), decide4<DC, DL>(rc, qb, xb, yb, rb)));
            }
            __syncthreads();
        }
    }
}

// f and g of the final sweep for the slab's walkers (Eq. 1), accumulated into
// s_F / s_G (shared, zeroed by the caller) at the thread's four walkers.
template <int DC, int DL, typename Fetch>
__device__ __forceinline__ void slab_energies(const BatchRun &d, const int4 *rec, Fetch fetch, int grp,
                                              int G, int lane_off, long long *s_F, int *s_G) {
    const int n = d.n;
    long long F0 = 0, F1 = 0, F2 = 0, F3 = 0;
    int g0 = 0, g1 = 0, g2 = 0, g3 = 0;
    for (int pos = grp; pos < n; pos += G) {
        if constexpr (DC == 0) {
            const int dc = d.dc, dl = d.dl;
            const int jo = wide_jpack_offset(dc, dl), ko = jo + dc / 2;
            const int *rc = reinterpret_cast<const int *>(rec) + static_cast<int64_t>(pos) * d.rec_vec * 4;
            const uint32_t xs = fetch(pos);
            int j0, j1, j2, j3;
            wide_coupling_sums<true>(rc, dc, jo, fetch, j0, j1, j2, j3);
            const int h4 = 2 * __ldg(rc + dc + dl + 1);
            F0 += static_cast<long long>(sbyte<0>(xs)) * (h4 + 2 * j0);
            F1 += static_cast<long long>(sbyte<1>(xs)) * (h4 + 2 * j1);
            F2 += static_cast<long long>(sbyte<2>(xs)) * (h4 + 2 * j2);
            F3 += static_cast<long long>(sbyte<3>(xs)) * (h4 + 2 * j3);
            // twice g: weighted links from both ends, twice k of a down spin
            for (int k = 0; k < dl; ++k) {
                const int lp = __ldg(rc + dc + k);
                if (lp == n) continue;  // padding link
                const uint32_t y = fetch(lp);
                const int w = d.penalty ? __ldg(rc + ko + k) : 1;
                g0 += w * (sbyte<0>(xs) != sbyte<0>(y));
                g1 += w * (sbyte<1>(xs) != sbyte<1>(y));
                g2 += w * (sbyte<2>(xs) != sbyte<2>(y));
                g3 += w * (sbyte<3>(xs) != sbyte<3>(y));
            }
            if (d.penalty) {
                const int k2 = 2 * __ldg(rc + ko + dl);
                g0 += sbyte<0>(xs) < 0 ? k2 : 0;
                g1 += sbyte<1>(xs) < 0 ? k2 : 0;
                g2 += sbyte<2>(xs) < 0 ? k2 : 0;
                g3 += sbyte<3>(xs) < 0 ? k2 : 0;
            }
        } else {
        Rec<DC, DL> rc;
        rc.load(rec, pos);
        const uint32_t xs = fetch(pos);
        const int h4 = 2 * rc.h2();
        int c0 = h4, c1 = h4, c2 = h4, cc = h4;
#pragma unroll
        for (int k = 0; k < DC; ++k) {
            const uint32_t x = fetch(rc.nb(k));
            const int j2 = rc.j2(k);
            c0 += j2 * sbyte<0>(x);
            c1 += j2 * sbyte<1>(x);
            c2 += j2 * sbyte<2>(x);
            cc += j2 * sbyte<3>(x);
        }
        F0 += static_cast<long long>(sbyte<0>(xs)) * c0;
        F1 += static_cast<long long>(sbyte<1>(xs)) * c1;
        F2 += static_cast<long long>(sbyte<2>(xs)) * c2;
        F3 += static_cast<long long>(sbyte<3>(xs)) * cc;
#pragma unroll
        for (int l = 0; l < DL; ++l) {
            if (rc.lk(l) == n) continue;  // padding link
            const uint32_t y = fetch(rc.lk(l));
            g0 += sbyte<0>(xs) != sbyte<0>(y);
            g1 += sbyte<1>(xs) != sbyte<1>(y);
            g2 += sbyte<2>(xs) != sbyte<2>(y);
            g3 += sbyte<3>(xs) != sbyte<3>(y);
        }
        }
    }
    unsigned long long *uf = reinterpret_cast<unsigned long long *>(s_F);
    atomicAdd(uf + lane_off + 0, static_cast<unsigned long long>(F0));
    atomicAdd(uf + lane_off + 1, static_cast<unsigned long long>(F1));
    atomicAdd(uf + lane_off + 2, static_cast<unsigned long long>(F2));
    atomicAdd(uf + lane_off + 3, static_cast<unsigned long long>(F3));
    atomicAdd(s_G + lane_off + 0, g0);
    atomicAdd(s_G + lane_off + 1, g1);
    atomicAdd(s_G + lane_off + 2, g2);
    atomicAdd(s_G + lane_off + 3, g3);
}

// Initial spin word of one quad at one position (Algorithm 1 input S0, the
// init stream of the plain kernels).
template <int DC, int DL>
__device__ __forceinline__ uint32_t init_word(const BatchRun &d, const int4 *rec, int pos, uint32_t lq) {
    const int pid_at = DC == 0 ? d.dc + d.dl : DC + DL;
    const uint32_t pid = static_cast<uint32_t>(
        reinterpret_cast<const int *>(rec)[static_cast<int64_t>(pos) * d.rec_vec * 4 + pid_at]);
    const uint4 r = philox4x32_10(make_uint4(pid, 0u, lq, (static_cast<uint32_t>(d.run) << 4) | kTagInit),
                                  d.k0, d.k1);
    return pack_signs(r.x < 0x80000000u ? -1.0f : 1.0f, r.y < 0x80000000u ? -1.0f : 1.0f,
                      r.z < 0x80000000u ? -1.0f : 1.0f, r.w < 0x80000000u ? -1.0f : 1.0f);
}

// Sweeps and f/g of one slab of int8 spins, held in shared memory (SMEM: the
// slab is SW columns wide there, loaded before and written back after) or
// worked on in place in global memory (row stride Rp).  Separate
// instantiations keep every spin access in one address space.
template <int DC, int DL, bool SMEM>
__device__ __forceinline__ void int8_slab(const BatchArgs &a, const BatchRun &d, const int4 *rec,
                                          const int32_t *cofs, const Quad &q, int8_t *S_g, int col0,
                                          int lane_off, int grp, int G, uint32_t lq, bool inited,
                                          int64_t sweeps_done, const uint4 *keys, long long *s_F,
                                          int *s_G) {
    extern __shared__ __align__(16) uint8_t batch_smem[];
    const int n = d.n, SW = d.sw, QL = SW >> 2;
    const int64_t Rp = d.Rp;
    int8_t *const Sg = S_g + col0;
    int8_t *const Ss = reinterpret_cast<int8_t *>(batch_smem);
    auto word = [&](int row, int byte) -> uint32_t * {
        if constexpr (SMEM)
            return reinterpret_cast<uint32_t *>(Ss + row * SW + byte);
        else
            return reinterpret_cast<uint32_t *>(Sg + row * Rp + byte);
    };
    if (!inited) {
        const int64_t total = static_cast<int64_t>(n) * QL;
        for (int64_t e = threadIdx.x; e < total; e += blockDim.x) {
            const int pos = static_cast<int>(e / QL);
            const int qq = static_cast<int>(e - static_cast<int64_t>(pos) * QL);
            *word(pos, 4 * qq) = init_word<DC, DL>(d, rec, pos, static_cast<uint32_t>((col0 >> 2) + qq));
        }
        for (int i = threadIdx.x; i < SW / 4; i += blockDim.x) *word(n, 4 * i) = 0u;
    } else if (SMEM) {
        if (SW >= 16) {
            const int vec = SW >> 4;
            const int nvec = (n + 1) * vec;
            for (int i = threadIdx.x; i < nvec; i += blockDim.x) {
                const int row = i / vec;
                const int part = i - row * vec;
                reinterpret_cast<uint4 *>(Ss)[i] = *reinterpret_cast<const uint4 *>(Sg + row * Rp + 16 * part);
            }
        } else {  // 8-walker slabs: one 8-byte word per row
            for (int row = threadIdx.x; row <= n; row += blockDim.x)
                reinterpret_cast<uint2 *>(Ss)[row] = *reinterpret_cast<const uint2 *>(Sg + row * Rp);
        }
    }
    __syncthreads();
    auto fetch = [&](int row) -> uint32_t { return *word(row, lane_off); };
    auto store = [&](int pos, uint32_t w) { *word(pos, lane_off) = w; };
    slab_sweeps<DC, DL>(a, d, rec, cofs, q, fetch, fetch, store, grp, G, lq, sweeps_done, keys);
    if (SMEM) {  // write the slab back (rows 0..n, the zero row included)
        if (SW >= 16) {
            const int vec = SW >> 4;
            const int nvec = (n + 1) * vec;
            for (int i = threadIdx.x; i < nvec; i += blockDim.x) {
                const int row = i / vec;
                const int part = i - row * vec;
                *reinterpret_cast<uint4 *>(Sg + row * Rp + 16 * part) = reinterpret_cast<const uint4 *>(Ss)[i];
            }
        } else {
            for (int row = threadIdx.x; row <= n; row += blockDim.x)
                *reinterpret_cast<uint2 *>(Sg + row * Rp) = reinterpret_cast<const uint2 *>(Ss)[row];
        }
    }
    for (int i = threadIdx.x; i < SW; i += blockDim.x) {
        s_F[i] = 0;
        s_G[i] = 0;
    }
    __syncthreads();
    slab_energies<DC, DL>(d, rec, fetch, grp, G, lane_off, s_F, s_G);
}

// int8_slab with 8 walkers (two quads) per thread, for runs with specialised
// records: the same slab storage, loads, stores and initial state, the sweep
// block of slab_sweeps8, and f and g per quad.
template <int DC, int DL, bool SMEM>
__device__ __forceinline__ void int8_slab8(const BatchArgs &a, const BatchRun &d, const int4 *rec,
                                           const int32_t *cofs, const Quad &qa, const Quad &qb, int8_t *S_g,
                                           int col0, int lane_off, int grp, int G, uint32_t lq, bool inited,
                                           int64_t sweeps_done, const uint4 *keys, long long *s_F, int *s_G) {
    extern __shared__ __align__(16) uint8_t batch_smem[];
    const int n = d.n, SW = d.sw, QL = SW >> 2;
    const int64_t Rp = d.Rp;
    int8_t *const Sg = S_g + col0;
    int8_t *const Ss = reinterpret_cast<int8_t *>(batch_smem);
    // byte `byte` of the slab's row `row` (8-byte aligned for byte = lane_off:
    // rows are SW >= 8 or Rp >= 16 bytes apart, the run's state 256-byte aligned)
    auto at = [&](int row, int byte) -> int8_t * {
        if constexpr (SMEM)
            return Ss + row * SW + byte;
        else
            return Sg + row * Rp + byte;
    };
    if (!inited) {
        const int64_t total = static_cast<int64_t>(n) * QL;
        for (int64_t e = threadIdx.x; e < total; e += blockDim.x) {
            const int pos = static_cast<int>(e / QL);
            const int qq = static_cast<int>(e - static_cast<int64_t>(pos) * QL);
            *reinterpret_cast<uint32_t *>(at(pos, 4 * qq)) =
                init_word<DC, DL>(d, rec, pos, static_cast<uint32_t>((col0 >> 2) + qq));
        }
        for (int i = threadIdx.x; i < SW / 4; i += blockDim.x) *reinterpret_cast<uint32_t *>(at(n, 4 * i)) = 0u;
    } else if (SMEM) {
        if (SW >= 16) {
            const int vec = SW >> 4;
            const int nvec = (n + 1) * vec;
            for (int i = threadIdx.x; i < nvec; i += blockDim.x) {
                const int row = i / vec;
                const int part = i - row * vec;
                reinterpret_cast<uint4 *>(Ss)[i] = *reinterpret_cast<const uint4 *>(Sg + row * Rp + 16 * part);
            }
        } else {  // 8-walker slabs: one 8-byte word per row
            for (int row = threadIdx.x; row <= n; row += blockDim.x)
                reinterpret_cast<uint2 *>(Ss)[row] = *reinterpret_cast<const uint2 *>(Sg + row * Rp);
        }
    }
    __syncthreads();
    auto fetch8 = [&](int row) -> uint2 { return *reinterpret_cast<const uint2 *>(at(row, lane_off)); };
    auto store8 = [&](int pos, uint2 w) { *reinterpret_cast<uint2 *>(at(pos, lane_off)) = w; };
    slab_sweeps8<DC, DL>(a, d, rec, cofs, qa, qb, fetch8, store8, grp, G, lq, sweeps_done, keys);
    if (SMEM) {  // write the slab back (rows 0..n, the zero row included)
        if (SW >= 16) {
            const int vec = SW >> 4;
            const int nvec = (n + 1) * vec;
            for (int i = threadIdx.x; i < nvec; i += blockDim.x) {
                const int row = i / vec;
                const int part = i - row * vec;
                *reinterpret_cast<uint4 *>(Sg + row * Rp + 16 * part) = reinterpret_cast<const uint4 *>(Ss)[i];
            }
        } else {
            for (int row = threadIdx.x; row <= n; row += blockDim.x)
                *reinterpret_cast<uint2 *>(Sg + row * Rp) = reinterpret_cast<const uint2 *>(Ss)[row];
        }
    }
    for (int i = threadIdx.x; i < SW; i += blockDim.x) {
        s_F[i] = 0;
        s_G[i] = 0;
    }
    __syncthreads();
    auto fetch_a = [&](int row) -> uint32_t { return *reinterpret_cast<const uint32_t *>(at(row, lane_off)); };
    auto fetch_b = [&](int row) -> uint32_t { return *reinterpret_cast<const uint32_t *>(at(row, lane_off + 4)); };
    slab_energies<DC, DL>(d, rec, fetch_a, grp, G, lane_off, s_F, s_G);
    slab_energies<DC, DL>(d, rec, fetch_b, grp, G, lane_off + 4, s_F, s_G);
}

// Beta and P of the current slots of walkers w0 .. w0 + 3 of a run (a quad).
__device__ __forceinline__ Quad batch_quad(const uint8_t *pool, const BatchRun &d, int w0, bool inited) {
    const float kNegL2E = -1.4426950408889634f;
    float b[4];
    int p[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int w = w0 + k;
        if (inited) {
            b[k] = reinterpret_cast<const float *>(pool + d.wparam)[w];
            p[k] = reinterpret_cast<const int32_t *>(pool + d.wparam + 4 * d.Rp)[w];
        } else {  // walker w starts in slot w
            b[k] = w < d.R ? reinterpret_cast<const float *>(pool + d.beta)[w / d.J] : 0.0f;
            p[k] = w < d.R ? reinterpret_cast<const int32_t *>(pool + d.P)[w % d.J] : 0;
        }
    }
    return Quad{b[0], b[1], b[2], b[3], b[0] * kNegL2E, b[1] * kNegL2E, b[2] * kNegL2E,
                b[3] * kNegL2E, p[0], p[1], p[2], p[3]};
}

// The end of one slab's event: f and g of its walkers (from s_F / s_G) to the
// run's arrays, then the run's swap event when this slab is the last of its run
// to finish (found with a fence and an atomic counter, so nothing waits).
template <int DC, int DL>
__device__ __forceinline__ void slab_finish(const BatchArgs &a, const BatchRun &d, const BatchItem it,
                                            uint8_t *small, const long long *s_F, const int *s_G) {
    uint8_t *pool = a.pool;
    const int col0 = it.slab * d.sw;
    __syncthreads();
    {
        int64_t *g_f = reinterpret_cast<int64_t *>(pool + d.fg);
        int32_t *g_g = reinterpret_cast<int32_t *>(pool + d.fg + 8 * d.Rp);
        for (int i = threadIdx.x; i < d.sw; i += blockDim.x) {
            g_f[col0 + i] = -(s_F[i] / 4);
            g_g[col0 + i] = s_G[i] / 2 + d.g0;
        }
    }
    __threadfence();
    __syncthreads();
    __shared__ int s_last;
    if (threadIdx.x == 0) {
        const int done = atomicAdd(reinterpret_cast<int32_t *>(pool + d.counter), 1);
        s_last = (done == d.nslab - 1) ? 1 : 0;
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        run_swap<DC, DL>(a, d, it.run, small);
    }
}

// One event of one int8 slab (shared or global memory) of a run with
// specialised records, 8 walkers per thread: lanes = SW / 8 threads per spin
// row, the thread's quads lq and lq + 1 of the run.
template <int DC, int DL>
__device__ __forceinline__ void slab_event_int8w8(const BatchArgs &a, const BatchItem it, uint8_t *dsm) {
    const BatchRun d = a.runs[it.run];
    uint8_t *pool = a.pool;
    const int SW = d.sw;
    const int lanes = SW >> 3;
    const int lane = threadIdx.x & (lanes - 1);
    const int grp = threadIdx.x / lanes;
    const int G = blockDim.x / lanes;
    const int col0 = it.slab * SW;   // first walker of the slab
    const int lane_off = 8 * lane;   // within the slab
    int8_t *S_g = reinterpret_cast<int8_t *>(pool + d.state);
    const int4 *rec = reinterpret_cast<const int4 *>(pool + d.rec);
    const int32_t *cofs = reinterpret_cast<const int32_t *>(pool + d.cofs);
    const int64_t *sc = reinterpret_cast<const int64_t *>(pool + d.scalars);
    const bool inited = sc[kScInited] != 0;
    const int64_t sweeps_done = sc[kScSweeps];
    const uint32_t lq = static_cast<uint32_t>((col0 >> 2) + 2 * lane);
    const Quad qa = batch_quad(pool, d, col0 + lane_off, inited);
    const Quad qb = batch_quad(pool, d, col0 + lane_off + 4, inited);
    uint8_t *small = dsm + a.smem_state;
    long long *s_F = reinterpret_cast<long long *>(small);
    int *s_G = reinterpret_cast<int *>(s_F + kMaxR);
    __shared__ uint4 s_keys8[5];  // the run's Philox round keys, visible after the next barrier
    stage_round_keys(s_keys8, d.k0, d.k1);
    if (d.mode == 1) {
        int8_slab8<DC, DL, true>(a, d, rec, cofs, qa, qb, S_g, col0, lane_off, grp, G, lq, inited, sweeps_done,
                                 s_keys8, s_F, s_G);
    } else {
        int8_slab8<DC, DL, false>(a, d, rec, cofs, qa, qb, S_g, col0, lane_off, grp, G, lq, inited, sweeps_done,
                                  s_keys8, s_F, s_G);
    }
    slab_finish<DC, DL>(a, d, it, small, s_F, s_G);
}

// One event of one slab of a runtime-degree run: sweeps, f and g, and the run's
// swap when this slab is the last of its run to finish.  The slab's spins are
// int8 in global memory (mode 0), int8 in shared memory (mode 1) or bit-packed
// in shared memory (mode 2: one bit per walker, a thread owns a nibble, a
// 16-entry table expands it to int8 spins, the two nibbles of a byte are merged
// by a shuffle).  Runs with specialised records take slab_event_int8w8 and
// slab_event_bits8.
template <int DC, int DL>
__device__ __forceinline__ void slab_event(const BatchArgs &a, const BatchItem it, uint8_t *dsm) {
    static_assert(DC == 0, "specialised records take slab_event_int8w8 or slab_event_bits8");
    const BatchRun d = a.runs[it.run];
    uint8_t *pool = a.pool;
    const int n = d.n, Rp = d.Rp;
    const int SW = d.sw;
    const int QL = SW >> 2;
    const int lane_q = threadIdx.x & (QL - 1);
    const int grp = threadIdx.x / QL;
    const int G = blockDim.x / QL;
    const int col0 = it.slab * SW;                 // first walker of the slab
    const int lane_off = 4 * lane_q;               // within the slab
    int8_t *S_g = reinterpret_cast<int8_t *>(pool + d.state);
    const int4 *rec = reinterpret_cast<const int4 *>(pool + d.rec);
    const int32_t *cofs = reinterpret_cast<const int32_t *>(pool + d.cofs);
    const int64_t *sc = reinterpret_cast<const int64_t *>(pool + d.scalars);
    const bool inited = sc[kScInited] != 0;
    const int64_t sweeps_done = sc[kScSweeps];
    const uint32_t lq = static_cast<uint32_t>((col0 >> 2) + lane_q);

    const Quad q = batch_quad(pool, d, col0 + lane_off, inited);  // this thread's four walkers
    uint8_t *small = dsm + a.smem_state;
    long long *s_F = reinterpret_cast<long long *>(small);
    int *s_G = reinterpret_cast<int *>(s_F + kMaxR);
    __shared__ uint4 s_keys[5];  // the run's Philox round keys, visible after the next barrier
    stage_round_keys(s_keys, d.k0, d.k1);

    if (d.mode == 2) {
        const int B = SW >> 3;
        const int byte_lane = lane_q >> 1;
        const int nib_shift = (lane_q & 1) * 4;
        extern __shared__ __align__(16) uint8_t batch_bits[];  // the dynamic shared memory
        uint8_t *bits = batch_bits;
        uint32_t *lut = reinterpret_cast<uint32_t *>(batch_bits + (((n + 1) * B + 15) & ~15));
        if (threadIdx.x < 16) lut[threadIdx.x] = word_of_bits(threadIdx.x);
        const int64_t nbytes = static_cast<int64_t>(n + 1) * B;
        for (int64_t i = threadIdx.x; i < nbytes; i += blockDim.x) {
            const int pos = static_cast<int>(i / B);
            const int b = static_cast<int>(i - static_cast<int64_t>(pos) * B);
            uint32_t lo = 0, hi = 0;
            if (pos == n) {
            } else if (!inited) {
                const uint32_t lq0 = static_cast<uint32_t>((col0 >> 2) + 2 * b);
                lo = bits_of_word(init_word<DC, DL>(d, rec, pos, lq0));
                hi = bits_of_word(init_word<DC, DL>(d, rec, pos, lq0 + 1));
            } else {
                const uint2 v = *reinterpret_cast<const uint2 *>(S_g + static_cast<int64_t>(pos) * Rp + col0 + 8 * b);
                lo = bits_of_word(v.x);
                hi = bits_of_word(v.y);
            }
            bits[i] = static_cast<uint8_t>(lo | (hi << 4));
        }
        __syncthreads();
        auto fetch = [&](int row) -> uint32_t { return lut[(bits[row * B + byte_lane] >> nib_shift) & 0xF]; };
        auto fetch_link = [&](int row) -> uint32_t { return row != n ? fetch(row) : 0u; };
        const unsigned pair = 0x3u << (threadIdx.x & 30);
        auto store = [&](int pos, uint32_t w) {
            const uint32_t nib = bits_of_word(w);
            const uint32_t other = __shfl_xor_sync(pair, nib, 1);
            if ((lane_q & 1) == 0) bits[pos * B + byte_lane] = static_cast<uint8_t>(nib | (other << 4));
        };
        slab_sweeps<DC, DL>(a, d, rec, cofs, q, fetch, fetch_link, store, grp, G, lq, sweeps_done, s_keys);
        const int64_t nout = static_cast<int64_t>(n) * B;  // rows 0..n-1 back as int8 spins
        for (int64_t i = threadIdx.x; i < nout; i += blockDim.x) {
            const int64_t row = i / B;
            const int b = static_cast<int>(i - row * B);
            const uint32_t byte = bits[i];
            *reinterpret_cast<uint2 *>(S_g + row * Rp + col0 + 8 * b) = make_uint2(lut[byte & 0xF], lut[byte >> 4]);
        }
        for (int i = threadIdx.x; i < SW; i += blockDim.x) {
            s_F[i] = 0;
            s_G[i] = 0;
        }
        __syncthreads();
        slab_energies<DC, DL>(d, rec, fetch, grp, G, lane_off, s_F, s_G);
    } else if (d.mode == 1) {
        int8_slab<DC, DL, true>(a, d, rec, cofs, q, S_g, col0, lane_off, grp, G, lq, inited, sweeps_done,
                                s_keys, s_F, s_G);
    } else {
        int8_slab<DC, DL, false>(a, d, rec, cofs, q, S_g, col0, lane_off, grp, G, lq, inited, sweeps_done,
                                 s_keys, s_F, s_G);
    }
    slab_finish<DC, DL>(a, d, it, small, s_F, s_G);
}

// One event of one bit-packed slab of a run with specialised records, one byte
// (8 walkers, two quads) per thread: the scheme of k_sweep_bits8.  A 256-entry
// table expands a byte to the two quads' int8 spin words with one 8-byte shared
// load; each position's record and each neighbour byte serve 8 walkers.  Slabs
// are >= 8 walkers and runs a power of two >= 8 wide, so a byte's two quads lie
// in one run.  The round keys are read from shared memory (philox_pair_shared):
// held in registers they took 20 of them and capped the CTA at 512 threads; at
// 896 threads the 1024-instance uneven mix runs 4.6 % faster.
template <int DC, int DL>
__device__ __forceinline__ void slab_event_bits8(const BatchArgs &a, const BatchItem it, uint8_t *dsm) {
    const BatchRun d = a.runs[it.run];
    uint8_t *pool = a.pool;
    const int n = d.n, Rp = d.Rp;
    const int SW = d.sw;
    const int B = SW >> 3;  // bytes per spin row = threads per row
    const int lane_b = threadIdx.x & (B - 1);
    const int grp = threadIdx.x / B;
    const int G = blockDim.x / B;
    const int col0 = it.slab * SW;
    const int lane_off = 8 * lane_b;  // the thread's first walker within the slab
    int8_t *S_g = reinterpret_cast<int8_t *>(pool + d.state);
    const int4 *rec = reinterpret_cast<const int4 *>(pool + d.rec);
    const int32_t *cofs = reinterpret_cast<const int32_t *>(pool + d.cofs);
    const int64_t *sc = reinterpret_cast<const int64_t *>(pool + d.scalars);
    const bool inited = sc[kScInited] != 0;
    const int64_t sweeps_done = sc[kScSweeps];
    const uint32_t lq = static_cast<uint32_t>((col0 >> 2) + 2 * lane_b);
    const Quad qa = batch_quad(pool, d, col0 + lane_off, inited);
    const Quad qb = batch_quad(pool, d, col0 + lane_off + 4, inited);
    uint8_t *small = dsm + a.smem_state;
    long long *s_F = reinterpret_cast<long long *>(small);
    int *s_G = reinterpret_cast<int *>(s_F + kMaxR);
    __shared__ uint4 s_keys[5];  // the run's Philox round keys, visible after the next barrier
    stage_round_keys(s_keys, d.k0, d.k1);
    uint8_t *bits = dsm;
    uint2 *lut = reinterpret_cast<uint2 *>(dsm + ((static_cast<int64_t>(n + 1) * B + 15) & ~int64_t{15}));
    for (int i = threadIdx.x; i < 256; i += blockDim.x) lut[i] = make_uint2(word_of_bits(i & 15), word_of_bits(i >> 4));
    const int64_t nbytes = static_cast<int64_t>(n + 1) * B;
    for (int64_t i = threadIdx.x; i < nbytes; i += blockDim.x) {
        const int pos = static_cast<int>(i / B);
        const int b = static_cast<int>(i - static_cast<int64_t>(pos) * B);
        uint32_t lo = 0, hi = 0;
        if (pos == n) {
        } else if (!inited) {
            const uint32_t lq0 = static_cast<uint32_t>((col0 >> 2) + 2 * b);
            lo = bits_of_word(init_word<DC, DL>(d, rec, pos, lq0));
            hi = bits_of_word(init_word<DC, DL>(d, rec, pos, lq0 + 1));
        } else {
            const uint2 v = *reinterpret_cast<const uint2 *>(S_g + static_cast<int64_t>(pos) * Rp + col0 + 8 * b);
            lo = bits_of_word(v.x);
            hi = bits_of_word(v.y);
        }
        bits[i] = static_cast<uint8_t>(lo | (hi << 4));
    }
    __syncthreads();
    const uint32_t c3 = (static_cast<uint32_t>(d.run) << 4) | kTagSweep;
    auto fetch8 = [&](int row) -> uint2 { return lut[bits[row * B + lane_b]]; };
    for (int t = 0; t < a.interval; ++t) {
        const uint32_t sweep = static_cast<uint32_t>(sweeps_done + t);
        for (int c = 0; c < d.C; ++c) {
            const int beg = __ldg(cofs + c), end = __ldg(cofs + c + 1);
            for (int pos = beg + grp; pos < end; pos += G) {
                Rec<DC, DL> rc;
                rc.load(rec, pos);
                uint32_t xa[DC], xb[DC], ya[DL], yb[DL];
#pragma unroll
                for (int k = 0; k < DC; ++k) {
                    const uint2 w = fetch8(rc.nb(k));
                    xa[k] = w.x;
                    xb[k] = w.y;
                }
#pragma unroll
                for (int l = 0; l < DL; ++l) {  // a missing link reads as no spin
                    const uint2 w = rc.lk(l) != n ? fetch8(rc.lk(l)) : make_uint2(0u, 0u);
                    ya[l] = w.x;
                    yb[l] = w.y;
                }
                const uint32_t id = static_cast<uint32_t>(rc.pid());
                uint4 ra = make_uint4(id, sweep, lq, c3), rb = make_uint4(id, sweep, lq + 1, c3);
                philox_pair_shared(s_keys, ra, rb);
                const uint32_t na = bits_of_word(decide4<DC, DL>(rc, qa, xa, ya, ra));
                const uint32_t nb = bits_of_word(decide4<DC, DL>(rc, qb, xb, yb, rb));
                bits[pos * B + lane_b] = static_cast<uint8_t>(na | (nb << 4));
            }
            __syncthreads();
        }
    }
    // rows 0..n-1 back as int8 spins
    const int64_t nout = static_cast<int64_t>(n) * B;
    for (int64_t i = threadIdx.x; i < nout; i += blockDim.x) {
        const int64_t row = i / B;
        const int b = static_cast<int>(i - row * B);
        *reinterpret_cast<uint2 *>(S_g + row * Rp + col0 + 8 * b) = lut[bits[i]];
    }
    for (int i = threadIdx.x; i < SW; i += blockDim.x) {
        s_F[i] = 0;
        s_G[i] = 0;
    }
    __syncthreads();
    // f and g of the final sweep for the thread's 8 walkers (Eq. 1), as in slab_energies
    {
        long long F[8];
        int g[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            F[i] = 0;
            g[i] = 0;
        }
        for (int pos = grp; pos < n; pos += G) {
            Rec<DC, DL> rc;
            rc.load(rec, pos);
            const uint2 xs = fetch8(pos);
            const int h4 = 2 * rc.h2();
            int cs[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) cs[i] = h4;
#pragma unroll
            for (int k = 0; k < DC; ++k) {
                const uint2 x = fetch8(rc.nb(k));
                const int j2 = rc.j2(k);
                cs[0] += j2 * sbyte<0>(x.x);
                cs[1] += j2 * sbyte<1>(x.x);
                cs[2] += j2 * sbyte<2>(x.x);
                cs[3] += j2 * sbyte<3>(x.x);
                cs[4] += j2 * sbyte<0>(x.y);
                cs[5] += j2 * sbyte<1>(x.y);
                cs[6] += j2 * sbyte<2>(x.y);
                cs[7] += j2 * sbyte<3>(x.y);
            }
            F[0] += static_cast<long long>(sbyte<0>(xs.x)) * cs[0];
            F[1] += static_cast<long long>(sbyte<1>(xs.x)) * cs[1];
            F[2] += static_cast<long long>(sbyte<2>(xs.x)) * cs[2];
            F[3] += static_cast<long long>(sbyte<3>(xs.x)) * cs[3];
            F[4] += static_cast<long long>(sbyte<0>(xs.y)) * cs[4];
            F[5] += static_cast<long long>(sbyte<1>(xs.y)) * cs[5];
            F[6] += static_cast<long long>(sbyte<2>(xs.y)) * cs[6];
            F[7] += static_cast<long long>(sbyte<3>(xs.y)) * cs[7];
#pragma unroll
            for (int l = 0; l < DL; ++l) {
                if (rc.lk(l) == n) continue;  // padding link
                const uint2 y = fetch8(rc.lk(l));
                g[0] += sbyte<0>(xs.x) != sbyte<0>(y.x);
                g[1] += sbyte<1>(xs.x) != sbyte<1>(y.x);
                g[2] += sbyte<2>(xs.x) != sbyte<2>(y.x);
                g[3] += sbyte<3>(xs.x) != sbyte<3>(y.x);
                g[4] += sbyte<0>(xs.y) != sbyte<0>(y.y);
                g[5] += sbyte<1>(xs.y) != sbyte<1>(y.y);
                g[6] += sbyte<2>(xs.y) != sbyte<2>(y.y);
                g[7] += sbyte<3>(xs.y) != sbyte<3>(y.y);
            }
        }
        unsigned long long *uf = reinterpret_cast<unsigned long long *>(s_F);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            atomicAdd(uf + lane_off + i, static_cast<unsigned long long>(F[i]));
            atomicAdd(s_G + lane_off + i, g[i]);
        }
    }
    slab_finish<DC, DL>(a, d, it, small, s_F, s_G);
}

// Bit-packed slabs of runs with specialised records (one launch per event,
// beside k_batch, which takes the int8 slabs).
template <int DC, int DL>
__global__ void __launch_bounds__(kBatchBits8Threads, 1) k_batch_bits8(BatchArgs a) {
    extern __shared__ __align__(16) uint8_t dsm[];
    __shared__ int s_item;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(a.queue, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= a.n_items) break;
        slab_event_bits8<DC, DL>(a, a.items[item], dsm);
    }
}

// The runtime-degree instantiation (DC = 0) runs at most 768 threads: at 80
// registers it needs no spills and is 5 % faster than at 1024 threads (64).
// The specialised ones take 8 walkers a thread at up to kBatchInt8Threads.
template <int DC, int DL>
__global__ void __launch_bounds__(DC == 0 ? kBatchGenericThreads : kBatchInt8Threads, 1) k_batch(BatchArgs a) {
    extern __shared__ __align__(16) uint8_t dsm[];
    __shared__ int s_item;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(a.queue, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= a.n_items) break;
        if constexpr (DC == 0) {
            slab_event<DC, DL>(a, a.items[item], dsm);
        } else {
            slab_event_int8w8<DC, DL>(a, a.items[item], dsm);
        }
    }
}

template <int DC, int DL>
cudaError_t launch_batch_variant(const BatchArgs &a, int grid, int threads, size_t smem, cudaStream_t st) {
    k_batch<DC, DL><<<grid, threads, smem, st>>>(a);
    return cudaGetLastError();
}

template <int DC, int DL>
cudaError_t launch_bits8_variant(const BatchArgs &a, int grid, int threads, size_t smem, cudaStream_t st) {
    cudaError_t e = allow_max_dynamic_smem<k_batch_bits8<DC, DL>>();
    if (e != cudaSuccess) return e;
    k_batch_bits8<DC, DL><<<grid, threads, smem, st>>>(a);
    return cudaGetLastError();
}

template <auto kernel>
int blocks_per_sm(int threads, size_t smem) {
    if (allow_max_dynamic_smem<kernel>() != cudaSuccess) return 1;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return nb > 0 ? nb : 1;
}

}  // namespace

int batch_blocks_per_sm(int DC, int DL, bool bits8, int threads, int smem_state) {
    const size_t smem = static_cast<size_t>(smem_state) + batch_small_smem_bytes();
    if (DL != 2) return 1;
    if (bits8) {
        if (DC == 3) return blocks_per_sm<k_batch_bits8<3, 2>>(threads, smem);
        if (DC == 4) return blocks_per_sm<k_batch_bits8<4, 2>>(threads, smem);
        if (DC == 6) return blocks_per_sm<k_batch_bits8<6, 2>>(threads, smem);
        return 1;
    }
    if (DC == 0) return blocks_per_sm<k_batch<0, 0>>(threads, smem);
    if (DC == 3) return blocks_per_sm<k_batch<3, 2>>(threads, smem);
    if (DC == 4) return blocks_per_sm<k_batch<4, 2>>(threads, smem);
    if (DC == 6) return blocks_per_sm<k_batch<6, 2>>(threads, smem);
    return 1;
}

size_t batch_small_smem_bytes() {
    return static_cast<size_t>(kMaxR) * (4 + 8 + 4 + 4 + 4);
}

cudaError_t batch_kernel_attributes(int DC, int DL, int smem_state) {
    if (smem_state < 0 || DL != 2) return cudaErrorInvalidValue;
    if (DC == 0) return allow_max_dynamic_smem<k_batch<0, 0>>();
    if (DC == 3) return allow_max_dynamic_smem<k_batch<3, 2>>();
    if (DC == 4) return allow_max_dynamic_smem<k_batch<4, 2>>();
    if (DC == 6) return allow_max_dynamic_smem<k_batch<6, 2>>();
    return cudaErrorInvalidValue;
}

cudaError_t launch_batch_bits8(const BatchArgs &a, int DC, int DL, int grid, int threads, cudaStream_t st) {
    const size_t smem = static_cast<size_t>(a.smem_state) + batch_small_smem_bytes();
    if (DL != 2) return cudaErrorInvalidValue;
    if (DC == 3) return launch_bits8_variant<3, 2>(a, grid, threads, smem, st);
    if (DC == 4) return launch_bits8_variant<4, 2>(a, grid, threads, smem, st);
    if (DC == 6) return launch_bits8_variant<6, 2>(a, grid, threads, smem, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_batch(const BatchArgs &a, int DC, int DL, int grid, int threads, cudaStream_t st) {
    const size_t smem = static_cast<size_t>(a.smem_state) + batch_small_smem_bytes();
    if (DL != 2) return cudaErrorInvalidValue;
    if (DC == 0) return launch_batch_variant<0, 0>(a, grid, threads, smem, st);
    if (DC == 3) return launch_batch_variant<3, 2>(a, grid, threads, smem, st);
    if (DC == 4) return launch_batch_variant<4, 2>(a, grid, threads, smem, st);
    if (DC == 6) return launch_batch_variant<6, 2>(a, grid, threads, smem, st);
    return cudaErrorInvalidValue;
}

}  // namespace pt2d
