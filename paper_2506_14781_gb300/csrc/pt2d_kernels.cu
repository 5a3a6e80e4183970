// CUDA kernels of the 2D-PT library (sm_103a).
//
//  k_init_spins      initial state S0 from the seeded init stream (Algorithm 1 input)
//  k_init_walkers    walker <-> slot identity, per-walker beta/P, best-state sentinels
//  k_sweep_smem      the sweep block of one event of Algorithm 1 (`nsweeps` heat-bath
//                    sweeps of every walker, colour class by colour class) with the
//                    CTA's replica slab held in shared memory for the whole block, then
//                    f and g of the final sweep (Eq. 1) as an epilogue
//  k_sweep_bits8     the same with the slab bit-packed in shared memory (one bit per
//                    walker), a thread owning a byte of 8 walkers (instances whose int8
//                    slab does not fit); k_sweep_bits: a thread owning a nibble
//  k_sweep_global    the same with the slab in global memory (instances whose slab does
//                    not fit in shared memory)
//  k_swap_event      one swap event per run: P-swaps (Eq. 2) or beta-swaps (Eq. 3) on
//                    odd/even pairs, then the bottom-right record (Algorithm 1)
//
// Sweep tiling.  Walkers evolve independently between swap events, so a CTA owns a
// slab of SW = 4*QL walker columns for every spin and runs all sweeps of the event
// with only __syncthreads() between colour classes; no grid-wide barrier is needed.
// A thread owns one quad (4 consecutive columns = one Philox call per spin) and keeps
// the quad's beta and P in registers for the whole launch.  QL lanes cover one spin
// row segment (4*QL bytes); the CTA's QL-lane groups take different spins of the
// current colour class.  Per spin the neighbour list is one packed record
// (positions, spin id, 2h, 2J) read with 16-byte loads.
//
// These kernels take the specialised record layouts (coupling width 3, 4 or 6,
// two copy links).  Runtime degrees are swept by pt2d_generic.cu, instances
// with small degrees and general penalty terms by pt2d_penalty.cu.
#include <cstdint>

#include "pt2d_device.cuh"
#include "pt2d_internal.h"
#include "pt2d_sweep.cuh"

namespace pt2d {
namespace {

// Per-walker f and g of the CTA's slab (epilogue of the sweep kernels); the
// thread owns NQ quads, its walkers are wbase .. wbase + 4 NQ - 1 of the slab.
// F = sum_a s_a (sum_b 2J_ab s_b + 2 * 2h_a) = 4 (sum_{a<b} J s s + sum h s), f = -F/4;
// g counts each broken link from both ends (padding links point at the zero row).
template <int DC, int DL, int NQ, typename Fetch, typename Own>
__device__ __forceinline__ void energies(const Layout &L, const Walkers &wk, Fetch fetch, Own own,
                                         int wbase, int grp, int G, int slab, int64_t col0) {
    __shared__ long long s_F[kMaxSlab];
    __shared__ int s_g[kMaxSlab];
    for (int i = threadIdx.x; i < slab; i += blockDim.x) {
        s_F[i] = 0;
        s_g[i] = 0;
    }
    __syncthreads();
    long long F[4 * NQ];
    int g[4 * NQ];
#pragma unroll
    for (int i = 0; i < 4 * NQ; ++i) {
        F[i] = 0;
        g[i] = 0;
    }
    for (int pos = grp; pos < L.n; pos += G) {
        Rec<DC, DL> rc;
        rc.load(L.rec, pos);
        const int h4 = 2 * rc.h2();
#pragma unroll
        for (int h = 0; h < NQ; ++h) {
            const uint32_t xs = own(pos, h);
            int c0 = h4, c1 = h4, c2 = h4, c3 = h4;
#pragma unroll
            for (int k = 0; k < DC; ++k) {
                const uint32_t x = fetch(rc.nb(k), h);
                const int j = rc.j2(k);
                c0 += j * sbyte<0>(x);
                c1 += j * sbyte<1>(x);
                c2 += j * sbyte<2>(x);
                c3 += j * sbyte<3>(x);
            }
            F[4 * h + 0] += static_cast<long long>(sbyte<0>(xs)) * c0;
            F[4 * h + 1] += static_cast<long long>(sbyte<1>(xs)) * c1;
            F[4 * h + 2] += static_cast<long long>(sbyte<2>(xs)) * c2;
            F[4 * h + 3] += static_cast<long long>(sbyte<3>(xs)) * c3;
#pragma unroll
            for (int l = 0; l < DL; ++l) {
                if (rc.lk(l) == L.pad_ref) continue;
                const uint32_t y = fetch(rc.lk(l), h);
                g[4 * h + 0] += sbyte<0>(xs) != sbyte<0>(y);
                g[4 * h + 1] += sbyte<1>(xs) != sbyte<1>(y);
                g[4 * h + 2] += sbyte<2>(xs) != sbyte<2>(y);
                g[4 * h + 3] += sbyte<3>(xs) != sbyte<3>(y);
            }
        }
    }
    unsigned long long *sF = reinterpret_cast<unsigned long long *>(s_F);
#pragma unroll
    for (int i = 0; i < 4 * NQ; ++i) {
        atomicAdd(sF + wbase + i, static_cast<unsigned long long>(F[i]));
        atomicAdd(&s_g[wbase + i], g[i]);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < slab; i += blockDim.x) {
        wk.f[col0 + i] = -(s_F[i] / 4);
        wk.g[col0 + i] = s_g[i] / 2 + L.g0;
    }
}

// Sweep block with the slab in shared memory: (n + 1) rows x SW bytes, loaded
// once, swept `nsweeps` times, written back once.  SW >= 16; each thread owns
// WPT = 4 or 8 consecutive walkers of the slab.
template <int DC, int DL, int WPT>
__global__ void __launch_bounds__(WPT == 4 ? 1024 : 768, 1)
    k_sweep_smem(Layout L, Walkers wk, int sw_shift, int32_t quads_per_run, RoundKeys rk,
                 uint32_t sweep0, int32_t nsweeps) {
    extern __shared__ __align__(16) int8_t sm[];
    constexpr int NQ = WPT / 4;
    const int SW = 1 << sw_shift;
    const int lanes = SW / WPT;  // threads per spin row segment
    const int lane = threadIdx.x & (lanes - 1);
    const int grp = threadIdx.x / lanes;
    const int G = blockDim.x / lanes;
    const int64_t col0 = static_cast<int64_t>(blockIdx.x) * SW;
    const int64_t quad = col0 / 4 + static_cast<int64_t>(lane) * NQ;
    const uint32_t run = static_cast<uint32_t>(quad / quads_per_run);
    const uint32_t lq = static_cast<uint32_t>(quad - static_cast<int64_t>(run) * quads_per_run);
    const uint32_t c3 = (run << 4) | kTagSweep;
    // the thread's second quad (WPT = 8) starts the next run when a run holds
    // an odd number of quads
    const uint32_t run_b = static_cast<uint32_t>((quad + 1) / quads_per_run);
    const uint32_t lqb = static_cast<uint32_t>(quad + 1 - static_cast<int64_t>(run_b) * quads_per_run);
    const uint32_t c3b = (run_b << 4) | kTagSweep;
    const int lane_off = WPT * lane;
    const Quad qa = load_quad(wk, col0 + lane_off);
    const Quad qb = NQ == 2 ? load_quad(wk, col0 + lane_off + 4) : qa;
    const KeysConst keys{rk};

    // load the slab, 16 bytes per access
    const int vec_per_row = SW >> 4;
    const int64_t nvec = static_cast<int64_t>(L.n + 1) * vec_per_row;
    for (int64_t i = threadIdx.x; i < nvec; i += blockDim.x) {
        const int64_t row = i / vec_per_row;
        const int part = static_cast<int>(i - row * vec_per_row);
        reinterpret_cast<uint4 *>(sm)[i] =
            *reinterpret_cast<const uint4 *>(L.S + row * L.Wc + col0 + 16 * part);
    }
    __syncthreads();

    // neighbour references in the records are byte offsets row * SW into the slab
    auto fetch4 = [&](int off) -> uint32_t {
        return *reinterpret_cast<const uint32_t *>(sm + off + lane_off);
    };
    auto fetch8 = [&](int off) -> uint2 {
        return *reinterpret_cast<const uint2 *>(sm + off + lane_off);
    };
    for (int t = 0; t < nsweeps; ++t) {
        const uint32_t sweep = sweep0 + static_cast<uint32_t>(t);
        for (int c = 0; c < L.C; ++c) {
            const int beg = __ldg(L.cofs + c), end = __ldg(L.cofs + c + 1);
            for (int pos = beg + grp; pos < end; pos += G) {
                Rec<DC, DL> rc;
                rc.load(L.rec, pos);
                int8_t *dst = sm + (pos << sw_shift) + lane_off;
                if (NQ == 1) {
                    *reinterpret_cast<uint32_t *>(dst) = update4<DC, DL>(rc, qa, fetch4, sweep, lq, c3, keys);
                } else {
                    *reinterpret_cast<uint2 *>(dst) = update8<DC, DL>(rc, qa, qb, fetch8, sweep, lq, c3, lqb, c3b, keys);
                }
            }
            __syncthreads();
        }
    }

    // write the slab back (rows 0..n-1)
    const int64_t nvec_out = static_cast<int64_t>(L.n) * vec_per_row;
    for (int64_t i = threadIdx.x; i < nvec_out; i += blockDim.x) {
        const int64_t row = i / vec_per_row;
        const int part = static_cast<int>(i - row * vec_per_row);
        *reinterpret_cast<uint4 *>(L.S + row * L.Wc + col0 + 16 * part) =
            reinterpret_cast<const uint4 *>(sm)[i];
    }
    auto fetch_q = [&](int off, int h) -> uint32_t {
        return *reinterpret_cast<const uint32_t *>(sm + off + lane_off + 4 * h);
    };
    auto own_q = [&](int pos, int h) -> uint32_t {
        return *reinterpret_cast<const uint32_t *>(sm + (pos << sw_shift) + lane_off + 4 * h);
    };
    energies<DC, DL, NQ>(L, wk, fetch_q, own_q, lane_off, grp, G, SW, col0);
}

// Sweep block with the slab bit-packed in shared memory: (n + 1) rows x SW/8
// bytes, bit k of a byte = spin of one walker (1 = -1), for instances whose
// int8 slab does not fit.  A thread owns one nibble (4 walkers); a 16-entry
// table expands a nibble to four int8 spins so the field and decision code is
// the int8 kernel's; the two nibbles of a byte are merged with one shuffle.
// Missing copy links (a bit cannot hold 0) are skipped by predicate.
template <int DC, int DL>
__global__ void __launch_bounds__(1024, 1) k_sweep_bits(Layout L, Walkers wk, int sw_shift,
                                                        int32_t quads_per_run, RoundKeys rk,
                                                        uint32_t sweep0, int32_t nsweeps) {
    extern __shared__ __align__(16) uint8_t smb[];
    const int SW = 1 << sw_shift;  // walkers per CTA, >= 8
    const int B = SW >> 3;         // bytes per spin row
    const int QL = SW >> 2;        // threads per spin row (two per byte)
    const int lane_q = threadIdx.x & (QL - 1);
    const int grp = threadIdx.x >> (sw_shift - 2);
    const int G = blockDim.x >> (sw_shift - 2);
    const int byte_lane = lane_q >> 1;
    const int nib_shift = (lane_q & 1) * 4;
    const int64_t col0 = static_cast<int64_t>(blockIdx.x) * SW;
    const int64_t quad = col0 / 4 + lane_q;
    const uint32_t run = static_cast<uint32_t>(quad / quads_per_run);
    const uint32_t lq = static_cast<uint32_t>(quad - static_cast<int64_t>(run) * quads_per_run);
    const uint32_t c3 = (run << 4) | kTagSweep;
    const Quad q = load_quad(wk, col0 + 4 * lane_q);
    const KeysConst keys{rk};
    const int n = L.n;
    uint8_t *bits = smb;
    uint32_t *lut = reinterpret_cast<uint32_t *>(smb + ((static_cast<int64_t>(n + 1) * B + 15) & ~15LL));
    if (threadIdx.x < 16) lut[threadIdx.x] = word_of_bits(threadIdx.x);
    // load: 8 int8 spins of global memory -> one byte of bits
    const int64_t nbytes = static_cast<int64_t>(n + 1) * B;
    for (int64_t i = threadIdx.x; i < nbytes; i += blockDim.x) {
        const int64_t row = i / B;
        const int b = static_cast<int>(i - row * B);
        const uint2 v = *reinterpret_cast<const uint2 *>(L.S + row * L.Wc + col0 + 8 * b);
        bits[i] = static_cast<uint8_t>(bits_of_word(v.x) | (bits_of_word(v.y) << 4));
    }
    __syncthreads();

    // neighbour references in the records are byte offsets row * B
    auto fetch = [&](int off) -> uint32_t { return lut[(bits[off + byte_lane] >> nib_shift) & 0xF]; };
    const int pad = L.pad_ref;
    for (int t = 0; t < nsweeps; ++t) {
        const uint32_t sweep = sweep0 + static_cast<uint32_t>(t);
        for (int c = 0; c < L.C; ++c) {
            const int beg = __ldg(L.cofs + c), end = __ldg(L.cofs + c + 1);
            for (int pos = beg + grp; pos < end; pos += G) {
                Rec<DC, DL> rc;
                rc.load(L.rec, pos);
                uint32_t x[DC], y[DL];
#pragma unroll
                for (int k = 0; k < DC; ++k) x[k] = fetch(rc.nb(k));
#pragma unroll
                for (int l = 0; l < DL; ++l) y[l] = rc.lk(l) != pad ? fetch(rc.lk(l)) : 0u;
                const uint4 r = keys(make_uint4(static_cast<uint32_t>(rc.pid()), sweep, lq, c3));
                const uint32_t nib = bits_of_word(decide4<DC, DL>(rc, q, x, y, r));
                const uint32_t other = __shfl_xor_sync(0x3u << (threadIdx.x & 30), nib, 1);
                if ((lane_q & 1) == 0) bits[pos * B + byte_lane] = static_cast<uint8_t>(nib | (other << 4));
            }
            __syncthreads();
        }
    }
    // write back rows 0..n-1 as int8 spins
    const int64_t nb_out = static_cast<int64_t>(n) * B;
    for (int64_t i = threadIdx.x; i < nb_out; i += blockDim.x) {
        const int64_t row = i / B;
        const int b = static_cast<int>(i - row * B);
        const uint32_t byte = bits[i];
        *reinterpret_cast<uint2 *>(L.S + row * L.Wc + col0 + 8 * b) = make_uint2(lut[byte & 0xF], lut[byte >> 4]);
    }
    auto fetch_q = [&](int off, int) -> uint32_t { return fetch(off); };
    auto own_q = [&](int p, int) -> uint32_t { return fetch(p * B); };
    energies<DC, DL, 1>(L, wk, fetch_q, own_q, 4 * lane_q, grp, G, SW, col0);
}

// Bit-packed slab with one byte (8 walkers, two quads) per thread: a 256-entry
// table expands a byte to both quads' int8 spin words with one 8-byte shared
// load, so no nibble shift and no pair shuffle; the byte is written whole.
template <int DC, int DL>
__global__ void __launch_bounds__(kBits8Threads, 1) k_sweep_bits8(Layout L, Walkers wk, int sw_shift,
                                                        int32_t quads_per_run, RoundKeys rk,
                                                        uint32_t sweep0, int32_t nsweeps) {
    extern __shared__ __align__(16) uint8_t smb[];
    const int SW = 1 << sw_shift;  // walkers per CTA, >= 8
    const int B = SW >> 3;         // bytes per spin row = threads per row
    const int lane_b = threadIdx.x & (B - 1);
    const int grp = threadIdx.x >> (sw_shift - 3);
    const int G = blockDim.x >> (sw_shift - 3);
    const int64_t col0 = static_cast<int64_t>(blockIdx.x) * SW;
    const int64_t quad = col0 / 4 + 2 * lane_b;
    const uint32_t run = static_cast<uint32_t>(quad / quads_per_run);
    const uint32_t lq = static_cast<uint32_t>(quad - static_cast<int64_t>(run) * quads_per_run);
    const uint32_t c3 = (run << 4) | kTagSweep;
    const uint32_t run_b = static_cast<uint32_t>((quad + 1) / quads_per_run);
    const uint32_t lqb = static_cast<uint32_t>(quad + 1 - static_cast<int64_t>(run_b) * quads_per_run);
    const uint32_t c3b = (run_b << 4) | kTagSweep;
    const Quad qa = load_quad(wk, col0 + 8 * lane_b);
    const Quad qb = load_quad(wk, col0 + 8 * lane_b + 4);
    const KeysConst keys{rk};
    const int n = L.n;
    uint8_t *bits = smb;
    uint2 *lut = reinterpret_cast<uint2 *>(smb + ((static_cast<int64_t>(n + 1) * B + 15) & ~15LL));
    for (int i = threadIdx.x; i < 256; i += blockDim.x) lut[i] = make_uint2(word_of_bits(i & 15), word_of_bits(i >> 4));
    const int64_t nbytes = static_cast<int64_t>(n + 1) * B;
    for (int64_t i = threadIdx.x; i < nbytes; i += blockDim.x) {
        const int64_t row = i / B;
        const int b = static_cast<int>(i - row * B);
        const uint2 v = *reinterpret_cast<const uint2 *>(L.S + row * L.Wc + col0 + 8 * b);
        bits[i] = static_cast<uint8_t>(bits_of_word(v.x) | (bits_of_word(v.y) << 4));
    }
    __syncthreads();
    auto fetch8 = [&](int off) -> uint2 { return lut[bits[off + lane_b]]; };
    const int pad = L.pad_ref;
    for (int t = 0; t < nsweeps; ++t) {
        const uint32_t sweep = sweep0 + static_cast<uint32_t>(t);
        for (int c = 0; c < L.C; ++c) {
            const int beg = __ldg(L.cofs + c), end = __ldg(L.cofs + c + 1);
            for (int pos = beg + grp; pos < end; pos += G) {
                Rec<DC, DL> rc;
                rc.load(L.rec, pos);
                uint32_t xa[DC], xb[DC], ya[DL], yb[DL];
#pragma unroll
                for (int k = 0; k < DC; ++k) {
                    const uint2 w = fetch8(rc.nb(k));
                    xa[k] = w.x;
                    xb[k] = w.y;
                }
#pragma unroll
                for (int l = 0; l < DL; ++l) {
                    const uint2 w = rc.lk(l) != pad ? fetch8(rc.lk(l)) : make_uint2(0u, 0u);
                    ya[l] = w.x;
                    yb[l] = w.y;
                }
                const uint32_t id = static_cast<uint32_t>(rc.pid());
                const uint4 ra = keys(make_uint4(id, sweep, lq, c3));
                const uint32_t na = bits_of_word(decide4<DC, DL>(rc, qa, xa, ya, ra));
                const uint4 rb = keys(make_uint4(id, sweep, lqb, c3b));
                const uint32_t nb = bits_of_word(decide4<DC, DL>(rc, qb, xb, yb, rb));
                bits[pos * B + lane_b] = static_cast<uint8_t>(na | (nb << 4));
            }
            __syncthreads();
        }
    }
    const int64_t nb_out = static_cast<int64_t>(n) * B;
    for (int64_t i = threadIdx.x; i < nb_out; i += blockDim.x) {
        const int64_t row = i / B;
        const int b = static_cast<int>(i - row * B);
        *reinterpret_cast<uint2 *>(L.S + row * L.Wc + col0 + 8 * b) = lut[bits[i]];
    }
    auto fetch_q = [&](int off, int h) -> uint32_t {
        const uint2 w = fetch8(off);
        return h ? w.y : w.x;
    };
    auto own_q = [&](int p, int h) -> uint32_t { return fetch_q(p * B, h); };
    energies<DC, DL, 2>(L, wk, fetch_q, own_q, 8 * lane_b, grp, G, SW, col0);
}

// Sweep block with the slab in global memory.
template <int DC, int DL>
__global__ void __launch_bounds__(256) k_sweep_global(Layout L, Walkers wk, int ql_shift,
                                                      int32_t quads_per_run, RoundKeys rk,
                                                      uint32_t sweep0, int32_t nsweeps) {
    const int QL = 1 << ql_shift;
    const int lane_q = threadIdx.x & (QL - 1);
    const int grp = threadIdx.x >> ql_shift;
    const int G = blockDim.x >> ql_shift;
    const int64_t quad = static_cast<int64_t>(blockIdx.x) * QL + lane_q;
    const int64_t col = quad * 4;
    const uint32_t run = static_cast<uint32_t>(quad / quads_per_run);
    const uint32_t lq = static_cast<uint32_t>(quad - static_cast<int64_t>(run) * quads_per_run);
    const uint32_t c3 = (run << 4) | kTagSweep;
    const Quad q = load_quad(wk, col);
    const KeysConst keys{rk};
    int8_t *__restrict__ S = L.S;
    const int64_t Wc = L.Wc;
    auto fetch = [&](int row) -> uint32_t {
        return *reinterpret_cast<const uint32_t *>(S + static_cast<int64_t>(row) * Wc + col);
    };
    for (int t = 0; t < nsweeps; ++t) {
        const uint32_t sweep = sweep0 + static_cast<uint32_t>(t);
        for (int c = 0; c < L.C; ++c) {
            const int beg = __ldg(L.cofs + c), end = __ldg(L.cofs + c + 1);
            for (int pos = beg + grp; pos < end; pos += G) {
                Rec<DC, DL> rc;
                rc.load(L.rec, pos);
                const uint32_t w = update4<DC, DL>(rc, q, fetch, sweep, lq, c3, keys);
                *reinterpret_cast<uint32_t *>(S + static_cast<int64_t>(pos) * Wc + col) = w;
            }
            __syncthreads();
        }
    }
    auto fetch_q = [&](int row, int) -> uint32_t { return fetch(row); };
    energies<DC, DL, 1>(L, wk, fetch_q, fetch_q, 4 * lane_q, grp, G, 4 * QL,
                        static_cast<int64_t>(blockIdx.x) * QL * 4);
}

__global__ void k_init_spins(Layout L, int32_t quads_per_run, uint32_t k0, uint32_t k1) {
    const int64_t quads = L.Wc / 4;
    const int64_t total = static_cast<int64_t>(L.n) * quads;
    const int *recs = reinterpret_cast<const int *>(L.rec);
    const int pid_at = L.DC + L.DL;
    for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t pos = e / quads;
        const int64_t quad = e - pos * quads;
        const uint32_t run = static_cast<uint32_t>(quad / quads_per_run);
        const uint32_t lq = static_cast<uint32_t>(quad - static_cast<int64_t>(run) * quads_per_run);
        const uint32_t pid = static_cast<uint32_t>(recs[pos * L.rec_vec * 4 + pid_at]);
        const uint4 r = philox4x32_10(make_uint4(pid, 0u, lq, (run << 4) | kTagInit), k0, k1);
        const uint32_t w = pack_signs(r.x < 0x80000000u ? -1.0f : 1.0f, r.y < 0x80000000u ? -1.0f : 1.0f,
                                      r.z < 0x80000000u ? -1.0f : 1.0f, r.w < 0x80000000u ? -1.0f : 1.0f);
        *reinterpret_cast<uint32_t *>(L.S + pos * L.Wc + quad * 4) = w;
    }
}

__global__ void k_init_walkers(RunState rs, Walkers wk) {
    const int run = blockIdx.x;
    const int64_t cb = static_cast<int64_t>(run) * rs.Rp;
    for (int s = threadIdx.x; s < rs.R; s += blockDim.x) {
        rs.walker_at[static_cast<int64_t>(run) * rs.R + s] = s;
        wk.wbeta[cb + s] = rs.beta[s / rs.J];
        wk.wP[cb + s] = rs.P[s % rs.J];
    }
    if (threadIdx.x == 0) {
        rs.best_f[run] = INT64_MAX;
        rs.best_event[run] = -1;
        rs.solved_event[run] = -1;
    }
}

__global__ void k_swap_event(Layout L, RunState rs, Walkers wk, uint32_t k0, uint32_t k1,
                             int64_t nev, int dir_p) {
    extern __shared__ int at[];
    __shared__ int s_copy;
    const int run = blockIdx.x;
    const int R = rs.R, I = rs.I, J = rs.J;
    const int64_t cb = static_cast<int64_t>(run) * rs.Rp;
    const int64_t rb = static_cast<int64_t>(run) * R;
    for (int s = threadIdx.x; s < R; s += blockDim.x) at[s] = rs.walker_at[rb + s];
    __syncthreads();
    const int *gw = wk.g + cb;
    const long long *fw = reinterpret_cast<const long long *>(wk.f) + cb;
    swap_pairs(at, [&](int w) { return fw[w]; }, [&](int w) { return gw[w]; }, rs.beta, rs.P, I, J,
               static_cast<uint32_t>(run), nev, dir_p, k0, k1, rs.acc_P + rb, rs.acc_B + rb);
    __syncthreads();
    for (int s = threadIdx.x; s < R; s += blockDim.x) {
        const int w = at[s];
        rs.walker_at[rb + s] = w;
        wk.wbeta[cb + w] = rs.beta[s / J];
        wk.wP[cb + w] = rs.P[s % J];
        const long long fw = wk.f[cb + w];
        const int gw = wk.g[cb + w];
        rs.sum_f[rb + s] += fw;
        rs.sum_g[rb + s] += gw;
        rs.n_feasible[rb + s] += (gw == 0);
    }
    if (threadIdx.x == 0) {
        const int wl = at[record_slot(at, [&](int w) { return static_cast<long long>(wk.f[cb + w]); },
                                      [&](int w) { return wk.g[cb + w]; }, I, J, rs.swap_mode)];
        const long long fl = wk.f[cb + wl];
        const int gl = wk.g[cb + wl];
        if (nev - 1 < rs.trace_cap) {
            rs.trace_f[run * rs.trace_cap + nev - 1] = fl;
            rs.trace_g[run * rs.trace_cap + nev - 1] = gl;
        }
        int copy = -1;
        if (gl == 0 && fl < rs.best_f[run]) {
            rs.best_f[run] = fl;
            rs.best_event[run] = nev;
            copy = wl;
        }
        if (rs.solved_event[run] < 0 && gl == 0 && fl <= rs.target[run]) rs.solved_event[run] = nev;
        s_copy = copy;
    }
    __syncthreads();
    const int wcopy = s_copy;
    if (wcopy >= 0) {
        const int *recs = reinterpret_cast<const int *>(L.rec);
        const int pid_at = L.DC + L.DL;
        for (int pos = threadIdx.x; pos < L.n; pos += blockDim.x)
            rs.best_state[static_cast<int64_t>(run) * L.n + recs[static_cast<int64_t>(pos) * L.rec_vec * 4 + pid_at]] =
                L.S[static_cast<int64_t>(pos) * L.Wc + cb + wcopy];
    }
}

// ---- diagnostics ----------------------------------------------------------
__global__ void k_diag_philox(const uint4 *ctr, const uint2 *key, uint4 *out, int64_t count) {
    const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (i < count) out[i] = philox4x32_10(ctr[i], key[i].x, key[i].y);
}

__global__ void k_diag_pt_exp(const float *x, float *y, int64_t count) {
    const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (i < count) y[i] = pt_exp(x[i]);
}

__global__ void k_diag_heatbath(const float *beta, const int32_t *H, const uint32_t *r, int8_t *s,
                                int64_t count) {
    const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (i < count) {
        const float b = beta[i];
        s[i] = static_cast<int8_t>(heatbath(b, b * -1.4426950408889634f, H[i], r[i]));
    }
}

__global__ void k_diag_swap(const float *x, const uint32_t *r, int8_t *a, int64_t count) {
    const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (i < count) a[i] = swap_accept(x[i], r[i]) ? 1 : 0;
}

template <typename T>
cudaError_t to_device(T **d, const T *h, int64_t count) {
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(d), sizeof(T) * (count > 0 ? count : 1));
    if (e != cudaSuccess) return e;
    return cudaMemcpy(*d, h, sizeof(T) * count, cudaMemcpyHostToDevice);
}

template <int DC, int DL, int WPT>
cudaError_t launch_smem_variant(const Layout &L, const Walkers &wk, const SweepTiling &tl,
                                int32_t qpr, const RoundKeys &rk, uint32_t sweep0,
                                int32_t nsweeps, cudaStream_t st) {
    int shift = 0;
    while ((1 << shift) < 4 * tl.lanes_per_spin) ++shift;
    const size_t smem = static_cast<size_t>(L.n + 1) << shift;
    cudaError_t e = allow_max_dynamic_smem<k_sweep_smem<DC, DL, WPT>>();
    if (e != cudaSuccess) return e;
    const unsigned blocks = static_cast<unsigned>(L.Wc >> shift);
    k_sweep_smem<DC, DL, WPT><<<blocks, tl.threads, smem, st>>>(L, wk, shift, qpr, rk, sweep0, nsweeps);
    return cudaGetLastError();
}

template <int DC, int DL>
cudaError_t launch_smem(const Layout &L, const Walkers &wk, const SweepTiling &tl, int32_t qpr,
                        const RoundKeys &rk, uint32_t sweep0, int32_t nsweeps, cudaStream_t st) {
    if (tl.walkers_per_thread == 8)
        return launch_smem_variant<DC, DL, 8>(L, wk, tl, qpr, rk, sweep0, nsweeps, st);
    return launch_smem_variant<DC, DL, 4>(L, wk, tl, qpr, rk, sweep0, nsweeps, st);
}

template <int DC, int DL>
cudaError_t launch_bits_variant(const Layout &L, const Walkers &wk, const SweepTiling &tl,
                                int32_t qpr, const RoundKeys &rk, uint32_t sweep0,
                                int32_t nsweeps, cudaStream_t st) {
    int shift = 0;
    while ((1 << shift) < 4 * tl.lanes_per_spin) ++shift;
    const size_t smem = bits_sweep_bytes(L.n, 1 << shift);
    if (tl.walkers_per_thread == 8) {
        cudaError_t e = allow_max_dynamic_smem<k_sweep_bits8<DC, DL>>();
        if (e != cudaSuccess) return e;
        const unsigned blocks = static_cast<unsigned>(L.Wc >> shift);
        k_sweep_bits8<DC, DL><<<blocks, tl.threads, smem, st>>>(L, wk, shift, qpr, rk, sweep0, nsweeps);
        return cudaGetLastError();
    }
    cudaError_t e = allow_max_dynamic_smem<k_sweep_bits<DC, DL>>();
    if (e != cudaSuccess) return e;
    const unsigned blocks = static_cast<unsigned>(L.Wc >> shift);
    k_sweep_bits<DC, DL><<<blocks, tl.threads, smem, st>>>(L, wk, shift, qpr, rk, sweep0, nsweeps);
    return cudaGetLastError();
}

template <int DC, int DL>
cudaError_t launch_global_variant(const Layout &L, const Walkers &wk, const SweepTiling &tl,
                                  int32_t qpr, const RoundKeys &rk, uint32_t sweep0,
                                  int32_t nsweeps, cudaStream_t st) {
    int shift = 0;
    while ((1 << shift) < tl.lanes_per_spin) ++shift;
    const unsigned blocks = static_cast<unsigned>(L.Wc / (4LL * tl.lanes_per_spin));
    k_sweep_global<DC, DL><<<blocks, tl.threads, 0, st>>>(L, wk, shift, qpr, rk, sweep0, nsweeps);
    return cudaGetLastError();
}

}  // namespace

size_t smem_sweep_bytes(int32_t n, int walkers_per_cta) {
    return static_cast<size_t>(n + 1) * static_cast<size_t>(walkers_per_cta);
}

size_t bits_sweep_bytes(int32_t n, int walkers_per_cta) {
    // the slab, then the byte table of k_sweep_bits8 (256 x 8 bytes; k_sweep_bits
    // uses the first 64 bytes as its nibble table)
    return ((static_cast<size_t>(n + 1) * (walkers_per_cta / 8) + 15) & ~static_cast<size_t>(15)) + 2048;
}

// ---- launchers --------------------------------------------------------------
cudaError_t launch_init(const Layout &L, const RunState &rs, const Walkers &wk, uint64_t seed,
                        cudaStream_t st) {
    const uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
    const int64_t total = static_cast<int64_t>(L.n) * (L.Wc / 4);
    int blocks = static_cast<int>((total + 255) / 256);
    if (blocks > 152 * 32) blocks = 152 * 32;
    if (blocks < 1) blocks = 1;
    k_init_spins<<<blocks, 256, 0, st>>>(L, rs.Rp / 4, k0, k1);
    k_init_walkers<<<rs.runs, 256, 0, st>>>(rs, wk);
    return cudaGetLastError();
}

cudaError_t launch_sweeps(const Layout &L, const Walkers &wk, const SweepTiling &tl,
                          int32_t quads_per_run, uint64_t seed, uint32_t sweep0, int32_t nsweeps,
                          cudaStream_t st) {
    if (L.penalty) return cudaErrorInvalidValue;  // specialised records only
    const RoundKeys rk = round_keys(seed);
    if (tl.bits) {
        if (L.DC == 3 && L.DL == 2) return launch_bits_variant<3, 2>(L, wk, tl, quads_per_run, rk, sweep0, nsweeps, st);
        if (L.DC == 4 && L.DL == 2) return launch_bits_variant<4, 2>(L, wk, tl, quads_per_run, rk, sweep0, nsweeps, st);
        if (L.DC == 6 && L.DL == 2) return launch_bits_variant<6, 2>(L, wk, tl, quads_per_run, rk, sweep0, nsweeps, st);
        return cudaErrorInvalidValue;
    }
    if (tl.smem) {
        if (L.DC == 3 && L.DL == 2) return launch_smem<3, 2>(L, wk, tl, quads_per_run, rk, sweep0, nsweeps, st);
        if (L.DC == 4 && L.DL == 2) return launch_smem<4, 2>(L, wk, tl, quads_per_run, rk, sweep0, nsweeps, st);
        if (L.DC == 6 && L.DL == 2) return launch_smem<6, 2>(L, wk, tl, quads_per_run, rk, sweep0, nsweeps, st);
        return cudaErrorInvalidValue;
    }
    if (L.DC == 3 && L.DL == 2) return launch_global_variant<3, 2>(L, wk, tl, quads_per_run, rk, sweep0, nsweeps, st);
    if (L.DC == 4 && L.DL == 2) return launch_global_variant<4, 2>(L, wk, tl, quads_per_run, rk, sweep0, nsweeps, st);
    if (L.DC == 6 && L.DL == 2) return launch_global_variant<6, 2>(L, wk, tl, quads_per_run, rk, sweep0, nsweeps, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_swap_event(const Layout &L, const RunState &rs, const Walkers &wk,
                              uint64_t seed, int64_t event, cudaStream_t st) {
    // Algorithm 1: direction +1 (P-swaps) for events 1, 2, then -1 (beta-swaps) for
    // 3, 4, ...: the direction flips after every even event; odd events use the
    // pairs starting at the first replica, even events those starting at the second.
    // The J-column PT baseline swaps along beta at every event.
    const int dir_p = event_dir_p(event, rs.swap_mode);
    const uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
    k_swap_event<<<rs.runs, 256, sizeof(int) * rs.R, st>>>(L, rs, wk, k0, k1, event, dir_p);
    return cudaGetLastError();
}

// ---- diagnostics (synchronous) -------------------------------------------------
cudaError_t diag_philox(const uint32_t *ctr, const uint32_t *key, uint32_t *out, int64_t count) {
    uint4 *dc = nullptr, *dout = nullptr;
    uint2 *dk = nullptr;
    cudaError_t e = to_device(&dc, reinterpret_cast<const uint4 *>(ctr), count);
    if (e == cudaSuccess) e = to_device(&dk, reinterpret_cast<const uint2 *>(key), count);
    if (e == cudaSuccess) e = cudaMalloc(&dout, sizeof(uint4) * (count > 0 ? count : 1));
    if (e == cudaSuccess && count > 0) {
        k_diag_philox<<<static_cast<unsigned>((count + 255) / 256), 256>>>(dc, dk, dout, count);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, sizeof(uint4) * count, cudaMemcpyDeviceToHost);
    cudaFree(dc);
    cudaFree(dk);
    cudaFree(dout);
    return e;
}

cudaError_t diag_pt_exp(const float *x, float *y, int64_t count) {
    float *dx = nullptr, *dy = nullptr;
    cudaError_t e = to_device(&dx, x, count);
    if (e == cudaSuccess) e = cudaMalloc(&dy, sizeof(float) * (count > 0 ? count : 1));
    if (e == cudaSuccess && count > 0) {
        k_diag_pt_exp<<<static_cast<unsigned>((count + 255) / 256), 256>>>(dx, dy, count);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(y, dy, sizeof(float) * count, cudaMemcpyDeviceToHost);
    cudaFree(dx);
    cudaFree(dy);
    return e;
}

cudaError_t diag_heatbath(const float *beta, const int32_t *H, const uint32_t *r, int8_t *spin,
                          int64_t count) {
    float *db = nullptr;
    int32_t *dh = nullptr;
    uint32_t *dr = nullptr;
    int8_t *ds = nullptr;
    cudaError_t e = to_device(&db, beta, count);
    if (e == cudaSuccess) e = to_device(&dh, H, count);
    if (e == cudaSuccess) e = to_device(&dr, r, count);
    if (e == cudaSuccess) e = cudaMalloc(&ds, count > 0 ? count : 1);
    if (e == cudaSuccess && count > 0) {
        k_diag_heatbath<<<static_cast<unsigned>((count + 255) / 256), 256>>>(db, dh, dr, ds, count);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(spin, ds, count, cudaMemcpyDeviceToHost);
    cudaFree(db);
    cudaFree(dh);
    cudaFree(dr);
    cudaFree(ds);
    return e;
}

cudaError_t diag_swap_accept(const float *x, const uint32_t *r, int8_t *acc, int64_t count) {
    float *dx = nullptr;
    uint32_t *dr = nullptr;
    int8_t *da = nullptr;
    cudaError_t e = to_device(&dx, x, count);
    if (e == cudaSuccess) e = to_device(&dr, r, count);
    if (e == cudaSuccess) e = cudaMalloc(&da, count > 0 ? count : 1);
    if (e == cudaSuccess && count > 0) {
        k_diag_swap<<<static_cast<unsigned>((count + 255) / 256), 256>>>(dx, dr, da, count);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(acc, da, count, cudaMemcpyDeviceToHost);
    cudaFree(dx);
    cudaFree(dr);
    cudaFree(da);
    return e;
}

}  // namespace pt2d
