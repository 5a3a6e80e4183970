// Shared-memory sweep kernels for instances with general penalty terms (Eq. 1
// with a constraint function g beyond copy links: weighted links K, penalty
// fields k, constant g0) and small degrees.
//
//  k_sweep_penalty_smem<DC, DL>  the sweep block of one event of Algorithm 1
//      with the CTA's int8 replica slab in shared memory, as k_sweep_smem,
//      reading the penalty record layout [nb x DC, lk x DL, pid, 2h,
//      2J x DC, K x DL, k] with compile-time offsets (16-byte loads, unrolled
//      neighbour loops), then f and g of the final sweep.
//  k_sweep_penalty_bits8<DC, DL>  the same with the slab bit-packed in shared
//      memory (instances whose int8 slab does not fit), as k_sweep_bits8:
//      one bit per walker, a thread owning a byte of 8 walkers that a
//      256-entry table expands to int8 spins; padding links (a bit cannot hold
//      the zero row's 0) are skipped by predicate.  k_sweep_penalty_bits: the
//      same with a nibble of 4 walkers per thread, as k_sweep_bits.
//
// The heat-bath field of spin a is H_a = 2 sum_b J_ab s_b + 2h_a +
// P (sum_l K_al s_l + k_a); padding neighbours and links point at the slab's
// zero row (and carry J = 0 / K = 0), so they add nothing.  The arithmetic
// (Philox counters, decision sequence, exact integer fields) is the same as in
// the runtime-degree kernels, so results are bit-identical to them.
#include <cstdint>

#include "pt2d_device.cuh"
#include "pt2d_internal.h"
#include "pt2d_penalty.h"
#include "pt2d_sweep.cuh"

namespace pt2d {
namespace {

template <int DC, int DL>
struct PenRec {
    static constexpr int kInts = 2 * DC + 2 * DL + 3;
    static constexpr int kVec = (kInts + 3) / 4;
    int v[kVec * 4];
    __device__ __forceinline__ void load(const int4 *base, int pos) {
        const int4 *p = base + static_cast<int64_t>(pos) * kVec;
#pragma unroll
        for (int i = 0; i < kVec; ++i) reinterpret_cast<int4 *>(v)[i] = __ldg(p + i);
    }
    __device__ __forceinline__ int nb(int k) const { return v[k]; }
    __device__ __forceinline__ int lk(int l) const { return v[DC + l]; }
    __device__ __forceinline__ int pid() const { return v[DC + DL]; }
    __device__ __forceinline__ int h2() const { return v[DC + DL + 1]; }
    __device__ __forceinline__ int j2(int k) const { return v[DC + DL + 2 + k]; }
    __device__ __forceinline__ int w(int l) const { return v[2 * DC + DL + 2 + l]; }
    __device__ __forceinline__ int kk() const { return v[2 * DC + 2 * DL + 2]; }
};

// Neighbour references in the records are byte offsets row * SW into the slab.
template <int DC, int DL>
__global__ void __launch_bounds__(1024, 1) k_sweep_penalty_smem(Layout L, Walkers wk, int sw_shift,
                                                                int32_t quads_per_run, RoundKeys rk,
                                                                uint32_t sweep0, int32_t nsweeps) {
    extern __shared__ __align__(16) int8_t smp[];
    const int SW = 1 << sw_shift;
    const int QL = SW >> 2;
    const int lane = threadIdx.x & (QL - 1);
    const int grp = threadIdx.x >> (sw_shift - 2);
    const int G = blockDim.x >> (sw_shift - 2);
    const int64_t col0 = static_cast<int64_t>(blockIdx.x) * SW;
    const int64_t quad = col0 / 4 + lane;
    const uint32_t run = static_cast<uint32_t>(quad / quads_per_run);
    const uint32_t lq = static_cast<uint32_t>(quad - static_cast<int64_t>(run) * quads_per_run);
    const uint32_t c3 = (run << 4) | kTagSweep;
    const int lane_off = 4 * lane;
    const Quad q = load_quad(wk, col0 + lane_off);
    const KeysConst keys{rk};
    const int vec_per_row = SW >> 4;
    const int64_t nvec = static_cast<int64_t>(L.n + 1) * vec_per_row;
    for (int64_t i = threadIdx.x; i < nvec; i += blockDim.x) {
        const int64_t row = i / vec_per_row;
        const int part = static_cast<int>(i - row * vec_per_row);
        reinterpret_cast<uint4 *>(smp)[i] =
            *reinterpret_cast<const uint4 *>(L.S + row * L.Wc + col0 + 16 * part);
    }
    __syncthreads();
    auto word = [&](int off) -> uint32_t { return *reinterpret_cast<const uint32_t *>(smp + off + lane_off); };
    for (int t = 0; t < nsweeps; ++t) {
        const uint32_t sweep = sweep0 + static_cast<uint32_t>(t);
        for (int c = 0; c < L.C; ++c) {
            const int beg = __ldg(L.cofs + c), end = __ldg(L.cofs + c + 1);
            for (int pos = beg + grp; pos < end; pos += G) {
                PenRec<DC, DL> rc;
                rc.load(L.rec, pos);
                uint32_t x[DC], y[DL];
#pragma unroll
                for (int k = 0; k < DC; ++k) x[k] = word(rc.nb(k));
#pragma unroll
                for (int l = 0; l < DL; ++l) y[l] = word(rc.lk(l));
                const uint4 r = keys(make_uint4(static_cast<uint32_t>(rc.pid()), sweep, lq, c3));
                int a0 = rc.h2(), a1 = a0, a2 = a0, a3 = a0;
#pragma unroll
                for (int k = 0; k < DC; ++k) {
                    const int j = rc.j2(k);
                    a0 += j * sbyte<0>(x[k]);
                    a1 += j * sbyte<1>(x[k]);
                    a2 += j * sbyte<2>(x[k]);
                    a3 += j * sbyte<3>(x[k]);
                }
                int l0 = rc.kk(), l1 = l0, l2 = l0, l3 = l0;
#pragma unroll
                for (int l = 0; l < DL; ++l) {
                    const int w = rc.w(l);
                    l0 += w * sbyte<0>(y[l]);
                    l1 += w * sbyte<1>(y[l]);
                    l2 += w * sbyte<2>(y[l]);
                    l3 += w * sbyte<3>(y[l]);
                }
                *reinterpret_cast<uint32_t *>(smp + (pos << sw_shift) + lane_off) =
                    decide_fields(q, a0 + q.p0 * l0, a1 + q.p1 * l1, a2 + q.p2 * l2, a3 + q.p3 * l3, r);
            }
            __syncthreads();
        }
    }
    const int64_t nvec_out = static_cast<int64_t>(L.n) * vec_per_row;
    for (int64_t i = threadIdx.x; i < nvec_out; i += blockDim.x) {
        const int64_t row = i / vec_per_row;
        const int part = static_cast<int>(i - row * vec_per_row);
        *reinterpret_cast<uint4 *>(L.S + row * L.Wc + col0 + 16 * part) = reinterpret_cast<const uint4 *>(smp)[i];
    }
    // f and g of the final sweep: F = sum_a s_a (sum_b 2J s_b + 2 * 2h_a) = -4 f;
    // twice g: each link from both ends (weight K), twice k of a down spin
    __shared__ long long s_F[kMaxSlab];
    __shared__ int s_g[kMaxSlab];
    for (int i = threadIdx.x; i < SW; i += blockDim.x) {
        s_F[i] = 0;
        s_g[i] = 0;
    }
    __syncthreads();
    long long F0 = 0, F1 = 0, F2 = 0, F3 = 0;
    int g0 = 0, g1 = 0, g2 = 0, g3 = 0;
    for (int pos = grp; pos < L.n; pos += G) {
        PenRec<DC, DL> rc;
        rc.load(L.rec, pos);
        const uint32_t xs = word(pos << sw_shift);
        const int h4 = 2 * rc.h2();
        int c0 = h4, c1 = h4, c2 = h4, c3x = h4;
#pragma unroll
        for (int k = 0; k < DC; ++k) {
            const uint32_t x = word(rc.nb(k));
            const int j = rc.j2(k);
            c0 += j * sbyte<0>(x);
            c1 += j * sbyte<1>(x);
            c2 += j * sbyte<2>(x);
            c3x += j * sbyte<3>(x);
        }
        F0 += static_cast<long long>(sbyte<0>(xs)) * c0;
        F1 += static_cast<long long>(sbyte<1>(xs)) * c1;
        F2 += static_cast<long long>(sbyte<2>(xs)) * c2;
        F3 += static_cast<long long>(sbyte<3>(xs)) * c3x;
#pragma unroll
        for (int l = 0; l < DL; ++l) {
            if (rc.lk(l) == L.pad_ref) continue;
            const uint32_t y = word(rc.lk(l));
            const int w = rc.w(l);
            g0 += w * (sbyte<0>(xs) != sbyte<0>(y));
            g1 += w * (sbyte<1>(xs) != sbyte<1>(y));
            g2 += w * (sbyte<2>(xs) != sbyte<2>(y));
            g3 += w * (sbyte<3>(xs) != sbyte<3>(y));
        }
        const int k2 = 2 * rc.kk();
        g0 += sbyte<0>(xs) < 0 ? k2 : 0;
        g1 += sbyte<1>(xs) < 0 ? k2 : 0;
        g2 += sbyte<2>(xs) < 0 ? k2 : 0;
        g3 += sbyte<3>(xs) < 0 ? k2 : 0;
    }
    unsigned long long *sF = reinterpret_cast<unsigned long long *>(s_F);
    atomicAdd(sF + lane_off + 0, static_cast<unsigned long long>(F0));
    atomicAdd(sF + lane_off + 1, static_cast<unsigned long long>(F1));
    atomicAdd(sF + lane_off + 2, static_cast<unsigned long long>(F2));
    atomicAdd(sF + lane_off + 3, static_cast<unsigned long long>(F3));
    atomicAdd(&s_g[lane_off + 0], g0);
    atomicAdd(&s_g[lane_off + 1], g1);
    atomicAdd(&s_g[lane_off + 2], g2);
    atomicAdd(&s_g[lane_off + 3], g3);
    __syncthreads();
    for (int i = threadIdx.x; i < SW; i += blockDim.x) {
        wk.f[col0 + i] = -(s_F[i] / 4);
        wk.g[col0 + i] = s_g[i] / 2 + L.g0;
    }
}

// Neighbour references in the records are byte offsets row * SW / 8 into the
// bit-packed slab.
template <int DC, int DL>
__global__ void __launch_bounds__(1024, 1) k_sweep_penalty_bits(Layout L, Walkers wk, int sw_shift,
                                                                int32_t quads_per_run, RoundKeys rk,
                                                                uint32_t sweep0, int32_t nsweeps) {
    extern __shared__ __align__(16) uint8_t spb[];
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
    uint8_t *bits = spb;
    uint32_t *lut = reinterpret_cast<uint32_t *>(spb + ((static_cast<int64_t>(n + 1) * B + 15) & ~15LL));
    if (threadIdx.x < 16) lut[threadIdx.x] = word_of_bits(threadIdx.x);
    const int64_t nbytes = static_cast<int64_t>(n + 1) * B;
    for (int64_t i = threadIdx.x; i < nbytes; i += blockDim.x) {
        const int64_t row = i / B;
        const int b = static_cast<int>(i - row * B);
        const uint2 v = *reinterpret_cast<const uint2 *>(L.S + row * L.Wc + col0 + 8 * b);
        bits[i] = static_cast<uint8_t>(bits_of_word(v.x) | (bits_of_word(v.y) << 4));
    }
    __syncthreads();

    auto fetch = [&](int off) -> uint32_t { return lut[(bits[off + byte_lane] >> nib_shift) & 0xF]; };
    const int pad = L.pad_ref;
    for (int t = 0; t < nsweeps; ++t) {
        const uint32_t sweep = sweep0 + static_cast<uint32_t>(t);
        for (int c = 0; c < L.C; ++c) {
            const int beg = __ldg(L.cofs + c), end = __ldg(L.cofs + c + 1);
            for (int pos = beg + grp; pos < end; pos += G) {
                PenRec<DC, DL> rc;
                rc.load(L.rec, pos);
                uint32_t x[DC], y[DL];
#pragma unroll
                for (int k = 0; k < DC; ++k) x[k] = fetch(rc.nb(k));
#pragma unroll
                for (int l = 0; l < DL; ++l) y[l] = rc.lk(l) != pad ? fetch(rc.lk(l)) : 0u;
                const uint4 r = keys(make_uint4(static_cast<uint32_t>(rc.pid()), sweep, lq, c3));
                int a0 = rc.h2(), a1 = a0, a2 = a0, a3 = a0;
#pragma unroll
                for (int k = 0; k < DC; ++k) {
                    const int j = rc.j2(k);
                    a0 += j * sbyte<0>(x[k]);
                    a1 += j * sbyte<1>(x[k]);
                    a2 += j * sbyte<2>(x[k]);
                    a3 += j * sbyte<3>(x[k]);
                }
                int l0 = rc.kk(), l1 = l0, l2 = l0, l3 = l0;
#pragma unroll
                for (int l = 0; l < DL; ++l) {
                    const int w = rc.w(l);
                    l0 += w * sbyte<0>(y[l]);
                    l1 += w * sbyte<1>(y[l]);
                    l2 += w * sbyte<2>(y[l]);
                    l3 += w * sbyte<3>(y[l]);
                }
                const uint32_t nib = bits_of_word(
                    decide_fields(q, a0 + q.p0 * l0, a1 + q.p1 * l1, a2 + q.p2 * l2, a3 + q.p3 * l3, r));
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
    // f and g of the final sweep, as in k_sweep_penalty_smem
    __shared__ long long s_F[kMaxSlab];
    __shared__ int s_g[kMaxSlab];
    for (int i = threadIdx.x; i < SW; i += blockDim.x) {
        s_F[i] = 0;
        s_g[i] = 0;
    }
    __syncthreads();
    long long F0 = 0, F1 = 0, F2 = 0, F3 = 0;
    int g0 = 0, g1 = 0, g2 = 0, g3 = 0;
    for (int pos = grp; pos < n; pos += G) {
        PenRec<DC, DL> rc;
        rc.load(L.rec, pos);
        const uint32_t xs = fetch(pos * B);
        const int h4 = 2 * rc.h2();
        int c0 = h4, c1 = h4, c2 = h4, c3x = h4;
#pragma unroll
        for (int k = 0; k < DC; ++k) {
            const uint32_t x = fetch(rc.nb(k));
            const int j = rc.j2(k);
            c0 += j * sbyte<0>(x);
            c1 += j * sbyte<1>(x);
            c2 += j * sbyte<2>(x);
            c3x += j * sbyte<3>(x);
        }
        F0 += static_cast<long long>(sbyte<0>(xs)) * c0;
        F1 += static_cast<long long>(sbyte<1>(xs)) * c1;
        F2 += static_cast<long long>(sbyte<2>(xs)) * c2;
        F3 += static_cast<long long>(sbyte<3>(xs)) * c3x;
#pragma unroll
        for (int l = 0; l < DL; ++l) {
            if (rc.lk(l) == pad) continue;
            const uint32_t y = fetch(rc.lk(l));
            const int w = rc.w(l);
            g0 += w * (sbyte<0>(xs) != sbyte<0>(y));
            g1 += w * (sbyte<1>(xs) != sbyte<1>(y));
            g2 += w * (sbyte<2>(xs) != sbyte<2>(y));
            g3 += w * (sbyte<3>(xs) != sbyte<3>(y));
        }
        const int k2 = 2 * rc.kk();
        g0 += sbyte<0>(xs) < 0 ? k2 : 0;
        g1 += sbyte<1>(xs) < 0 ? k2 : 0;
        g2 += sbyte<2>(xs) < 0 ? k2 : 0;
        g3 += sbyte<3>(xs) < 0 ? k2 : 0;
    }
    const int w0 = 4 * lane_q;
    unsigned long long *sF = reinterpret_cast<unsigned long long *>(s_F);
    atomicAdd(sF + w0 + 0, static_cast<unsigned long long>(F0));
    atomicAdd(sF + w0 + 1, static_cast<unsigned long long>(F1));
    atomicAdd(sF + w0 + 2, static_cast<unsigned long long>(F2));
    atomicAdd(sF + w0 + 3, static_cast<unsigned long long>(F3));
    atomicAdd(&s_g[w0 + 0], g0);
    atomicAdd(&s_g[w0 + 1], g1);
    atomicAdd(&s_g[w0 + 2], g2);
    atomicAdd(&s_g[w0 + 3], g3);
    __syncthreads();
    for (int i = threadIdx.x; i < SW; i += blockDim.x) {
        wk.f[col0 + i] = -(s_F[i] / 4);
        wk.g[col0 + i] = s_g[i] / 2 + L.g0;
    }
}

// The same with one byte (8 walkers, two quads) per thread, as k_sweep_bits8: a
// 256-entry table expands a byte to both quads' int8 spin words with one 8-byte
// shared load; the byte is written whole (no shuffle).
template <int DC, int DL>
__global__ void __launch_bounds__(kPenaltyBits8Threads, 1) k_sweep_penalty_bits8(Layout L, Walkers wk, int sw_shift,
                                                                int32_t quads_per_run, RoundKeys rk,
                                                                uint32_t sweep0, int32_t nsweeps) {
    extern __shared__ __align__(16) uint8_t spb[];
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
    // the second quad starts the next run when a run holds an odd number of quads
    const uint32_t run_b = static_cast<uint32_t>((quad + 1) / quads_per_run);
    const uint32_t lqb = static_cast<uint32_t>(quad + 1 - static_cast<int64_t>(run_b) * quads_per_run);
    const uint32_t c3b = (run_b << 4) | kTagSweep;
    const Quad qa = load_quad(wk, col0 + 8 * lane_b);
    const Quad qb = load_quad(wk, col0 + 8 * lane_b + 4);
    const KeysConst keys{rk};
    const int n = L.n;
    uint8_t *bits = spb;
    uint2 *lut = reinterpret_cast<uint2 *>(spb + ((static_cast<int64_t>(n + 1) * B + 15) & ~15LL));
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
    // fields of one quad (walkers of word x / y) at one position, the decision, four bits
    auto quad_bits = [&](const PenRec<DC, DL> &rc, const Quad &q, const uint32_t *x, const uint32_t *y,
                         const uint4 &r) -> uint32_t {
        int a0 = rc.h2(), a1 = a0, a2 = a0, a3 = a0;
#pragma unroll
        for (int k = 0; k < DC; ++k) {
            const int j = rc.j2(k);
            a0 += j * sbyte<0>(x[k]);
            a1 += j * sbyte<1>(x[k]);
            a2 += j * sbyte<2>(x[k]);
            a3 += j * sbyte<3>(x[k]);
        }
        int l0 = rc.kk(), l1 = l0, l2 = l0, l3 = l0;
#pragma unroll
        for (int l = 0; l < DL; ++l) {
            const int w = rc.w(l);
            l0 += w * sbyte<0>(y[l]);
            l1 += w * sbyte<1>(y[l]);
            l2 += w * sbyte<2>(y[l]);
            l3 += w * sbyte<3>(y[l]);
        }
        return bits_of_word(
            decide_fields(q, a0 + q.p0 * l0, a1 + q.p1 * l1, a2 + q.p2 * l2, a3 + q.p3 * l3, r));
    };
    const int pad = L.pad_ref;
    for (int t = 0; t < nsweeps; ++t) {
        const uint32_t sweep = sweep0 + static_cast<uint32_t>(t);
        for (int c = 0; c < L.C; ++c) {
            const int beg = __ldg(L.cofs + c), end = __ldg(L.cofs + c + 1);
            for (int pos = beg + grp; pos < end; pos += G) {
                PenRec<DC, DL> rc;
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
                const uint32_t na = quad_bits(rc, qa, xa, ya, keys(make_uint4(id, sweep, lq, c3)));
                const uint32_t nb = quad_bits(rc, qb, xb, yb, keys(make_uint4(id, sweep, lqb, c3b)));
                bits[pos * B + lane_b] = static_cast<uint8_t>(na | (nb << 4));
            }
            __syncthreads();
        }
    }
    // write back rows 0..n-1 as int8 spins
    const int64_t nb_out = static_cast<int64_t>(n) * B;
    for (int64_t i = threadIdx.x; i < nb_out; i += blockDim.x) {
        const int64_t row = i / B;
        const int b = static_cast<int>(i - row * B);
        *reinterpret_cast<uint2 *>(L.S + row * L.Wc + col0 + 8 * b) = lut[bits[i]];
    }
    // f and g of the final sweep, as in k_sweep_penalty_smem, for the thread's 8 walkers
    __shared__ long long s_F[kMaxSlab];
    __shared__ int s_g[kMaxSlab];
    for (int i = threadIdx.x; i < SW; i += blockDim.x) {
        s_F[i] = 0;
        s_g[i] = 0;
    }
    __syncthreads();
    long long F[8];
    int g[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        F[i] = 0;
        g[i] = 0;
    }
    auto sb = [](const uint2 &w, int i) -> int {
        const uint32_t x = i < 4 ? w.x : w.y;
        return sbyte_rt(x, i & 3);
    };
    for (int pos = grp; pos < n; pos += G) {
        PenRec<DC, DL> rc;
        rc.load(L.rec, pos);
        const uint2 xs = fetch8(pos * B);
        const int h4 = 2 * rc.h2();
        int cs[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) cs[i] = h4;
#pragma unroll
        for (int k = 0; k < DC; ++k) {
            const uint2 x = fetch8(rc.nb(k));
            const int j = rc.j2(k);
#pragma unroll
            for (int i = 0; i < 8; ++i) cs[i] += j * sb(x, i);
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) F[i] += static_cast<long long>(sb(xs, i)) * cs[i];
#pragma unroll
        for (int l = 0; l < DL; ++l) {
            if (rc.lk(l) == pad) continue;
            const uint2 y = fetch8(rc.lk(l));
            const int w = rc.w(l);
#pragma unroll
            for (int i = 0; i < 8; ++i) g[i] += w * (sb(xs, i) != sb(y, i));
        }
        const int k2 = 2 * rc.kk();
#pragma unroll
        for (int i = 0; i < 8; ++i) g[i] += sb(xs, i) < 0 ? k2 : 0;
    }
    const int w0 = 8 * lane_b;
    unsigned long long *sF = reinterpret_cast<unsigned long long *>(s_F);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        atomicAdd(sF + w0 + i, static_cast<unsigned long long>(F[i]));
        atomicAdd(&s_g[w0 + i], g[i]);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < SW; i += blockDim.x) {
        wk.f[col0 + i] = -(s_F[i] / 4);
        wk.g[col0 + i] = s_g[i] / 2 + L.g0;
    }
}

template <int DC, int DL>
cudaError_t launch_bits_variant(const Layout &L, const Walkers &wk, const SweepTiling &tl, int32_t qpr,
                                const RoundKeys &rk, uint32_t sweep0, int32_t nsweeps, cudaStream_t st) {
    int shift = 0;
    while ((1 << shift) < 4 * tl.lanes_per_spin) ++shift;
    const size_t smem = bits_sweep_bytes(L.n, 1 << shift);
    if (tl.walkers_per_thread == 8) {
        cudaError_t e = allow_max_dynamic_smem<k_sweep_penalty_bits8<DC, DL>>();
        if (e != cudaSuccess) return e;
        const unsigned blocks = static_cast<unsigned>(L.Wc >> shift);
        k_sweep_penalty_bits8<DC, DL><<<blocks, tl.threads, smem, st>>>(L, wk, shift, qpr, rk, sweep0, nsweeps);
        return cudaGetLastError();
    }
    cudaError_t e = allow_max_dynamic_smem<k_sweep_penalty_bits<DC, DL>>();
    if (e != cudaSuccess) return e;
    const unsigned blocks = static_cast<unsigned>(L.Wc >> shift);
    k_sweep_penalty_bits<DC, DL><<<blocks, tl.threads, smem, st>>>(L, wk, shift, qpr, rk, sweep0, nsweeps);
    return cudaGetLastError();
}

template <int DC, int DL>
cudaError_t launch_variant(const Layout &L, const Walkers &wk, const SweepTiling &tl, int32_t qpr,
                           const RoundKeys &rk, uint32_t sweep0, int32_t nsweeps, cudaStream_t st) {
    int shift = 0;
    while ((1 << shift) < 4 * tl.lanes_per_spin) ++shift;
    const size_t smem = smem_sweep_bytes(L.n, 1 << shift);
    cudaError_t e = allow_max_dynamic_smem<k_sweep_penalty_smem<DC, DL>>();
    if (e != cudaSuccess) return e;
    const unsigned blocks = static_cast<unsigned>(L.Wc >> shift);
    k_sweep_penalty_smem<DC, DL><<<blocks, tl.threads, smem, st>>>(L, wk, shift, qpr, rk, sweep0, nsweeps);
    return cudaGetLastError();
}

}  // namespace

bool penalty_kernel_degrees(int DC, int DL) {
    return (DC == 3 || DC == 4 || DC == 6) && (DL == 2 || DL == 3);
}

cudaError_t launch_penalty_sweeps(const Layout &L, const Walkers &wk, const SweepTiling &tl,
                                  int32_t quads_per_run, uint64_t seed, uint32_t sweep0, int32_t nsweeps,
                                  cudaStream_t st) {
    if (!L.penalty || (tl.walkers_per_thread != 4 && !(tl.bits && tl.walkers_per_thread == 8)))
        return cudaErrorInvalidValue;
    const RoundKeys rk = round_keys(seed);
    const int k = L.DC * 8 + L.DL;
    if (tl.bits) {
        if (tl.lanes_per_spin < 2) return cudaErrorInvalidValue;  // slabs of >= 8 walkers
        switch (k) {
            case 3 * 8 + 2: return launch_bits_variant<3, 2>(L, wk, tl, quads_per_run, rk, sweep0, nsweeps, st);
            case 3 * 8 + 3: return launch_bits_variant<3, 3>(L, wk, tl, quads_per_run, rk, sweep0, nsweeps, st);
            case 4 * 8 + 2: return launch_bits_variant<4, 2>(L, wk, tl, quads_per_run, rk, sweep0, nsweeps, st);
            case 4 * 8 + 3: return launch_bits_variant<4, 3>(L, wk, tl, quads_per_run, rk, sweep0, nsweeps, st);
            case 6 * 8 + 2: return launch_bits_variant<6, 2>(L, wk, tl, quads_per_run, rk, sweep0, nsweeps, st);
            case 6 * 8 + 3: return launch_bits_variant<6, 3>(L, wk, tl, quads_per_run, rk, sweep0, nsweeps, st);
            default: return cudaErrorInvalidValue;
        }
    }
    if (!tl.smem || tl.lanes_per_spin < 4) return cudaErrorInvalidValue;
    switch (k) {
        case 3 * 8 + 2: return launch_variant<3, 2>(L, wk, tl, quads_per_run, rk, sweep0, nsweeps, st);
        case 3 * 8 + 3: return launch_variant<3, 3>(L, wk, tl, quads_per_run, rk, sweep0, nsweeps, st);
        case 4 * 8 + 2: return launch_variant<4, 2>(L, wk, tl, quads_per_run, rk, sweep0, nsweeps, st);
        case 4 * 8 + 3: return launch_variant<4, 3>(L, wk, tl, quads_per_run, rk, sweep0, nsweeps, st);
        case 6 * 8 + 2: return launch_variant<6, 2>(L, wk, tl, quads_per_run, rk, sweep0, nsweeps, st);
        case 6 * 8 + 3: return launch_variant<6, 3>(L, wk, tl, quads_per_run, rk, sweep0, nsweeps, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pt2d
