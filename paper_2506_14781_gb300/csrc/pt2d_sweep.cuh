// Device building blocks shared by the sweep kernels of the plain contexts and
// the batched persistent kernel: spin-word byte access, packed neighbour
// records, the four-walker heat-bath update and the swap event of Algorithm 1.
#pragma once

#include <cstdint>

#include "pt2d_device.cuh"
#include "pt2d_internal.h"
#include "pt2d_wide.cuh"

namespace pt2d {

// Philox key source of the plain sweep loops: the ten round keys as kernel
// parameters (one seed per launch, read from constant memory).
struct KeysConst {
    RoundKeys rk;
    __device__ __forceinline__ uint4 operator()(uint4 x) const { return philox4x32_10(x, rk); }
};
// Round keys read from shared memory at every use, two rounds per 16-byte load
// (a run's keys staged by stage_round_keys; the batched kernels, a seed per run).
struct KeysShared {
    const uint4 *rk;
    __device__ __forceinline__ uint4 operator()(uint4 x) const {
#pragma unroll
        for (int r = 0; r < 5; ++r) {
            const uint4 kk = rk[r];
            x = philox_round(x, kk.x, kk.y);
            x = philox_round(x, kk.z, kk.w);
        }
        return x;
    }
};
// Two Philox calls with one run's staged round keys, one 16-byte shared load
// per two rounds serving both.
__device__ __forceinline__ void philox_pair_shared(const uint4 *rk, uint4 &x, uint4 &y) {
#pragma unroll
    for (int r = 0; r < 5; ++r) {
        const uint4 kk = rk[r];
        x = philox_round(x, kk.x, kk.y);
        y = philox_round(y, kk.x, kk.y);
        x = philox_round(x, kk.z, kk.w);
        y = philox_round(y, kk.z, kk.w);
    }
}
// A run's round keys staged in shared memory, two rounds per 16-byte word:
// dst[r] = (k0 of round 2r, k1 of round 2r, k0 of round 2r+1, k1 of round 2r+1).
__device__ __forceinline__ void stage_round_keys(uint4 *dst, uint32_t k0, uint32_t k1) {
    if (threadIdx.x < 5) {
        const uint32_t r = 2 * threadIdx.x;
        dst[threadIdx.x] = make_uint4(k0 + r * kWeyl0, k1 + r * kWeyl1, k0 + (r + 1) * kWeyl0,
                                      k1 + (r + 1) * kWeyl1);
    }
}

// byte b of x, sign-extended (one PRMT in sign-replicate mode)
template <int b>
__device__ __forceinline__ int sbyte(uint32_t x) {
    constexpr uint32_t n = 8u | b;
    constexpr uint32_t sel = (n << 12) | (n << 8) | (n << 4) | static_cast<uint32_t>(b);
    uint32_t d;
    asm("prmt.b32 %0, %1, 0, %2;" : "=r"(d) : "r"(x), "n"(sel));
    return static_cast<int>(d);
}

__device__ __forceinline__ int sbyte_rt(uint32_t x, int b) {
    return static_cast<int>(static_cast<int8_t>(static_cast<uint8_t>(x >> (8 * b))));
}

// Spin word from the sign bits of four decision values: byte k = 0x01 (+1) when
// t_k < 0, 0xFF (-1) otherwise.
__device__ __forceinline__ uint32_t pack_signs(float t0, float t1, float t2, float t3) {
    uint32_t lo, hi, m;
    asm("prmt.b32 %0, %1, %2, 0x00FB;" : "=r"(lo) : "r"(__float_as_uint(t0)), "r"(__float_as_uint(t1)));
    asm("prmt.b32 %0, %1, %2, 0x00FB;" : "=r"(hi) : "r"(__float_as_uint(t2)), "r"(__float_as_uint(t3)));
    asm("prmt.b32 %0, %1, %2, 0x5410;" : "=r"(m) : "r"(lo), "r"(hi));
    return ~m | 0x01010101u;
}

constexpr int kMaxSlab = 128;  // walkers per CTA

// Packed neighbour record of one position: [nb_0..nb_{DC-1}, lk_0..lk_{DL-1},
// pid, 2h, 2J_0..2J_{DC-1}] padded to whole int4s.  With DC = 3 and DL = 2
// the two padding ints hold J_0..J_2 as packed low and high bytes (byte k =
// J_k & 0xff, resp. J_k >> 8; byte 3 zero) for the byte dot products of
// decide4.
template <int DC, int DL>
struct Rec {
    static constexpr int kInts = 2 * DC + DL + 2;
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
};

struct Quad {
    float b0, b1, b2, b3;  // beta of each walker's slot
    float c0, c1, c2, c3;  // -beta * log2(e)
    int p0, p1, p2, p3;    // P of each walker's slot
};

__device__ __forceinline__ Quad load_quad(const Walkers &wk, int64_t col) {
    const float4 bt = *reinterpret_cast<const float4 *>(wk.wbeta + col);
    const int4 pj = *reinterpret_cast<const int4 *>(wk.wP + col);
    const float kNegL2E = -1.4426950408889634f;
    return Quad{bt.x, bt.y, bt.z, bt.w, bt.x * kNegL2E, bt.y * kNegL2E, bt.z * kNegL2E,
                bt.w * kNegL2E, pj.x, pj.y, pj.z, pj.w};
}

// New spin word of a quad from its four local fields H (Eq. 1 energy
// differences) and Philox block r: the fast decision, with the exact contract
// inside the uncertainty band.
__device__ __forceinline__ uint32_t decide_fields(const Quad &q, int a0, int a1, int a2, int a3,
                                                  const uint4 &r) {
    float t0 = heatbath_fast(q.c0, a0, r.x), t1 = heatbath_fast(q.c1, a1, r.y);
    float t2 = heatbath_fast(q.c2, a2, r.z), t3 = heatbath_fast(q.c3, a3, r.w);
    // one branch for the four band tests; inside it the exact contract decides
    if (fminf(fminf(fabsf(t0), fabsf(t1)), fminf(fabsf(t2), fabsf(t3))) <= kBand) {
        if (fabsf(t0) <= kBand) t0 = heatbath_exact(q.b0, a0, r.x) > 0 ? -1.0f : 1.0f;
        if (fabsf(t1) <= kBand) t1 = heatbath_exact(q.b1, a1, r.y) > 0 ? -1.0f : 1.0f;
        if (fabsf(t2) <= kBand) t2 = heatbath_exact(q.b2, a2, r.z) > 0 ? -1.0f : 1.0f;
        if (fabsf(t3) <= kBand) t3 = heatbath_exact(q.b3, a3, r.w) > 0 ? -1.0f : 1.0f;
    }
    return pack_signs(t0, t1, t2, t3);
}

// New spin word of one quad at one position.  `fetch(row)` returns the quad's
// spin word of a row (shared or global memory).
template <int DC, int DL>
__device__ __forceinline__ uint32_t decide4(const Rec<DC, DL> &rc, const Quad &q, const uint32_t *x,
                                            const uint32_t *y, const uint4 &r) {
    if constexpr (DC == 3 && DL == 2) {
        // Byte-transpose (x0, x1, x2, y0) into one word per walker; then the
        // coupling sum is two dp4a against the packed J bytes (sum J s =
        // sum lo s + 256 sum hi s, exact) and the link sum one dp4a picking
        // byte 3 plus the second link: the same integers as the loop below,
        // with sign extraction moved from the ALU to the FMA pipe (~5 %).
        uint32_t w0, w1, w2, w3;
        transpose4(x[0], x[1], x[2], y[0], w0, w1, w2, w3);
        const uint32_t lo = static_cast<uint32_t>(rc.v[10]), hi = static_cast<uint32_t>(rc.v[11]);
        const int h2 = rc.h2();
        const int a0 = h2 + 2 * dp4a_su(w0, lo, 256 * dp4a_ss(w0, hi, 0));
        const int a1 = h2 + 2 * dp4a_su(w1, lo, 256 * dp4a_ss(w1, hi, 0));
        const int a2 = h2 + 2 * dp4a_su(w2, lo, 256 * dp4a_ss(w2, hi, 0));
        const int a3 = h2 + 2 * dp4a_su(w3, lo, 256 * dp4a_ss(w3, hi, 0));
        const uint32_t e3 = 0x01000000u;  // picks the first link's spin from a transposed word
        const int l0 = dp4a_ss(w0, e3, sbyte<0>(y[1]));
        const int l1 = dp4a_ss(w1, e3, sbyte<1>(y[1]));
        const int l2 = dp4a_ss(w2, e3, sbyte<2>(y[1]));
        const int l3 = dp4a_ss(w3, e3, sbyte<3>(y[1]));
        return decide_fields(q, a0 + q.p0 * l0, a1 + q.p1 * l1, a2 + q.p2 * l2, a3 + q.p3 * l3, r);
    }
    int a0 = rc.h2(), a1 = a0, a2 = a0, a3 = a0;
#pragma unroll
    for (int k = 0; k < DC; ++k) {
        const int j = rc.j2(k);
        a0 += j * sbyte<0>(x[k]);
        a1 += j * sbyte<1>(x[k]);
        a2 += j * sbyte<2>(x[k]);
        a3 += j * sbyte<3>(x[k]);
    }
    int l0 = 0, l1 = 0, l2 = 0, l3 = 0;
#pragma unroll
    for (int l = 0; l < DL; ++l) {
        l0 += sbyte<0>(y[l]);
        l1 += sbyte<1>(y[l]);
        l2 += sbyte<2>(y[l]);
        l3 += sbyte<3>(y[l]);
    }
    return decide_fields(q, a0 + q.p0 * l0, a1 + q.p1 * l1, a2 + q.p2 * l2, a3 + q.p3 * l3, r);
}

template <int DC, int DL, typename Fetch, typename Keys>
__device__ __forceinline__ uint32_t update4(const Rec<DC, DL> &rc, const Quad &q, Fetch fetch,
                                            uint32_t sweep, uint32_t lq, uint32_t c3,
                                            const Keys &keys) {
    uint32_t x[DC], y[DL];
#pragma unroll
    for (int k = 0; k < DC; ++k) x[k] = fetch(rc.nb(k));
#pragma unroll
    for (int l = 0; l < DL; ++l) y[l] = fetch(rc.lk(l));
    const uint4 r = keys(make_uint4(static_cast<uint32_t>(rc.pid()), sweep, lq, c3));
    return decide4<DC, DL>(rc, q, x, y, r);
}

// Eight walkers (two quads) at one position: one 8-byte fetch per neighbour,
// two independent Philox calls (quad lq of run c3, and quad lqb of run c3b:
// the next quad, which starts the next run when a run holds an odd number of
// quads).
template <int DC, int DL, typename Fetch8>
__device__ __forceinline__ uint2 update8(const Rec<DC, DL> &rc, const Quad &qa, const Quad &qb,
                                         Fetch8 fetch8, uint32_t sweep, uint32_t lq, uint32_t c3,
                                         uint32_t lqb, uint32_t c3b, const KeysConst &keys) {
    uint32_t xa[DC], ya[DL], xb[DC], yb[DL];
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
    const uint4 ra = keys(make_uint4(id, sweep, lq, c3));
    const uint4 rb = keys(make_uint4(id, sweep, lqb, c3b));
    return make_uint2(decide4<DC, DL>(rc, qa, xa, ya, ra), decide4<DC, DL>(rc, qb, xb, yb, rb));
}

// Spin bits of four int8 spins: bit k is 1 iff byte k holds -1 (0xFF); the
// multiply gathers the four sign bits (no two product bits share a position).
__device__ __forceinline__ uint32_t bits_of_word(uint32_t w) {
    const uint32_t m = (w >> 7) & 0x01010101u;
    return ((m * 0x00204081u) >> 21) & 0xFu;
}

// Nibble -> four int8 spins (bit k set: byte k = -1), the table a bit-packed
// slab uses to expand a quad's spins.
__device__ __forceinline__ uint32_t word_of_bits(uint32_t nib) {
    uint32_t w = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) w |= ((nib >> k) & 1u ? 0xFFu : 0x01u) << (8 * k);
    return w;
}

// The slot an event records: the bottom-right replica (beta_I, P_J) in 2D-PT
// (swap_mode 0); in the J-column PT baseline (swap_mode 1) the last row's
// replica of lowest g, then lowest f, then lowest column.
template <typename FW, typename GW>
__device__ __forceinline__ int record_slot(const int *at, FW fw, GW gw, int I, int J, int swap_mode) {
    if (swap_mode == 0) return I * J - 1;
    int best = (I - 1) * J;
    for (int j = 1; j < J; ++j) {
        const int s = (I - 1) * J + j;
        const long long g = gw(at[s]), gb = gw(at[best]);
        if (g < gb || (g == gb && fw(at[s]) < fw(at[best]))) best = s;
    }
    return best;
}

// The pair loop of one swap event of Algorithm 1 for one run, by the calling
// CTA's threads (pairs of one event are disjoint, so they run in parallel).
// at: slot -> walker (shared memory, permuted in place); fw / gw: f and g by
// walker; acc_P / acc_B: accepted swaps by lower slot.  Event n uses the pairs
// starting at the first replica when n is odd and at the second when n is
// even; dir_p selects P-swaps inside rows (Eq. 2), otherwise beta-swaps inside
// columns (Eq. 3).  Uniform: Philox SWAP stream at (lower slot, n, 0).
template <typename FW, typename GW>
__device__ __forceinline__ void swap_pairs(int *at, FW fw, GW gw, const float *beta,
                                           const int32_t *P, int I, int J, uint32_t run,
                                           int64_t nev, int dir_p, uint32_t k0, uint32_t k1,
                                           int64_t *acc_P, int64_t *acc_B) {
    const int parity = (nev % 2 == 0) ? 1 : 0;
    const uint32_t c3 = (run << 4) | kTagSwap;
    const uint32_t n32 = static_cast<uint32_t>(nev);
    if (dir_p) {
        const int per_row = (J - parity) / 2;
        const int total = I * per_row;
        for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
            const int i = idx / per_row;
            const int j = parity + 2 * (idx - i * per_row);
            const int sa = i * J + j, sb = sa + 1;
            const int wa = at[sa], wb = at[sb];
            const long long dP = static_cast<long long>(P[j + 1]) - P[j];
            const long long dg = static_cast<long long>(gw(wb)) - gw(wa);
            const float x = __fmul_rn(beta[i], __ll2float_rn(dP * dg));
            const uint32_t r = philox4x32_10(make_uint4(static_cast<uint32_t>(sa), n32, 0u, c3), k0, k1).x;
            if (swap_accept(x, r)) {
                at[sa] = wb;
                at[sb] = wa;
                acc_P[sa] += 1;
            }
        }
    } else {
        const int per_col = (I - parity) / 2;
        const int total = J * per_col;
        for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
            const int j = idx / per_col;
            const int i = parity + 2 * (idx - j * per_col);
            const int sa = i * J + j, sb = sa + J;
            const int wa = at[sa], wb = at[sb];
            const float dbeta = __fsub_rn(beta[i + 1], beta[i]);
            const long long Ea = fw(wa) + static_cast<long long>(P[j]) * gw(wa);
            const long long Eb = fw(wb) + static_cast<long long>(P[j]) * gw(wb);
            const float x = __fmul_rn(dbeta, __ll2float_rn(Eb - Ea));
            const uint32_t r = philox4x32_10(make_uint4(static_cast<uint32_t>(sa), n32, 0u, c3), k0, k1).x;
            if (swap_accept(x, r)) {
                at[sa] = wb;
                at[sb] = wa;
                acc_B[sa] += 1;
            }
        }
    }
}

// Direction of event n (Algorithm 1): +1 (P-swaps) for n = 1, 2, then -1 for
// 3, 4, and so on, flipping after every even event.
__host__ __device__ __forceinline__ int event_is_pswap(int64_t nev) {
    return ((nev - 1) / 2) % 2 == 0 ? 1 : 0;
}

// Swap direction of event n: P-swaps (1) or beta-swaps (0); the J-column PT
// baseline (swap_mode 1) swaps along beta at every event.
__host__ __device__ __forceinline__ int event_dir_p(int64_t nev, int swap_mode) {
    return swap_mode == 0 ? event_is_pswap(nev) : 0;
}

}  // namespace pt2d
