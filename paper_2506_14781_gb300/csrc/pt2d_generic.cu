// Runtime-degree sweep kernels of the plain contexts (any coupling and link
// degree, optional general penalty terms), on wide records (pt2d_wide.cuh).
//
//  k_sweep_generic_smem  the sweep block of one event of Algorithm 1 with the
//                        CTA's int8 replica slab in shared memory for the whole
//                        block (as k_sweep_smem), then f and g (Eq. 1)
//  k_sweep_generic       the same with the slab in global memory
//
// Couplings are summed four at a time: four neighbour words of the quad are
// byte-transposed into one word per walker and dotted with the packed coupling
// bytes (two dp4a per walker and group); links and penalty terms follow one by
// one.  All arithmetic is exact integer up to the fixed FP32 decision sequence,
// so the results are those of the oracle bit for bit.
#include <cstdint>

#include "pt2d_device.cuh"
#include "pt2d_generic.h"
#include "pt2d_internal.h"
#include "pt2d_sweep.cuh"
#include "pt2d_wide.cuh"

namespace pt2d {
namespace {

// Local fields of a quad at one position (Eq. 1 energy differences):
// a_b = 2h + 2 sum_k J_k s_kb + P_b (sum_l K_l s_lb + k).
template <typename Fetch>
__device__ __forceinline__ void wide_fields(const Layout &L, const int *rc, int jo, Fetch fetch, const Quad &q,
                                            int &a0, int &a1, int &a2, int &a3) {
    const int DC = L.DC, DL = L.DL;
    int j0, j1, j2, j3;  // sum_k J_k s_k per walker
    wide_coupling_sums<false>(rc, DC, jo, fetch, j0, j1, j2, j3);
    const int h2 = __ldg(rc + DC + DL + 1);
    const int ko = jo + DC / 2;  // link weights, then the penalty field
    int l0 = L.penalty ? __ldg(rc + ko + DL) : 0;
    int l1 = l0, l2 = l0, l3 = l0;
    for (int k = 0; k < DL; ++k) {
        const uint32_t y = fetch(__ldg(rc + DC + k));
        const int w = L.penalty ? __ldg(rc + ko + k) : 1;
        l0 += w * sbyte<0>(y);
        l1 += w * sbyte<1>(y);
        l2 += w * sbyte<2>(y);
        l3 += w * sbyte<3>(y);
    }
    a0 = h2 + 2 * j0 + q.p0 * l0;
    a1 = h2 + 2 * j1 + q.p1 * l1;
    a2 = h2 + 2 * j2 + q.p2 * l2;
    a3 = h2 + 2 * j3 + q.p3 * l3;
}

// f and g of the final sweep for the thread's quad, summed over its positions
// and merged into s_F / s_g (shared, zeroed):  F = sum_a s_a (2h_a + ... ) as in
// the specialised kernels, f = -F/4; twice g: each link from both ends
// (weight K), twice k of a down spin.
template <typename Fetch, typename Own>
__device__ __forceinline__ void wide_energies(const Layout &L, int jo, Fetch fetch, Own own, int grp, int G,
                                              long long *s_F, int *s_g, int lane_off) {
    const int DC = L.DC, DL = L.DL;
    const int rec_ints = L.rec_vec * 4;
    const int *recs = reinterpret_cast<const int *>(L.rec);
    const int ko = jo + DC / 2;
    long long F0 = 0, F1 = 0, F2 = 0, F3 = 0;
    int g0 = 0, g1 = 0, g2 = 0, g3 = 0;
    for (int pos = grp; pos < L.n; pos += G) {
        const int *rc = recs + static_cast<int64_t>(pos) * rec_ints;
        const uint32_t xs = own(pos);
        int j0, j1, j2, j3;
        wide_coupling_sums<false>(rc, DC, jo, fetch, j0, j1, j2, j3);
        const int h4 = 2 * __ldg(rc + DC + DL + 1);
        F0 += static_cast<long long>(sbyte<0>(xs)) * (h4 + 2 * j0);
        F1 += static_cast<long long>(sbyte<1>(xs)) * (h4 + 2 * j1);
        F2 += static_cast<long long>(sbyte<2>(xs)) * (h4 + 2 * j2);
        F3 += static_cast<long long>(sbyte<3>(xs)) * (h4 + 2 * j3);
        for (int k = 0; k < DL; ++k) {
            const int lp = __ldg(rc + DC + k);
            if (lp == L.pad_ref) continue;
            const uint32_t y = fetch(lp);
            const int w = L.penalty ? __ldg(rc + ko + k) : 1;
            g0 += w * (sbyte<0>(xs) != sbyte<0>(y));
            g1 += w * (sbyte<1>(xs) != sbyte<1>(y));
            g2 += w * (sbyte<2>(xs) != sbyte<2>(y));
            g3 += w * (sbyte<3>(xs) != sbyte<3>(y));
        }
        if (L.penalty) {
            const int k2 = 2 * __ldg(rc + ko + DL);
            g0 += sbyte<0>(xs) < 0 ? k2 : 0;
            g1 += sbyte<1>(xs) < 0 ? k2 : 0;
            g2 += sbyte<2>(xs) < 0 ? k2 : 0;
            g3 += sbyte<3>(xs) < 0 ? k2 : 0;
        }
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
}

// Slab in global memory; neighbour references are row indices.
__global__ void __launch_bounds__(256) k_sweep_generic(Layout L, Walkers wk, int ql_shift, int32_t quads_per_run,
                                                       RoundKeys rk, uint32_t sweep0, int32_t nsweeps) {
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
    const int rec_ints = L.rec_vec * 4;
    const int *recs = reinterpret_cast<const int *>(L.rec);
    const int jo = wide_jpack_offset(L.DC, L.DL);
    int8_t *__restrict__ S = L.S;
    const int64_t Wc = L.Wc;
    auto word = [&](int row) -> uint32_t {
        return *reinterpret_cast<const uint32_t *>(S + static_cast<int64_t>(row) * Wc + col);
    };
    for (int t = 0; t < nsweeps; ++t) {
        const uint32_t sweep = sweep0 + static_cast<uint32_t>(t);
        for (int c = 0; c < L.C; ++c) {
            const int beg = __ldg(L.cofs + c), end = __ldg(L.cofs + c + 1);
            for (int pos = beg + grp; pos < end; pos += G) {
                const int *rc = recs + static_cast<int64_t>(pos) * rec_ints;
                int a0, a1, a2, a3;
                wide_fields(L, rc, jo, word, q, a0, a1, a2, a3);
                const uint4 r = keys(make_uint4(static_cast<uint32_t>(__ldg(rc + L.DC + L.DL)), sweep, lq, c3));
                *reinterpret_cast<uint32_t *>(S + static_cast<int64_t>(pos) * Wc + col) =
                    decide_fields(q, a0, a1, a2, a3, r);
            }
            __syncthreads();
        }
    }
    __shared__ long long s_F[kMaxSlab];
    __shared__ int s_g[kMaxSlab];
    for (int i = threadIdx.x; i < 4 * QL; i += blockDim.x) {
        s_F[i] = 0;
        s_g[i] = 0;
    }
    __syncthreads();
    wide_energies(L, jo, word, word, grp, G, s_F, s_g, 4 * lane_q);
    __syncthreads();
    const int64_t col0 = static_cast<int64_t>(blockIdx.x) * QL * 4;
    for (int i = threadIdx.x; i < 4 * QL; i += blockDim.x) {
        wk.f[col0 + i] = -(s_F[i] / 4);
        wk.g[col0 + i] = s_g[i] / 2 + L.g0;
    }
}

// Slab in shared memory for the whole block; neighbour references are byte
// offsets row * SW into the slab.
__global__ void __launch_bounds__(1024, 1) k_sweep_generic_smem(Layout L, Walkers wk, int sw_shift,
                                                                int32_t quads_per_run, RoundKeys rk,
                                                                uint32_t sweep0, int32_t nsweeps) {
    extern __shared__ __align__(16) int8_t smg[];
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
    const int rec_ints = L.rec_vec * 4;
    const int *recs = reinterpret_cast<const int *>(L.rec);
    const int jo = wide_jpack_offset(L.DC, L.DL);
    const int vec_per_row = SW >> 4;
    const int64_t nvec = static_cast<int64_t>(L.n + 1) * vec_per_row;
    for (int64_t i = threadIdx.x; i < nvec; i += blockDim.x) {
        const int64_t row = i / vec_per_row;
        const int part = static_cast<int>(i - row * vec_per_row);
        reinterpret_cast<uint4 *>(smg)[i] =
            *reinterpret_cast<const uint4 *>(L.S + row * L.Wc + col0 + 16 * part);
    }
    __syncthreads();
    auto word = [&](int off) -> uint32_t { return *reinterpret_cast<const uint32_t *>(smg + off + lane_off); };
    for (int t = 0; t < nsweeps; ++t) {
        const uint32_t sweep = sweep0 + static_cast<uint32_t>(t);
        for (int c = 0; c < L.C; ++c) {
            const int beg = __ldg(L.cofs + c), end = __ldg(L.cofs + c + 1);
            for (int pos = beg + grp; pos < end; pos += G) {
                const int *rc = recs + static_cast<int64_t>(pos) * rec_ints;
                int a0, a1, a2, a3;
                wide_fields(L, rc, jo, word, q, a0, a1, a2, a3);
                const uint4 r = keys(make_uint4(static_cast<uint32_t>(__ldg(rc + L.DC + L.DL)), sweep, lq, c3));
                *reinterpret_cast<uint32_t *>(smg + (pos << sw_shift) + lane_off) = decide_fields(q, a0, a1, a2, a3, r);
            }
            __syncthreads();
        }
    }
    const int64_t nvec_out = static_cast<int64_t>(L.n) * vec_per_row;
    for (int64_t i = threadIdx.x; i < nvec_out; i += blockDim.x) {
        const int64_t row = i / vec_per_row;
        const int part = static_cast<int>(i - row * vec_per_row);
        *reinterpret_cast<uint4 *>(L.S + row * L.Wc + col0 + 16 * part) = reinterpret_cast<const uint4 *>(smg)[i];
    }
    __shared__ long long s_F[kMaxSlab];
    __shared__ int s_g[kMaxSlab];
    for (int i = threadIdx.x; i < SW; i += blockDim.x) {
        s_F[i] = 0;
        s_g[i] = 0;
    }
    __syncthreads();
    auto own = [&](int pos) -> uint32_t { return word(pos << sw_shift); };
    wide_energies(L, jo, word, own, grp, G, s_F, s_g, lane_off);
    __syncthreads();
    for (int i = threadIdx.x; i < SW; i += blockDim.x) {
        wk.f[col0 + i] = -(s_F[i] / 4);
        wk.g[col0 + i] = s_g[i] / 2 + L.g0;
    }
}

}  // namespace

cudaError_t launch_generic_sweeps(const Layout &L, const Walkers &wk, const SweepTiling &tl,
                                  int32_t quads_per_run, uint64_t seed, uint32_t sweep0, int32_t nsweeps,
                                  cudaStream_t st) {
    if (L.DC % 4 != 0 || tl.bits) return cudaErrorInvalidValue;
    const RoundKeys rk = round_keys(seed);
    if (tl.smem) {
        int shift = 0;
        while ((1 << shift) < 4 * tl.lanes_per_spin) ++shift;
        if (shift < 4) return cudaErrorInvalidValue;
        const size_t smem = smem_sweep_bytes(L.n, 1 << shift);
        cudaError_t e = allow_max_dynamic_smem<k_sweep_generic_smem>();
        if (e != cudaSuccess) return e;
        const unsigned blocks = static_cast<unsigned>(L.Wc >> shift);
        k_sweep_generic_smem<<<blocks, tl.threads, smem, st>>>(L, wk, shift, quads_per_run, rk, sweep0, nsweeps);
        return cudaGetLastError();
    }
    int shift = 0;
    while ((1 << shift) < tl.lanes_per_spin) ++shift;
    const unsigned blocks = static_cast<unsigned>(L.Wc / (4LL * tl.lanes_per_spin));
    k_sweep_generic<<<blocks, tl.threads, 0, st>>>(L, wk, shift, quads_per_run, rk, sweep0, nsweeps);
    return cudaGetLastError();
}

}  // namespace pt2d
