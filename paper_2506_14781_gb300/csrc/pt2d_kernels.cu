// CUDA kernels of the 2D-PT library (sm_103a).
//
//  k_init_spins     initial state S0 from the seeded init stream (Algorithm 1 input)
//  k_init_walkers   walker <-> slot identity, per-walker beta/P, best-state sentinels
//  k_sweep<DC,DL>   `nsweeps` heat-bath sweeps of every walker (the sweep block of one
//                   event of Algorithm 1), colour class by colour class, then f and g
//                   of the final sweep (Eq. 1) fused as an epilogue
//  k_swap_event     one swap event per run: P-swaps (Eq. 2) or beta-swaps (Eq. 3) on
//                   odd/even pairs, then the bottom-right record (Algorithm 1)
//
// Sweep tiling.  Walkers evolve independently between swap events, so a CTA owns a
// slab of 4*QL walker columns for every spin and loops over all sweeps of the event
// with only __syncthreads() between colour classes; no grid-wide barrier is needed.
// A thread owns one quad (4 consecutive columns = one Philox call per spin) and
// keeps that quad's beta and P in registers for the whole launch.  QL lanes cover
// one spin row segment (4*QL bytes, coalesced); the CTA's QL-lane groups take
// different spins of the current colour class.
#include <cstdint>
#include <cstdio>

#include "pt2d_device.cuh"
#include "pt2d_internal.h"

namespace pt2d {
namespace {

__device__ __forceinline__ int sbyte(uint32_t x, int b) {
    return static_cast<int>(static_cast<int8_t>(static_cast<uint8_t>(x >> (8 * b))));
}

__device__ __forceinline__ uint32_t ld_word(const int8_t *p) {
    return *reinterpret_cast<const uint32_t *>(p);
}

__device__ __forceinline__ void st_word(int8_t *p, uint32_t v) {
    *reinterpret_cast<uint32_t *>(p) = v;
}

__device__ __forceinline__ uint32_t pack4(int s0, int s1, int s2, int s3) {
    return (static_cast<uint32_t>(s0) & 0xffu) | ((static_cast<uint32_t>(s1) & 0xffu) << 8) |
           ((static_cast<uint32_t>(s2) & 0xffu) << 16) | ((static_cast<uint32_t>(s3) & 0xffu) << 24);
}

constexpr int kMaxSlab = 128;  // walkers per CTA (QL <= 32)

// DC / DL: padded coupling / link degree (compile time), or -1 for the generic
// kernel that reads them from the layout.
template <int DC, int DL>
__global__ void __launch_bounds__(256) k_sweep(Layout L, Walkers wk, int ql_shift,
                                                int32_t quads_per_run, uint32_t k0, uint32_t k1,
                                                uint32_t sweep0, int32_t nsweeps) {
    const int dc = DC > 0 ? DC : L.DC;
    const int dl = DL >= 0 ? DL : L.DL;
    const int QL = 1 << ql_shift;
    const int lane_q = threadIdx.x & (QL - 1);
    const int grp = threadIdx.x >> ql_shift;
    const int G = blockDim.x >> ql_shift;
    const int64_t quad = static_cast<int64_t>(blockIdx.x) * QL + lane_q;
    const int64_t col = quad * 4;
    const uint32_t run = static_cast<uint32_t>(quad / quads_per_run);
    const uint32_t lq = static_cast<uint32_t>(quad - static_cast<int64_t>(run) * quads_per_run);
    const uint32_t c3 = (run << 4) | kTagSweep;

    const float4 bt = *reinterpret_cast<const float4 *>(wk.wbeta + col);
    const int4 pj = *reinterpret_cast<const int4 *>(wk.wP + col);
    const float kNegL2E = -1.4426950408889634f;
    const float n0 = bt.x * kNegL2E, n1 = bt.y * kNegL2E, n2 = bt.z * kNegL2E, n3 = bt.w * kNegL2E;
    int8_t *__restrict__ S = L.S;
    const int64_t Wc = L.Wc;

    for (int t = 0; t < nsweeps; ++t) {
        const uint32_t sweep = sweep0 + static_cast<uint32_t>(t);
        for (int c = 0; c < L.C; ++c) {
            const int beg = __ldg(L.cofs + c), end = __ldg(L.cofs + c + 1);
            for (int pos = beg + grp; pos < end; pos += G) {
                const int h2 = __ldg(L.h2 + pos);
                int a0 = h2, a1 = h2, a2 = h2, a3 = h2;
                const int32_t *nbp = L.nb + static_cast<int64_t>(pos) * dc;
                const int32_t *jvp = L.jv + static_cast<int64_t>(pos) * dc;
#pragma unroll
                for (int k = 0; k < (DC > 0 ? DC : 1); ++k) {
                    // compile-time trip count when DC > 0; generic loop below otherwise
                    if (DC <= 0) break;
                    const int j2 = __ldg(jvp + k);
                    const uint32_t x = ld_word(S + static_cast<int64_t>(__ldg(nbp + k)) * Wc + col);
                    a0 += j2 * sbyte(x, 0);
                    a1 += j2 * sbyte(x, 1);
                    a2 += j2 * sbyte(x, 2);
                    a3 += j2 * sbyte(x, 3);
                }
                if (DC <= 0) {
                    for (int k = 0; k < dc; ++k) {
                        const int j2 = __ldg(jvp + k);
                        const uint32_t x =
                            ld_word(S + static_cast<int64_t>(__ldg(nbp + k)) * Wc + col);
                        a0 += j2 * sbyte(x, 0);
                        a1 += j2 * sbyte(x, 1);
                        a2 += j2 * sbyte(x, 2);
                        a3 += j2 * sbyte(x, 3);
                    }
                }
                int l0 = 0, l1 = 0, l2 = 0, l3 = 0;
                const int32_t *lkp = L.lk + static_cast<int64_t>(pos) * dl;
#pragma unroll
                for (int k = 0; k < (DL > 0 ? DL : 1); ++k) {
                    if (DL <= 0) break;
                    const uint32_t y = ld_word(S + static_cast<int64_t>(__ldg(lkp + k)) * Wc + col);
                    l0 += sbyte(y, 0);
                    l1 += sbyte(y, 1);
                    l2 += sbyte(y, 2);
                    l3 += sbyte(y, 3);
                }
                if (DL < 0) {
                    for (int k = 0; k < dl; ++k) {
                        const uint32_t y =
                            ld_word(S + static_cast<int64_t>(__ldg(lkp + k)) * Wc + col);
                        l0 += sbyte(y, 0);
                        l1 += sbyte(y, 1);
                        l2 += sbyte(y, 2);
                        l3 += sbyte(y, 3);
                    }
                }
                a0 += pj.x * l0;
                a1 += pj.y * l1;
                a2 += pj.z * l2;
                a3 += pj.w * l3;
                const uint4 r = philox4x32_10(
                    make_uint4(static_cast<uint32_t>(__ldg(L.pid + pos)), sweep, lq, c3), k0, k1);
                const int s0 = heatbath(bt.x, n0, a0, r.x);
                const int s1 = heatbath(bt.y, n1, a1, r.y);
                const int s2 = heatbath(bt.z, n2, a2, r.z);
                const int s3 = heatbath(bt.w, n3, a3, r.w);
                st_word(S + static_cast<int64_t>(pos) * Wc + col, pack4(s0, s1, s2, s3));
            }
            __syncthreads();
        }
    }

    // Epilogue: f and g of the final sweep for the CTA's walkers (Eq. 1).
    // F = sum_a s_a (sum_b 2J_ab s_b + 2 * 2h_a) = 4 (sum_{a<b} J s s + sum h s), f = -F/4;
    // g counts each broken link from both ends.
    __shared__ long long s_F[kMaxSlab];
    __shared__ int s_g[kMaxSlab];
    for (int i = threadIdx.x; i < 4 * QL; i += blockDim.x) {
        s_F[i] = 0;
        s_g[i] = 0;
    }
    __syncthreads();
    long long F0 = 0, F1 = 0, F2 = 0, F3 = 0;
    int g0 = 0, g1 = 0, g2 = 0, g3 = 0;
    for (int pos = grp; pos < L.n; pos += G) {
        const uint32_t xs = ld_word(S + static_cast<int64_t>(pos) * Wc + col);
        const int h4 = 2 * __ldg(L.h2 + pos);
        int c0 = h4, c1 = h4, c2 = h4, cc3 = h4;
        for (int k = 0; k < dc; ++k) {
            const int j2 = __ldg(L.jv + static_cast<int64_t>(pos) * dc + k);
            const uint32_t x =
                ld_word(S + static_cast<int64_t>(__ldg(L.nb + static_cast<int64_t>(pos) * dc + k)) * Wc + col);
            c0 += j2 * sbyte(x, 0);
            c1 += j2 * sbyte(x, 1);
            c2 += j2 * sbyte(x, 2);
            cc3 += j2 * sbyte(x, 3);
        }
        F0 += static_cast<long long>(sbyte(xs, 0)) * c0;
        F1 += static_cast<long long>(sbyte(xs, 1)) * c1;
        F2 += static_cast<long long>(sbyte(xs, 2)) * c2;
        F3 += static_cast<long long>(sbyte(xs, 3)) * cc3;
        for (int k = 0; k < dl; ++k) {
            const int lp = __ldg(L.lk + static_cast<int64_t>(pos) * dl + k);
            if (lp == L.n) continue;
            const uint32_t y = ld_word(S + static_cast<int64_t>(lp) * Wc + col);
            g0 += sbyte(xs, 0) != sbyte(y, 0);
            g1 += sbyte(xs, 1) != sbyte(y, 1);
            g2 += sbyte(xs, 2) != sbyte(y, 2);
            g3 += sbyte(xs, 3) != sbyte(y, 3);
        }
    }
    atomicAdd(reinterpret_cast<unsigned long long *>(&s_F[lane_q * 4 + 0]), static_cast<unsigned long long>(F0));
    atomicAdd(reinterpret_cast<unsigned long long *>(&s_F[lane_q * 4 + 1]), static_cast<unsigned long long>(F1));
    atomicAdd(reinterpret_cast<unsigned long long *>(&s_F[lane_q * 4 + 2]), static_cast<unsigned long long>(F2));
    atomicAdd(reinterpret_cast<unsigned long long *>(&s_F[lane_q * 4 + 3]), static_cast<unsigned long long>(F3));
    atomicAdd(&s_g[lane_q * 4 + 0], g0);
    atomicAdd(&s_g[lane_q * 4 + 1], g1);
    atomicAdd(&s_g[lane_q * 4 + 2], g2);
    atomicAdd(&s_g[lane_q * 4 + 3], g3);
    __syncthreads();
    const int64_t col0 = static_cast<int64_t>(blockIdx.x) * QL * 4;
    for (int i = threadIdx.x; i < 4 * QL; i += blockDim.x) {
        wk.f[col0 + i] = -(s_F[i] / 4);
        wk.g[col0 + i] = s_g[i] / 2;
    }
}

__global__ void k_init_spins(Layout L, int32_t quads_per_run, uint32_t k0, uint32_t k1) {
    const int64_t quads = L.Wc / 4;
    const int64_t total = static_cast<int64_t>(L.n) * quads;
    for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t pos = e / quads;
        const int64_t quad = e - pos * quads;
        const uint32_t run = static_cast<uint32_t>(quad / quads_per_run);
        const uint32_t lq = static_cast<uint32_t>(quad - static_cast<int64_t>(run) * quads_per_run);
        const uint4 r = philox4x32_10(
            make_uint4(static_cast<uint32_t>(L.pid[pos]), 0u, lq, (run << 4) | kTagInit), k0, k1);
        const uint32_t w = pack4(r.x < 0x80000000u ? 1 : -1, r.y < 0x80000000u ? 1 : -1,
                                 r.z < 0x80000000u ? 1 : -1, r.w < 0x80000000u ? 1 : -1);
        st_word(L.S + pos * L.Wc + quad * 4, w);
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
                             int64_t nev, int dir_p, int parity) {
    extern __shared__ int at[];
    __shared__ int s_copy;
    const int run = blockIdx.x;
    const int R = rs.R, I = rs.I, J = rs.J;
    const int64_t cb = static_cast<int64_t>(run) * rs.Rp;
    const int64_t rb = static_cast<int64_t>(run) * R;
    for (int s = threadIdx.x; s < R; s += blockDim.x) at[s] = rs.walker_at[rb + s];
    __syncthreads();
    const uint32_t c3 = (static_cast<uint32_t>(run) << 4) | kTagSwap;
    const uint32_t n32 = static_cast<uint32_t>(nev);
    if (dir_p) {
        const int per_row = (J - parity) / 2;
        const int total = I * per_row;
        for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
            const int i = idx / per_row;
            const int j = parity + 2 * (idx - i * per_row);
            const int sa = i * J + j, sb = sa + 1;
            const int wa = at[sa], wb = at[sb];
            const long long dP = static_cast<long long>(rs.P[j + 1]) - rs.P[j];
            const long long dg = static_cast<long long>(wk.g[cb + wb]) - wk.g[cb + wa];
            const float x = __fmul_rn(rs.beta[i], __ll2float_rn(dP * dg));
            const uint32_t r = philox4x32_10(make_uint4(static_cast<uint32_t>(sa), n32, 0u, c3), k0, k1).x;
            if (swap_accept(x, r)) {
                at[sa] = wb;
                at[sb] = wa;
                rs.acc_P[rb + sa] += 1;
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
            const float dbeta = __fsub_rn(rs.beta[i + 1], rs.beta[i]);
            const long long Ea = wk.f[cb + wa] + static_cast<long long>(rs.P[j]) * wk.g[cb + wa];
            const long long Eb = wk.f[cb + wb] + static_cast<long long>(rs.P[j]) * wk.g[cb + wb];
            const float x = __fmul_rn(dbeta, __ll2float_rn(Eb - Ea));
            const uint32_t r = philox4x32_10(make_uint4(static_cast<uint32_t>(sa), n32, 0u, c3), k0, k1).x;
            if (swap_accept(x, r)) {
                at[sa] = wb;
                at[sb] = wa;
                rs.acc_B[rb + sa] += 1;
            }
        }
    }
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
        const int wl = at[R - 1];
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
        for (int pos = threadIdx.x; pos < L.n; pos += blockDim.x)
            rs.best_state[static_cast<int64_t>(run) * L.n + L.pid[pos]] =
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

}  // namespace

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
    const uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
    int shift = 0;
    while ((1 << shift) < tl.lanes_per_spin) ++shift;
    const int64_t slab = 4LL * tl.lanes_per_spin;
    const unsigned blocks = static_cast<unsigned>(L.Wc / slab);
    const int threads = tl.threads;
    if (L.DC == 3 && L.DL == 2)
        k_sweep<3, 2><<<blocks, threads, 0, st>>>(L, wk, shift, quads_per_run, k0, k1, sweep0, nsweeps);
    else if (L.DC == 4 && L.DL == 2)
        k_sweep<4, 2><<<blocks, threads, 0, st>>>(L, wk, shift, quads_per_run, k0, k1, sweep0, nsweeps);
    else if (L.DC == 6 && L.DL == 2)
        k_sweep<6, 2><<<blocks, threads, 0, st>>>(L, wk, shift, quads_per_run, k0, k1, sweep0, nsweeps);
    else
        k_sweep<-1, -1><<<blocks, threads, 0, st>>>(L, wk, shift, quads_per_run, k0, k1, sweep0, nsweeps);
    return cudaGetLastError();
}

cudaError_t launch_swap_event(const Layout &L, const RunState &rs, const Walkers &wk,
                              uint64_t seed, int64_t event, cudaStream_t st) {
    // Algorithm 1: direction +1 (P-swaps) for events 1, 2, then -1 (beta-swaps) for
    // 3, 4, ...: the direction flips after every even event; odd events use the
    // pairs starting at the first replica, even events those starting at the second.
    const int parity = (event % 2 == 0) ? 1 : 0;
    const int dir_p = (((event - 1) / 2) % 2 == 0) ? 1 : 0;
    const uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
    int threads = 256;
    k_swap_event<<<rs.runs, threads, sizeof(int) * rs.R, st>>>(L, rs, wk, k0, k1, event, dir_p, parity);
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
