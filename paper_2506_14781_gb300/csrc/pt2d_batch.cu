// Batched persistent 2D-PT kernel: many independent runs of many instances of
// uneven size, each with its own ladders and seed, in one launch.
//
// A CTA owns one whole run (all its replicas, R <= 128) at a time and carries it
// through `events` swap events of Algorithm 1 without leaving the kernel: the
// sweep block (colour classes separated by __syncthreads), f and g of the final
// sweep, the swap event and the bottom-right record.  CTAs pull runs from an
// atomic work counter over a list sorted by decreasing work, so a few large
// instances do not leave SMs idle at the end.  A run's spins sit in shared
// memory for the whole launch when (n + 1) * Rp bytes fit, else in its own
// region of global memory.  The arithmetic (keys, decisions, swaps) is that of
// the plain kernels, so every run follows exactly the trajectory a plain
// context with the same instance, ladders, seed and run index follows.
#include <cstdint>

#include "pt2d_batch.h"
#include "pt2d_device.cuh"
#include "pt2d_internal.h"
#include "pt2d_sweep.cuh"

namespace pt2d {
namespace {

constexpr int kMaxR = kBatchMaxReplicas;  // replicas per run (a CTA's whole slab)

template <int DC, int DL>
__device__ void run_events(const BatchArgs &a, const BatchRun &d, uint8_t *dsm) {
    uint8_t *pool = a.pool;
    const int n = d.n, Rp = d.Rp, R = d.R, I = d.I, J = d.J;
    const int QL = Rp >> 2;
    const int lane_q = threadIdx.x & (QL - 1);
    const int grp = threadIdx.x / QL;
    const int G = blockDim.x / QL;
    const int lane_off = 4 * lane_q;
    const bool smem = d.use_smem != 0;
    int8_t *S = smem ? reinterpret_cast<int8_t *>(dsm) : reinterpret_cast<int8_t *>(pool + d.state);
    const int4 *rec = reinterpret_cast<const int4 *>(pool + d.rec);
    const int32_t *cofs = reinterpret_cast<const int32_t *>(pool + d.cofs);
    int32_t *g_at = reinterpret_cast<int32_t *>(pool + d.walker_at);
    int64_t *g_f = reinterpret_cast<int64_t *>(pool + d.fg);
    int32_t *g_g = reinterpret_cast<int32_t *>(pool + d.fg + 8 * Rp);
    int64_t *acc_P = reinterpret_cast<int64_t *>(pool + d.stats);
    int64_t *acc_B = acc_P + R;
    int64_t *sum_f = acc_B + R;
    int64_t *sum_g = sum_f + R;
    int64_t *n_feas = sum_g + R;
    int64_t *trace_f = reinterpret_cast<int64_t *>(pool + d.trace);
    int64_t *trace_g = trace_f + d.trace_cap;
    int8_t *best_state = reinterpret_cast<int8_t *>(pool + d.best_state);
    int64_t *sc = reinterpret_cast<int64_t *>(pool + d.scalars);  // see BatchScalar

    // small per-run arrays after the state buffer
    uint8_t *small = dsm + a.smem_state;
    int *s_at = reinterpret_cast<int *>(small);                       // [kMaxR] slot -> walker
    int *s_slot = s_at + kMaxR;                                       // [kMaxR] walker -> slot
    long long *s_f = reinterpret_cast<long long *>(s_slot + kMaxR);   // [kMaxR]
    int *s_g = reinterpret_cast<int *>(s_f + kMaxR);                  // [kMaxR]
    float *s_beta = reinterpret_cast<float *>(s_g + kMaxR);           // [kMaxR]
    int *s_P = reinterpret_cast<int *>(s_beta + kMaxR);               // [kMaxR]
    __shared__ int s_copy;

    const int pid_at = DC + DL;
    const uint32_t k0 = d.k0, k1 = d.k1;
    const KeysBase keys{k0, k1};
    const uint32_t run = static_cast<uint32_t>(d.run);

    for (int i = threadIdx.x; i < I; i += blockDim.x) s_beta[i] = reinterpret_cast<const float *>(pool + d.beta)[i];
    for (int j = threadIdx.x; j < J; j += blockDim.x) s_P[j] = reinterpret_cast<const int32_t *>(pool + d.P)[j];
    const bool inited = sc[kScInited] != 0;
    if (!inited) {
        // initial state S0 from the init stream; walker w starts in slot w
        const int64_t total = static_cast<int64_t>(n) * QL;
        for (int64_t e = threadIdx.x; e < total; e += blockDim.x) {
            const int pos = static_cast<int>(e / QL);
            const int q = static_cast<int>(e - static_cast<int64_t>(pos) * QL);
            const uint32_t pid = static_cast<uint32_t>(
                reinterpret_cast<const int *>(rec)[static_cast<int64_t>(pos) * d.rec_vec * 4 + pid_at]);
            const uint4 r = philox4x32_10(make_uint4(pid, 0u, static_cast<uint32_t>(q), (run << 4) | kTagInit), k0, k1);
            *reinterpret_cast<uint32_t *>(S + static_cast<int64_t>(pos) * Rp + 4 * q) =
                pack_signs(r.x < 0x80000000u ? -1.0f : 1.0f, r.y < 0x80000000u ? -1.0f : 1.0f,
                           r.z < 0x80000000u ? -1.0f : 1.0f, r.w < 0x80000000u ? -1.0f : 1.0f);
        }
        for (int i = threadIdx.x; i < Rp; i += blockDim.x) S[static_cast<int64_t>(n) * Rp + i] = 0;
        for (int s = threadIdx.x; s < R; s += blockDim.x) s_at[s] = s;
    } else {
        if (smem) {
            const int64_t nvec = (static_cast<int64_t>(n + 1) * Rp) >> 4;
            const uint4 *src = reinterpret_cast<const uint4 *>(pool + d.state);
            for (int64_t i = threadIdx.x; i < nvec; i += blockDim.x) reinterpret_cast<uint4 *>(S)[i] = src[i];
        }
        for (int s = threadIdx.x; s < R; s += blockDim.x) s_at[s] = g_at[s];
    }
    __syncthreads();
    if (threadIdx.x == 0 && !inited) {
        sc[kScBestF] = INT64_MAX;
        sc[kScBestEvent] = -1;
        sc[kScSolvedEvent] = -1;
        sc[kScInited] = 1;
    }
    int64_t sweeps_done = sc[kScSweeps];
    int64_t events_done = sc[kScEvents];

    auto fetch = [&](int row) -> uint32_t {
        return *reinterpret_cast<const uint32_t *>(S + static_cast<int64_t>(row) * Rp + lane_off);
    };
    const float kNegL2E = -1.4426950408889634f;

    for (int e = 0; e < a.events; ++e) {
        const int64_t nev = events_done + 1;
        // walker -> slot, and this thread's four walkers' beta and P
        for (int w = threadIdx.x; w < Rp; w += blockDim.x) s_slot[w] = -1;
        __syncthreads();
        for (int s = threadIdx.x; s < R; s += blockDim.x) s_slot[s_at[s]] = s;
        __syncthreads();
        Quad q;
        {
            float b[4];
            int p[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int sl = s_slot[lane_off + k];
                b[k] = sl >= 0 ? s_beta[sl / J] : 0.0f;
                p[k] = sl >= 0 ? s_P[sl % J] : 0;
            }
            q = Quad{b[0], b[1], b[2], b[3], b[0] * kNegL2E, b[1] * kNegL2E, b[2] * kNegL2E,
                     b[3] * kNegL2E, p[0], p[1], p[2], p[3]};
        }
        const uint32_t c3 = (run << 4) | kTagSweep;
        for (int t = 0; t < a.interval; ++t) {
            const uint32_t sweep = static_cast<uint32_t>(sweeps_done + t);
            for (int c = 0; c < d.C; ++c) {
                const int beg = __ldg(cofs + c), end = __ldg(cofs + c + 1);
                for (int pos = beg + grp; pos < end; pos += G) {
                    Rec<DC, DL> rc;
                    rc.load(rec, pos);
                    const uint32_t w = update4<DC, DL>(rc, q, fetch, sweep, static_cast<uint32_t>(lane_q), c3, keys);
                    *reinterpret_cast<uint32_t *>(S + static_cast<int64_t>(pos) * Rp + lane_off) = w;
                }
                __syncthreads();
            }
        }
        // f and g of the final sweep (Eq. 1), reduced over the CTA's spin groups
        for (int i = threadIdx.x; i < Rp; i += blockDim.x) {
            s_f[i] = 0;
            s_g[i] = 0;
        }
        __syncthreads();
        {
            long long F0 = 0, F1 = 0, F2 = 0, F3 = 0;
            int g0 = 0, g1 = 0, g2 = 0, g3 = 0;
            for (int pos = grp; pos < n; pos += G) {
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
                    if (rc.lk(l) == n) continue;
                    const uint32_t y = fetch(rc.lk(l));
                    g0 += sbyte<0>(xs) != sbyte<0>(y);
                    g1 += sbyte<1>(xs) != sbyte<1>(y);
                    g2 += sbyte<2>(xs) != sbyte<2>(y);
                    g3 += sbyte<3>(xs) != sbyte<3>(y);
                }
            }
            unsigned long long *uf = reinterpret_cast<unsigned long long *>(s_f);
            atomicAdd(uf + lane_off + 0, static_cast<unsigned long long>(F0));
            atomicAdd(uf + lane_off + 1, static_cast<unsigned long long>(F1));
            atomicAdd(uf + lane_off + 2, static_cast<unsigned long long>(F2));
            atomicAdd(uf + lane_off + 3, static_cast<unsigned long long>(F3));
            atomicAdd(s_g + lane_off + 0, g0);
            atomicAdd(s_g + lane_off + 1, g1);
            atomicAdd(s_g + lane_off + 2, g2);
            atomicAdd(s_g + lane_off + 3, g3);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < Rp; i += blockDim.x) {
            s_f[i] = -(s_f[i] / 4);
            s_g[i] = s_g[i] / 2;
        }
        __syncthreads();
        // swap event (Eq. 2 / Eq. 3, Algorithm 1)
        swap_pairs(s_at, [&](int w) { return s_f[w]; }, [&](int w) { return s_g[w]; }, s_beta, s_P,
                   I, J, run, nev, event_is_pswap(nev), k0, k1, acc_P, acc_B);
        __syncthreads();
        // per-slot sums and the bottom-right record
        for (int s = threadIdx.x; s < R; s += blockDim.x) {
            const int w = s_at[s];
            sum_f[s] += s_f[w];
            sum_g[s] += s_g[w];
            n_feas[s] += (s_g[w] == 0);
        }
        if (threadIdx.x == 0) {
            const int wl = s_at[R - 1];
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
            s_copy = copy;
        }
        __syncthreads();
        if (s_copy >= 0) {
            const int wc = s_copy;
            for (int pos = threadIdx.x; pos < n; pos += blockDim.x)
                best_state[reinterpret_cast<const int *>(rec)[static_cast<int64_t>(pos) * d.rec_vec * 4 + pid_at]] =
                    S[static_cast<int64_t>(pos) * Rp + wc];
        }
        sweeps_done += a.interval;
        events_done = nev;
        __syncthreads();
    }
    // write back
    for (int s = threadIdx.x; s < R; s += blockDim.x) g_at[s] = s_at[s];
    for (int i = threadIdx.x; i < Rp; i += blockDim.x) {
        g_f[i] = s_f[i];
        g_g[i] = s_g[i];
    }
    if (smem) {
        const int64_t nvec = (static_cast<int64_t>(n + 1) * Rp) >> 4;
        uint4 *dst = reinterpret_cast<uint4 *>(pool + d.state);
        for (int64_t i = threadIdx.x; i < nvec; i += blockDim.x) dst[i] = reinterpret_cast<const uint4 *>(S)[i];
    }
    if (threadIdx.x == 0) {
        sc[kScSweeps] = sweeps_done;
        sc[kScEvents] = events_done;
    }
}

__device__ void write_status(const BatchArgs &a, int item, const BatchRun &d) {
    const int64_t *sc = reinterpret_cast<const int64_t *>(a.pool + d.scalars);
    a.status[2 * item] = sc[kScSolvedEvent];
    a.status[2 * item + 1] = sc[kScEvents];
}

template <int DC, int DL>
__global__ void __launch_bounds__(1024, 1) k_batch(BatchArgs a) {
    extern __shared__ __align__(16) uint8_t dsm[];
    __shared__ int s_item;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(a.queue, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= a.n_runs) break;
        const BatchRun d = a.runs[item];
        run_events<DC, DL>(a, d, dsm);
        __syncthreads();
        if (threadIdx.x == 0) write_status(a, item, d);
    }
}

template <int DC, int DL>
cudaError_t launch_batch_variant(const BatchArgs &a, int grid, int threads, size_t smem, cudaStream_t st) {
    k_batch<DC, DL><<<grid, threads, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

size_t batch_small_smem_bytes() {
    return static_cast<size_t>(kMaxR) * (4 + 4 + 8 + 4 + 4 + 4);
}

cudaError_t batch_kernel_attributes(int DC, int DL, int smem_state) {
    const int smem = smem_state + static_cast<int>(batch_small_smem_bytes());
    if (DL != 2) return cudaErrorInvalidValue;
    if (DC == 3) return cudaFuncSetAttribute(k_batch<3, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (DC == 4) return cudaFuncSetAttribute(k_batch<4, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (DC == 6) return cudaFuncSetAttribute(k_batch<6, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    return cudaErrorInvalidValue;
}

cudaError_t launch_batch(const BatchArgs &a, int DC, int DL, int grid, int threads, cudaStream_t st) {
    const size_t smem = static_cast<size_t>(a.smem_state) + batch_small_smem_bytes();
    if (DL != 2) return cudaErrorInvalidValue;
    if (DC == 3) return launch_batch_variant<3, 2>(a, grid, threads, smem, st);
    if (DC == 4) return launch_batch_variant<4, 2>(a, grid, threads, smem, st);
    if (DC == 6) return launch_batch_variant<6, 2>(a, grid, threads, smem, st);
    return cudaErrorInvalidValue;
}

}  // namespace pt2d
