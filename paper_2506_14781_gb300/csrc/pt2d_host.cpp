// Host side of the 2D-PT C ABI (include/pt2d.h): validation, greedy colouring,
// device layout, the Algorithm 1 event loop and the read/write interface.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <map>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/pt2d.h"
#include "pt2d_generic.h"
#include "pt2d_internal.h"
#include "pt2d_penalty.h"
#include "pt2d_prep.h"
#include "pt2d_trace.h"
#include "pt2d_wide.cuh"

namespace {

constexpr int64_t kHBound = int64_t(1) << 24;  // |H| must stay exact in float32
constexpr int64_t kMaxSlots = 8192;             // I * J per run

// Sum of sizes with 256-byte alignment; two passes (size, then assignment).
struct Carver {
    char *base;
    size_t off = 0;
    explicit Carver(void *b) : base(static_cast<char *>(b)) {}
    template <typename T>
    T *take(int64_t count) {
        off = (off + 255) & ~size_t(255);
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += sizeof(T) * static_cast<size_t>(count > 0 ? count : 1);
        return p;
    }
};

std::atomic<int32_t> g_fail_allocs{0};  // injected allocation failures still to come

// Validates a symmetric CSR (no self loops, no duplicates, equal values both
// ways; `val` may be NULL for unweighted links) and returns sorted adjacency.
// Adjacency of a validated CSR: one flat array of (neighbour, value) pairs,
// each row sorted by neighbour (a row per spin, no allocation per row).
struct Adjacency {
    std::vector<int32_t> ptr;
    std::vector<std::pair<int32_t, int32_t>> e;
    struct Row {
        std::pair<int32_t, int32_t> *b, *en;
        std::pair<int32_t, int32_t> *begin() const { return b; }
        std::pair<int32_t, int32_t> *end() const { return en; }
        size_t size() const { return static_cast<size_t>(en - b); }
        std::pair<int32_t, int32_t> &operator[](size_t i) const { return b[i]; }
    };
    Row operator[](int32_t a) { return Row{e.data() + ptr[a], e.data() + ptr[a + 1]}; }
};

int check_csr(int32_t n, const int32_t *ptr, const int32_t *col, const int16_t *val, Adjacency *adj) {
    if (!ptr) return PT2D_ERR_INVALID_ARG;
    if (ptr[0] != 0) return PT2D_ERR_INVALID_ARG;
    for (int32_t a = 0; a < n; ++a)
        if (ptr[a + 1] < ptr[a]) return PT2D_ERR_INVALID_ARG;
    if (ptr[n] > 0 && !col) return PT2D_ERR_INVALID_ARG;
    adj->ptr.assign(ptr, ptr + n + 1);
    adj->e.resize(static_cast<size_t>(ptr[n]));
    for (int32_t a = 0; a < n; ++a) {
        for (int32_t k = ptr[a]; k < ptr[a + 1]; ++k) {
            const int32_t b = col[k];
            if (b < 0 || b >= n || b == a) return PT2D_ERR_INVALID_ARG;
            adj->e[k] = {b, val ? static_cast<int32_t>(val[k]) : 0};
        }
        auto v = (*adj)[a];
        std::sort(v.begin(), v.end());
        for (size_t i = 1; i < v.size(); ++i)
            if (v[i].first == v[i - 1].first) return PT2D_ERR_INVALID_ARG;  // duplicate edge
    }
    // symmetry with equal values
    for (int32_t a = 0; a < n; ++a)
        for (const auto &e : (*adj)[a]) {
            const auto w = (*adj)[e.first];
            auto it = std::lower_bound(w.begin(), w.end(), std::make_pair(a, INT32_MIN));
            if (it == w.end() || it->first != a || it->second != e.second) return PT2D_ERR_INVALID_ARG;
        }
    return PT2D_OK;
}

}  // namespace

namespace pt2d {

cudaError_t device_alloc(void **ptr, size_t bytes) {
    int32_t left = g_fail_allocs.load();
    while (left > 0) {
        if (g_fail_allocs.compare_exchange_weak(left, left - 1)) return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(ptr, bytes);
}

int check_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PT2D_ERR_UNSUPPORTED;
    int major = 0, minor = 0;
    if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess)
        return PT2D_ERR_UNSUPPORTED;
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (major != 10 || minor != 3) return PT2D_ERR_UNSUPPORTED;
    return PT2D_OK;
}

int prepare(const pt2d_instance *inst, int32_t I, const float *beta, int32_t J, const int32_t *P,
            int32_t runs, const pt2d_options *opt, Prep &pp, int force_dc, bool records) {
    if (!inst || inst->n < 1 || I < 1 || J < 1 || runs < 1) return PT2D_ERR_INVALID_ARG;
    // the swap kernel keeps one run's slot -> walker map in shared memory
    if (static_cast<int64_t>(I) * J > kMaxSlots) return PT2D_ERR_INVALID_ARG;
    if (runs >= (1 << 27)) return PT2D_ERR_INVALID_ARG;
    const int32_t n = inst->n;
    Adjacency cadj, ladj;
    if (!inst->cp_ptr || !inst->lk_ptr) return PT2D_ERR_INVALID_ARG;
    if (inst->cp_ptr[n] > 0 && !inst->cp_J) return PT2D_ERR_INVALID_ARG;
    int st = check_csr(n, inst->cp_ptr, inst->cp_col, inst->cp_J, &cadj);
    if (st) return st;
    st = check_csr(n, inst->lk_ptr, inst->lk_col, inst->lk_w, &ladj);
    if (st) return st;
    // penalty terms: link weights K (1 without lk_w), penalty field k, constant g0
    bool penalty = false;
    int64_t gbound = std::abs(inst->g0);
    for (int32_t a = 0; a < n; ++a) {
        for (auto &e : ladj[a]) {
            if (!inst->lk_w) e.second = 1;
            if (e.second != 1) penalty = true;
            gbound += std::abs(static_cast<int64_t>(e.second));  // each link twice: 2x bound
        }
        if (inst->hk) {
            if (inst->hk[a] != 0) penalty = true;
            gbound += std::abs(static_cast<int64_t>(inst->hk[a]));
        }
    }
    if (gbound >= (int64_t(1) << 31)) return PT2D_ERR_INVALID_ARG;
    if (force_dc > 0 && (penalty || inst->g0 != 0)) return PT2D_ERR_INVALID_ARG;
    pp.penalty = penalty;
    pp.g0 = static_cast<int32_t>(inst->g0);
    // ladders: beta >= 0 finite and ascending, P >= 0 ascending
    if (beta) {
        for (int32_t i = 0; i < I; ++i) {
            if (!(beta[i] >= 0.0f) || !(beta[i] < 3.0e38f)) return PT2D_ERR_INVALID_ARG;
            if (i > 0 && beta[i] < beta[i - 1]) return PT2D_ERR_INVALID_ARG;
        }
    }
    int64_t Pmax = 0;
    if (P) {
        for (int32_t j = 0; j < J; ++j) {
            if (P[j] < 0) return PT2D_ERR_INVALID_ARG;
            if (j > 0 && P[j] < P[j - 1]) return PT2D_ERR_INVALID_ARG;
            Pmax = std::max<int64_t>(Pmax, P[j]);
        }
    }
    // local-field bound |H_a| < 2^24
    for (int32_t a = 0; a < n; ++a) {
        int64_t b = 0;
        for (const auto &e : cadj[a]) b += 2 * std::abs(static_cast<int64_t>(e.second));
        if (inst->h) b += 2 * std::abs(static_cast<int64_t>(inst->h[a]));
        int64_t pen = inst->hk ? std::abs(static_cast<int64_t>(inst->hk[a])) : 0;
        for (const auto &e : ladj[a]) pen += std::abs(static_cast<int64_t>(e.second));
        b += Pmax * pen;
        if (b >= kHBound) return PT2D_ERR_INVALID_ARG;
    }
    // colouring: given (must be proper) or greedy over couplings and links
    pp.color.assign(n, -1);
    if (inst->color) {
        for (int32_t a = 0; a < n; ++a) {
            if (inst->color[a] < 0 || inst->color[a] >= 4096) return PT2D_ERR_INVALID_ARG;
            pp.color[a] = inst->color[a];
        }
        for (int32_t a = 0; a < n; ++a) {
            for (const auto &e : cadj[a])
                if (pp.color[e.first] == pp.color[a]) return PT2D_ERR_INVALID_ARG;
            for (const auto &e : ladj[a])
                if (pp.color[e.first] == pp.color[a]) return PT2D_ERR_INVALID_ARG;
        }
    } else {
        std::vector<char> used;
        for (int32_t a = 0; a < n; ++a) {
            used.assign(cadj[a].size() + ladj[a].size() + 2, 0);
            for (const auto &e : cadj[a])
                if (e.first < a && pp.color[e.first] < static_cast<int32_t>(used.size()))
                    used[pp.color[e.first]] = 1;
            for (const auto &e : ladj[a])
                if (e.first < a && pp.color[e.first] < static_cast<int32_t>(used.size()))
                    used[pp.color[e.first]] = 1;
            int32_t c = 0;
            while (used[c]) ++c;
            pp.color[a] = c;
        }
    }
    int32_t C = 0;
    for (int32_t a = 0; a < n; ++a) C = std::max(C, pp.color[a] + 1);
    // positions: spins sorted by (colour, id)
    pp.cofs.assign(C + 1, 0);
    for (int32_t a = 0; a < n; ++a) pp.cofs[pp.color[a] + 1]++;
    for (int32_t c = 0; c < C; ++c) pp.cofs[c + 1] += pp.cofs[c];
    pp.pid.assign(n, 0);
    pp.pos_of.assign(n, 0);
    {
        std::vector<int32_t> fill(pp.cofs.begin(), pp.cofs.end() - 1);
        for (int32_t a = 0; a < n; ++a) {
            const int32_t p = fill[pp.color[a]]++;
            pp.pid[p] = a;
            pp.pos_of[a] = p;
        }
    }
    // padded degrees
    int32_t dcmax = 0, dlmax = 0;
    for (int32_t a = 0; a < n; ++a) {
        dcmax = std::max<int32_t>(dcmax, static_cast<int32_t>(cadj[a].size()));
        dlmax = std::max<int32_t>(dlmax, static_cast<int32_t>(ladj[a].size()));
    }
    // Record layout.  Without penalty terms and with coupling degree <= 6 and
    // two copy links: the specialised layouts (coupling width 3, 4 or 6), or the
    // width a batch forces.  Otherwise decided after the tiling: the
    // penalty-specialised layout when that kernel will sweep the instance, else
    // the wide layout of the runtime-degree kernels (force_dc < 0 asks for it).
    int32_t DC = 0, DL = 0;
    const bool spec_layout = force_dc > 0 || (force_dc == 0 && !penalty && dlmax <= 2 && dcmax <= 6);
    if (force_dc > 0) {
        if (dlmax > 2 || dcmax > force_dc) return PT2D_ERR_INVALID_ARG;
        DC = force_dc;
        DL = 2;
    } else if (spec_layout) {
        DL = 2;
        DC = dcmax <= 3 ? 3 : (dcmax <= 4 ? 4 : 6);
    }
    pp.dcmax = dcmax;
    pp.n = n;
    pp.I = I;
    pp.J = J;
    pp.R = I * J;
    pp.Rp = (pp.R + 3) / 4 * 4;
    pp.runs = runs;
    pp.C = C;
    pp.trace_cap = opt ? std::max<int32_t>(opt->trace_capacity, 0) : 1024;
    // Sweep tiling.  The shared-memory kernels hold a CTA's whole slab,
    // (n + 1) x SW bytes (int8) or (n + 1) x SW / 8 bytes (bit-packed, the
    // specialised layouts only), for the swap interval; otherwise the slab
    // stays in global memory.
    int sms = 152, smem_max = 232448;
    {
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess) {
            int v = 0;
            if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
                sms = v;
            if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess &&
                v > 0)
                smem_max = v;
        } else {
            cudaGetLastError();
        }
    }
    const int mode = opt ? opt->sweep_kernel : 0;
    if (mode < 0 || mode > 3) return PT2D_ERR_INVALID_ARG;
    if (opt && opt->swap_mode != PT2D_SWAP_2D && opt->swap_mode != PT2D_SWAP_JCOLUMN)
        return PT2D_ERR_INVALID_ARG;
    const bool specialised = !penalty && DL == 2 && (DC == 3 || DC == 4 || DC == 6);
    // penalty terms with small degrees: the penalty-specialised kernels (int8 or bit-packed slab)
    const bool pen_ok = !spec_layout && force_dc == 0 && penalty && dcmax <= 6 && dlmax <= 3;
    // bit-packed slabs: specialised and penalty-specialised layouts only
    if (mode == 3 && !specialised && !pen_ok) return PT2D_ERR_INVALID_ARG;
    const int64_t walkers = static_cast<int64_t>(runs) * pp.Rp;
    auto fits = [&](int sw) {
        return pt2d::smem_sweep_bytes(n, sw) + pt2d::kSweepStaticSmem <= static_cast<size_t>(smem_max);
    };
    const int req_w = opt ? opt->walkers_per_cta : 0;
    if (req_w != 0 && (req_w < 4 || req_w > 128 || (req_w & (req_w - 1)))) return PT2D_ERR_INVALID_ARG;
    // Slab width choice.  Wider slabs share each neighbour record among more
    // walkers; narrower ones give more CTAs.  A CTA (up to 1024 threads, ~60
    // registers each, most of shared memory) holds an SM alone, so the grid runs
    // in waves of `sms` CTAs and a last partial wave leaves SMs idle.  Take the
    // widest fitting width that fills at least one wave with waves at least 85 %
    // full, else the one with the fullest waves (the wider on ties); when no
    // width fills one wave, the narrowest (most CTAs, most spin groups per CTA).
    auto pick_width = [&](int widest, int narrowest, auto fits_width) -> int {
        int best = 0, smallest = 0;
        double best_eff = -1.0;
        for (int cand = widest; cand >= narrowest; cand /= 2) {
            if (!fits_width(cand)) continue;
            smallest = cand;
            const int64_t ctas = (walkers + cand - 1) / cand;
            if (ctas < sms) continue;
            const double waves = static_cast<double>(ctas) / sms;
            const double eff = waves / std::ceil(waves);
            if (eff >= 0.85) return cand;
            if (eff > best_eff) {
                best_eff = eff;
                best = cand;
            }
        }
        return best ? best : smallest;
    };
    // int8 shared-memory slab width (0 = global kernel): the specialised, the
    // penalty-specialised or the runtime-degree shared-memory kernel.
    int sw = 0;
    if (mode == 0 || mode == 2) {
        if (req_w) {
            if (req_w >= 16 && fits(req_w)) sw = req_w;
        } else {
            sw = pick_width(128, 16, fits);
        }
    }
    // bit-packed shared-memory slab when the int8 one does not fit (or when forced)
    int bw = 0;
    auto fits_bits = [&](int cand) {
        return pt2d::bits_sweep_bytes(n, cand) + pt2d::kSweepStaticSmem <= static_cast<size_t>(smem_max);
    };
    if ((specialised || pen_ok) && (mode == 3 || (mode == 0 && sw == 0))) {
        sw = 0;
        if (req_w) {
            if (req_w >= 8 && fits_bits(req_w)) bw = req_w;
        } else {
            bw = pick_width(128, 8, fits_bits);
        }
        if (mode == 3 && bw == 0) return PT2D_ERR_INVALID_ARG;
    }
    if (mode == 2 && sw == 0) return PT2D_ERR_INVALID_ARG;
    int ql, threads, wpt = 4;
    if (bw) {
        // a thread owns a byte of 8 walkers (k_sweep_bits8 / k_sweep_penalty_bits8),
        // or a nibble of 4 when asked for or when more threads than those kernels
        // take are asked for (k_sweep_bits / k_sweep_penalty_bits)
        const int req_t = opt ? opt->walkers_per_thread : 0;
        const int req_threads = opt ? opt->threads_per_cta : 0;
        if (req_t != 0 && req_t != 4 && req_t != 8) return PT2D_ERR_INVALID_ARG;
        // k_sweep_bits8 runs up to 896 threads at 72 registers (N = 800: 1.4 %
        // faster than 640 threads, which were 5 % faster than 512)
        const int tmax8 = specialised ? pt2d::kBits8Threads : pt2d::kPenaltyBits8Threads;
        wpt = req_t ? req_t : (req_threads <= tmax8 ? 8 : 4);
        ql = bw / 4;
        const int lanes = bw / wpt;  // threads per spin row
        const int tmax = wpt == 4 ? 1024 : tmax8;
        int32_t widest = 0;
        for (int32_t c = 0; c < C; ++c) widest = std::max(widest, pp.cofs[c + 1] - pp.cofs[c]);
        const int64_t want = (static_cast<int64_t>(widest) * lanes + 31) / 32 * 32;
        threads = req_threads > 0 ? req_threads : static_cast<int>(std::min<int64_t>(tmax, want));
        if (threads < 32 || threads > tmax || threads % 32 || threads < lanes) return PT2D_ERR_INVALID_ARG;
    } else
    if (sw) {
        ql = sw / 4;
        // the specialised layouts' int8 kernel: a thread owns 8 walkers (two
        // quads) at up to 768 threads unless 4 or more threads are asked for
        // (N = 200: 14.26 ms per launch against 14.84 with 4 walkers at 1024)
        const int req_t = opt ? opt->walkers_per_thread : 0;
        const int req_threads = opt ? opt->threads_per_cta : 0;
        if (req_t != 0 && req_t != 4 && req_t != 8) return PT2D_ERR_INVALID_ARG;
        if (req_t == 8 && !specialised) return PT2D_ERR_INVALID_ARG;
        wpt = req_t ? req_t : (specialised && req_threads <= 768 ? 8 : 4);
        const int lanes = sw / wpt;  // threads per spin row segment
        const int tmax = wpt == 4 ? 1024 : 768;
        int32_t widest = 0;
        for (int32_t c = 0; c < C; ++c) widest = std::max(widest, pp.cofs[c + 1] - pp.cofs[c]);
        const int64_t want = (static_cast<int64_t>(widest) * lanes + 31) / 32 * 32;
        // the runtime-degree kernel (wide records) runs smaller CTAs when there
        // are CTAs enough to put several on each SM: its colour classes are short
        // (three copies per node, N = 50 / 100 / 200: 4 or 5 classes of <= 200
        // spins), so a 1024-thread CTA waits at the class barriers, while CTAs
        // sharing an SM overlap one another's barriers (400 CTAs, N = 100: 1.99 ms
        // per launch at 256 threads against 2.06 at 320 and 2.29 at 1024; N = 50:
        // 0.79 against 0.95; N = 200: 6.54 / 7.32).  With no more CTAs than SMs
        // (one run of 400 replicas: 7) each keeps the full width.
        const bool wide_kernel = !spec_layout && !pen_ok;
        const int64_t ctas = (walkers + sw - 1) / sw;
        const int64_t per_sm = (ctas + sms - 1) / sms;
        const int tauto = wide_kernel && per_sm > 1
                              ? static_cast<int>(std::max<int64_t>(256, (1024 / (per_sm + 1)) / 32 * 32))
                              : tmax;
        threads = (opt && opt->threads_per_cta > 0) ? opt->threads_per_cta
                                                    : static_cast<int>(std::min<int64_t>(tauto, want));
        if (threads < 32 || threads > tmax || threads % 32 || threads < lanes) return PT2D_ERR_INVALID_ARG;
    } else {
        if (opt && opt->walkers_per_thread != 0 && opt->walkers_per_thread != 4)
            return PT2D_ERR_INVALID_ARG;
        if (req_w) {
            ql = req_w / 4;
        } else {
            const int64_t quads = walkers / 4;
            ql = 32;
            while (ql > 1 && (quads + ql - 1) / ql < 2LL * sms) ql /= 2;
        }
        threads = (opt && opt->threads_per_cta > 0) ? opt->threads_per_cta : 256;
        if (threads < 32 || threads > 256 || threads % 32 || threads < ql) return PT2D_ERR_INVALID_ARG;
    }
    pp.tiling.lanes_per_spin = ql;
    pp.tiling.threads = threads;
    pp.tiling.smem = sw != 0;
    pp.tiling.bits = bw != 0;
    pp.tiling.walkers_per_thread = wpt;
    pp.pen_kernel = pen_ok && ((sw != 0 && wpt == 4) || bw != 0);
    if (pp.pen_kernel) {
        // padded up to a layout of the penalty-specialised kernel (padding
        // entries point at the zero row with J = 0, K = 0)
        DC = dcmax <= 3 ? 3 : (dcmax <= 4 ? 4 : 6);
        DL = dlmax <= 2 ? 2 : 3;
        if (!pt2d::penalty_kernel_degrees(DC, DL)) return PT2D_ERR_INVALID_ARG;
    } else if (!spec_layout) {
        DC = std::max<int32_t>(4, (dcmax + 3) / 4 * 4);
        DL = dlmax;
    }
    pp.wide = !spec_layout && !pp.pen_kernel;
    pp.DC = DC;
    pp.DL = DL;
    // packed records (the spin id at DC + DL in every layout), padded to whole int4s:
    //  specialised / penalty-specialised: [nb x DC, lk x DL, pid, 2h, 2J x DC] and,
    //  with penalty terms, [K x DL, k];  wide: see pt2d_wide.cuh
    const int32_t jo = pt2d::wide_jpack_offset(DC, DL);
    const int32_t rec_ints = pp.wide ? pt2d::wide_record_ints(DC, DL, penalty)
                                     : 2 * DC + DL + 2 + (penalty ? DL + 1 : 0);
    const int32_t rec_vec = (rec_ints + 3) / 4;
    const size_t ri = static_cast<size_t>(rec_vec) * 4;
    pp.rec_vec = rec_vec;
    // neighbour references become byte offsets into the shared-memory slab
    const int scale = sw ? sw : (bw ? bw / 8 : 1);
    pp.pad_ref = n * scale;
    const int64_t slab = 4LL * ql;
    pp.Wc = (walkers + slab - 1) / slab * slab;
    if (!records) return PT2D_OK;
    pp.rec.assign(static_cast<size_t>(n) * ri, 0);
    for (int32_t p = 0; p < n; ++p) {
        const int32_t a = pp.pid[p];
        int32_t *r = pp.rec.data() + static_cast<size_t>(p) * ri;
        for (int32_t k = 0; k < DC; ++k) r[k] = n;
        for (int32_t k = 0; k < DL; ++k) r[DC + k] = n;
        for (size_t k = 0; k < cadj[a].size(); ++k) {
            r[k] = pp.pos_of[cadj[a][k].first];
            const int32_t Jk = cadj[a][k].second;
            if (pp.wide) {  // J = 256 hi + lo, byte k % 4 of group k / 4
                const uint32_t lo = static_cast<uint32_t>(Jk) & 0xFFu;
                const uint32_t hi = static_cast<uint32_t>(Jk >> 8) & 0xFFu;
                uint32_t *g = reinterpret_cast<uint32_t *>(r + jo + 2 * (k / 4));
                g[0] |= lo << (8 * (k % 4));
                g[1] |= hi << (8 * (k % 4));
            } else {
                r[DC + DL + 2 + k] = 2 * Jk;
            }
        }
        for (size_t k = 0; k < ladj[a].size(); ++k) r[DC + k] = pp.pos_of[ladj[a][k].first];
        r[DC + DL] = a;
        r[DC + DL + 1] = inst->h ? 2 * inst->h[a] : 0;
        if (spec_layout && DC == 3 && DL == 2) {  // packed J bytes for the dp4a field sums
            uint32_t lo = 0, hi = 0;
            for (size_t k = 0; k < cadj[a].size(); ++k) {
                lo |= (static_cast<uint32_t>(cadj[a][k].second) & 0xFFu) << (8 * k);
                hi |= (static_cast<uint32_t>(cadj[a][k].second >> 8) & 0xFFu) << (8 * k);
            }
            r[10] = static_cast<int32_t>(lo);
            r[11] = static_cast<int32_t>(hi);
        }
        if (penalty) {
            const int32_t ko = pp.wide ? jo + DC / 2 : 2 * DC + DL + 2;
            for (size_t k = 0; k < ladj[a].size(); ++k) r[ko + k] = ladj[a][k].second;
            r[ko + DL] = inst->hk ? inst->hk[a] : 0;
        }
    }
    if (scale > 1) {
        const size_t ri2 = static_cast<size_t>(pp.rec_vec) * 4;
        for (int32_t p = 0; p < n; ++p)
            for (int32_t k = 0; k < DC + DL; ++k) pp.rec[static_cast<size_t>(p) * ri2 + k] *= scale;
    }
    return PT2D_OK;
}

}  // namespace pt2d

namespace {

using pt2d::Prep;
using pt2d::prepare;


}  // namespace

struct pt2d_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_ws = false;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    Prep pp;
    pt2d::Layout L{};
    pt2d::Walkers wk{};
    pt2d::RunState rs{};
    float *d_beta = nullptr;
    int32_t *d_P = nullptr;
    int64_t *d_target = nullptr;
    std::vector<float> beta;
    std::vector<int32_t> P;
    int64_t sweeps_done = 0, events_done = 0, dir = 1, inited = 0;
    uint64_t seed = 0;
    int64_t launches = 0;
    int last_cuda = 0;
    bool adopt_seed = false;  // initialised by a checkpoint restore: take the next run's seed
    // kernel timing (opt.profile): pending event pairs per kernel kind, and totals
    bool profile = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending[2];
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> spare;
    double total_ms[2] = {0.0, 0.0};
    int64_t timed_launches[2] = {0, 0};
};

namespace {

size_t carve(pt2d_ctx *c, void *base) {
    Prep &pp = c->pp;
    Carver cv(base);
    const int64_t n = pp.n, RR = static_cast<int64_t>(pp.runs) * pp.R;
    c->L.S = cv.take<int8_t>((n + 1) * pp.Wc);
    c->L.rec = cv.take<int4>(n * pp.rec_vec);
    c->L.cofs = cv.take<int32_t>(pp.C + 1);
    c->wk.wbeta = cv.take<float>(pp.Wc);
    c->wk.wP = cv.take<int32_t>(pp.Wc);
    c->wk.f = cv.take<int64_t>(pp.Wc);
    c->wk.g = cv.take<int32_t>(pp.Wc);
    c->d_beta = cv.take<float>(pp.I);
    c->d_P = cv.take<int32_t>(pp.J);
    c->rs.walker_at = cv.take<int32_t>(RR);
    c->rs.acc_P = cv.take<int64_t>(RR);
    c->rs.acc_B = cv.take<int64_t>(RR);
    c->rs.sum_f = cv.take<int64_t>(RR);
    c->rs.sum_g = cv.take<int64_t>(RR);
    c->rs.n_feasible = cv.take<int64_t>(RR);
    c->rs.trace_f = cv.take<int64_t>(static_cast<int64_t>(pp.runs) * pp.trace_cap);
    c->rs.trace_g = cv.take<int64_t>(static_cast<int64_t>(pp.runs) * pp.trace_cap);
    c->rs.best_f = cv.take<int64_t>(pp.runs);
    c->rs.best_event = cv.take<int64_t>(pp.runs);
    c->rs.solved_event = cv.take<int64_t>(pp.runs);
    c->d_target = cv.take<int64_t>(pp.runs);
    c->rs.best_state = cv.take<int8_t>(static_cast<int64_t>(pp.runs) * n);
    return cv.off + 256;
}

std::pair<cudaEvent_t, cudaEvent_t> take_events(pt2d_ctx *c) {
    if (!c->spare.empty()) {
        auto p = c->spare.back();
        c->spare.pop_back();
        return p;
    }
    std::pair<cudaEvent_t, cudaEvent_t> p{nullptr, nullptr};
    cudaEventCreate(&p.first);
    cudaEventCreate(&p.second);
    return p;
}

// Fold finished event pairs into the totals (after a stream synchronisation).
cudaError_t drain_events(pt2d_ctx *c) {
    for (int k = 0; k < 2; ++k) {
        for (auto &p : c->pending[k]) {
            float ms = 0.0f;
            cudaError_t e = cudaEventElapsedTime(&ms, p.first, p.second);
            if (e != cudaSuccess) return e;
            c->total_ms[k] += ms;
            c->timed_launches[k] += 1;
            c->spare.push_back(p);
        }
        c->pending[k].clear();
    }
    return cudaSuccess;
}

int cuda_fail(pt2d_ctx *c, cudaError_t e) {
    if (c) c->last_cuda = static_cast<int>(e);
    return PT2D_ERR_CUDA;
}

#define CK(ctx, expr)                                   \
    do {                                                \
        cudaError_t _e = (expr);                        \
        if (_e != cudaSuccess) return cuda_fail(ctx, _e); \
    } while (0)

}  // namespace

// The code of a sweep tiling reported by pt2d_tiling and pt2d_plan_tiling.
namespace {
void tiling_code(const pt2d::Prep &pp, int32_t out[4]) {
    const pt2d::SweepTiling &t = pp.tiling;
    out[0] = t.bits ? (pp.pen_kernel ? 7 : 3) : t.smem ? (pp.pen_kernel ? 6 : (pp.wide ? 5 : 2)) : (pp.wide ? 4 : 1);
    out[1] = 4 * t.lanes_per_spin;
    out[2] = t.threads;
    out[3] = t.walkers_per_thread;
}
}  // namespace

extern "C" {

void pt2d_default_options(pt2d_options *opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->trace_capacity = 1024;
    opt->device = -1;
}

int32_t pt2d_debug_fail_allocations(int32_t count) {
    return g_fail_allocs.exchange(count > 0 ? count : 0);
}

const char *pt2d_strerror(int status) {
    switch (status) {
        case PT2D_OK: return "ok";
        case PT2D_ERR_INVALID_ARG: return "invalid argument";
        case PT2D_ERR_OOM: return "out of memory";
        case PT2D_ERR_CUDA: return "CUDA error";
        case PT2D_ERR_TIMEOUT: return "device wait timed out";
        case PT2D_ERR_STATE: return "invalid state for this call";
        case PT2D_ERR_UNSUPPORTED: return "unsupported device (needs sm_103)";
        default: return "unknown status";
    }
}

int pt2d_workspace_size(const pt2d_instance *inst, int32_t I, int32_t J, int32_t runs,
                        const pt2d_options *opt, size_t *bytes) {
    if (!bytes) return PT2D_ERR_INVALID_ARG;
    pt2d_ctx tmp;
    int st = prepare(inst, I, nullptr, J, nullptr, runs, opt, tmp.pp, 0, false);
    if (st) return st;
    *bytes = carve(&tmp, nullptr);
    return PT2D_OK;
}

int pt2d_create(pt2d_ctx **out, const pt2d_instance *inst, int32_t I, const float *beta, int32_t J,
                const int32_t *P, int32_t runs, const pt2d_options *opt) {
    pt2d::TraceRange trace("pt2d_create");
    if (!out || !beta || !P) return PT2D_ERR_INVALID_ARG;
    *out = nullptr;
    pt2d_options dflt;
    pt2d_default_options(&dflt);
    if (!opt) opt = &dflt;
    if (opt->device >= 0 && cudaSetDevice(opt->device) != cudaSuccess) return PT2D_ERR_UNSUPPORTED;
    int st = pt2d::check_device();
    if (st) return st;
    pt2d_ctx *c = new (std::nothrow) pt2d_ctx;
    if (!c) return PT2D_ERR_OOM;
    st = prepare(inst, I, beta, J, P, runs, opt, c->pp);
    if (st) {
        delete c;
        return st;
    }
    cudaGetDevice(&c->device);
    c->stream = static_cast<cudaStream_t>(opt->stream);
    c->profile = opt->profile != 0;
    const size_t need = carve(c, nullptr);
    if (opt->workspace) {
        if (opt->workspace_bytes < need || (reinterpret_cast<uintptr_t>(opt->workspace) & 255)) {
            delete c;
            return PT2D_ERR_INVALID_ARG;
        }
        c->ws = opt->workspace;
        c->ws_bytes = opt->workspace_bytes;
    } else {
        if (pt2d::device_alloc(&c->ws, need) != cudaSuccess) {
            cudaGetLastError();
            delete c;
            return PT2D_ERR_OOM;
        }
        c->own_ws = true;
        c->ws_bytes = need;
    }
    carve(c, c->ws);
    Prep &pp = c->pp;
    c->beta.assign(beta, beta + I);
    c->P.assign(P, P + J);
    c->L.Wc = pp.Wc;
    c->L.n = pp.n;
    c->L.C = pp.C;
    c->L.DC = pp.DC;
    c->L.DL = pp.DL;
    c->L.rec_vec = pp.rec_vec;
    c->L.pad_ref = pp.pad_ref;
    c->L.penalty = pp.penalty ? 1 : 0;
    c->L.g0 = pp.g0;
    c->rs.runs = pp.runs;
    c->rs.I = pp.I;
    c->rs.J = pp.J;
    c->rs.R = pp.R;
    c->rs.Rp = pp.Rp;
    c->rs.beta = c->d_beta;
    c->rs.P = c->d_P;
    c->rs.trace_cap = pp.trace_cap;
    c->rs.target = c->d_target;
    c->rs.swap_mode = opt->swap_mode;
    cudaStream_t s = c->stream;
    auto fail = [&](cudaError_t e) {
        c->last_cuda = static_cast<int>(e);
        pt2d_destroy(c);
        return PT2D_ERR_CUDA;
    };
    cudaError_t e = cudaMemsetAsync(c->ws, 0, need - 256, s);
    if (e != cudaSuccess) return fail(e);
    struct Up {
        void *d;
        const void *h;
        size_t b;
    } ups[] = {
        {const_cast<int4 *>(c->L.rec), pp.rec.data(), sizeof(int32_t) * pp.rec.size()},
        {const_cast<int32_t *>(c->L.cofs), pp.cofs.data(), sizeof(int32_t) * (pp.C + 1)},
        {c->d_beta, c->beta.data(), sizeof(float) * I},
        {c->d_P, c->P.data(), sizeof(int32_t) * J},
    };
    for (const auto &u : ups) {
        if (u.b == 0) continue;
        e = cudaMemcpyAsync(u.d, u.h, u.b, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return fail(e);
    }
    std::vector<int64_t> tgt(pp.runs, INT64_MIN);
    e = cudaMemcpyAsync(c->d_target, tgt.data(), sizeof(int64_t) * pp.runs, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return fail(e);
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(e);
    *out = c;
    return PT2D_OK;
}

void pt2d_destroy(pt2d_ctx *c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    if (c->own_ws && c->ws) cudaFree(c->ws);
    for (int k = 0; k < 2; ++k)
        for (auto &p : c->pending[k]) c->spare.push_back(p);
    for (auto &p : c->spare) {
        cudaEventDestroy(p.first);
        cudaEventDestroy(p.second);
    }
    delete c;
}

int pt2d_kernel_time(pt2d_ctx *c, int32_t kind, double *ms, int64_t *launches) {
    if (!c || kind < 0 || kind > 1 || !ms || !launches) return PT2D_ERR_INVALID_ARG;
    if (!c->profile) return PT2D_ERR_STATE;
    CK(c, cudaStreamSynchronize(c->stream));
    CK(c, drain_events(c));
    *ms = c->total_ms[kind];
    *launches = c->timed_launches[kind];
    return PT2D_OK;
}

int pt2d_cuda_error(const pt2d_ctx *c) { return c ? c->last_cuda : 0; }
int pt2d_num_colors(const pt2d_ctx *c) { return c ? c->pp.C : 0; }

int pt2d_tiling(const pt2d_ctx *c, int32_t out[4]) {
    if (!c || !out) return PT2D_ERR_INVALID_ARG;
    tiling_code(c->pp, out);
    return PT2D_OK;
}

int pt2d_plan_tiling(const pt2d_instance *inst, int32_t I, int32_t J, int32_t runs, const pt2d_options *opt,
                     int32_t out[4]) {
    if (!out) return PT2D_ERR_INVALID_ARG;
    pt2d::Prep pp;
    const int st = pt2d::prepare(inst, I, nullptr, J, nullptr, runs, opt, pp, 0, false);
    if (st) return st;
    tiling_code(pp, out);
    return PT2D_OK;
}
int64_t pt2d_launch_count(const pt2d_ctx *c) { return c ? c->launches : 0; }

int pt2d_run(pt2d_ctx *c, int64_t sweeps, int32_t interval, uint64_t seed) {
    pt2d::TraceRange trace("pt2d_run");
    if (!c || sweeps < 0 || interval < 1) return PT2D_ERR_INVALID_ARG;
    const int64_t nev = sweeps / interval;
    if (c->adopt_seed) {
        c->seed = seed;
        c->adopt_seed = false;
    }
    if (c->inited && seed != c->seed) return PT2D_ERR_INVALID_ARG;
    if (c->sweeps_done + nev * interval > (int64_t(1) << 32)) return PT2D_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    cudaStream_t s = c->stream;
    if (!c->inited) {
        c->seed = seed;
        CK(c, pt2d::launch_init(c->L, c->rs, c->wk, seed, s));
        c->launches += 2;
        c->inited = 1;
        c->dir = c->rs.swap_mode ? -1 : 1;
        c->sweeps_done = 0;
        c->events_done = 0;
    }
    for (int64_t e = 0; e < nev; ++e) {
        const int64_t event = c->events_done + 1;
        std::pair<cudaEvent_t, cudaEvent_t> ev[2];
        if (c->profile) {
            ev[0] = take_events(c);
            ev[1] = take_events(c);
            CK(c, cudaEventRecord(ev[0].first, s));
        }
        if (c->pp.pen_kernel) {
            CK(c, pt2d::launch_penalty_sweeps(c->L, c->wk, c->pp.tiling, c->pp.Rp / 4, seed,
                                              static_cast<uint32_t>(c->sweeps_done), interval, s));
        } else if (c->pp.wide) {
            CK(c, pt2d::launch_generic_sweeps(c->L, c->wk, c->pp.tiling, c->pp.Rp / 4, seed,
                                              static_cast<uint32_t>(c->sweeps_done), interval, s));
        } else {
            CK(c, pt2d::launch_sweeps(c->L, c->wk, c->pp.tiling, c->pp.Rp / 4, seed,
                                      static_cast<uint32_t>(c->sweeps_done), interval, s));
        }
        if (c->profile) {
            CK(c, cudaEventRecord(ev[0].second, s));
            CK(c, cudaEventRecord(ev[1].first, s));
        }
        CK(c, pt2d::launch_swap_event(c->L, c->rs, c->wk, seed, event, s));
        if (c->profile) {
            CK(c, cudaEventRecord(ev[1].second, s));
            c->pending[0].push_back(ev[0]);
            c->pending[1].push_back(ev[1]);
        }
        c->launches += 2;
        c->sweeps_done += interval;
        c->events_done = event;
        if (event % 2 == 0 && !c->rs.swap_mode) c->dir = -c->dir;
    }
    return PT2D_OK;
}

int pt2d_sync(pt2d_ctx *c) {
    if (!c) return PT2D_ERR_INVALID_ARG;
    CK(c, cudaStreamSynchronize(c->stream));
    return PT2D_OK;
}

size_t pt2d_array_bytes(const pt2d_ctx *c, int32_t what) {
    if (!c) return 0;
    const Prep &pp = c->pp;
    const size_t RR = static_cast<size_t>(pp.runs) * pp.R;
    switch (what) {
        case PT2D_STATES: return RR * pp.n;
        case PT2D_WALKER_AT: return RR * 4;
        case PT2D_F:
        case PT2D_G:
        case PT2D_ACC_P:
        case PT2D_ACC_B:
        case PT2D_SUM_F:
        case PT2D_SUM_G:
        case PT2D_N_FEASIBLE: return RR * 8;
        case PT2D_COUNTERS: return 4 * 8;
        case PT2D_TRACE_F:
        case PT2D_TRACE_G: return static_cast<size_t>(pp.runs) * pp.trace_cap * 8;
        case PT2D_BEST_F:
        case PT2D_BEST_EVENT:
        case PT2D_SOLVED_EVENT:
        case PT2D_TARGET: return static_cast<size_t>(pp.runs) * 8;
        case PT2D_BEST_STATE: return static_cast<size_t>(pp.runs) * pp.n;
        case PT2D_COLORS: return static_cast<size_t>(pp.n) * 4;
        default: return 0;
    }
}

static void *direct_ptr(pt2d_ctx *c, int32_t what) {
    switch (what) {
        case PT2D_WALKER_AT: return c->rs.walker_at;
        case PT2D_ACC_P: return c->rs.acc_P;
        case PT2D_ACC_B: return c->rs.acc_B;
        case PT2D_SUM_F: return c->rs.sum_f;
        case PT2D_SUM_G: return c->rs.sum_g;
        case PT2D_N_FEASIBLE: return c->rs.n_feasible;
        case PT2D_TRACE_F: return c->rs.trace_f;
        case PT2D_TRACE_G: return c->rs.trace_g;
        case PT2D_BEST_F: return c->rs.best_f;
        case PT2D_BEST_EVENT: return c->rs.best_event;
        case PT2D_SOLVED_EVENT: return c->rs.solved_event;
        case PT2D_TARGET: return c->d_target;
        case PT2D_BEST_STATE: return c->rs.best_state;
        default: return nullptr;
    }
}

int pt2d_read(pt2d_ctx *c, int32_t what, void *dst, size_t bytes) {
    if (!c || !dst) return PT2D_ERR_INVALID_ARG;
    const size_t need = pt2d_array_bytes(c, what);
    if (need == 0 || bytes != need) return PT2D_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    cudaStream_t s = c->stream;
    const Prep &pp = c->pp;
    if (what == PT2D_COUNTERS) {
        CK(c, cudaStreamSynchronize(s));
        int64_t v[4] = {c->sweeps_done, c->events_done, c->dir, c->inited};
        std::memcpy(dst, v, sizeof v);
        return PT2D_OK;
    }
    if (what == PT2D_COLORS) {
        std::memcpy(dst, pp.color.data(), need);
        return PT2D_OK;
    }
    if (void *src = direct_ptr(c, what)) {
        CK(c, cudaMemcpyAsync(dst, src, need, cudaMemcpyDeviceToHost, s));
        CK(c, cudaStreamSynchronize(s));
        return PT2D_OK;
    }
    if (what == PT2D_STATES) {
        if (!c->inited) return PT2D_ERR_STATE;
        std::vector<int8_t> tmp(static_cast<size_t>(pp.n) * pp.Wc);
        CK(c, cudaMemcpyAsync(tmp.data(), c->L.S, tmp.size(), cudaMemcpyDeviceToHost, s));
        CK(c, cudaStreamSynchronize(s));
        int8_t *o = static_cast<int8_t *>(dst);
        for (int32_t r = 0; r < pp.runs; ++r)
            for (int32_t w = 0; w < pp.R; ++w) {
                int8_t *row = o + (static_cast<size_t>(r) * pp.R + w) * pp.n;
                const size_t colw = static_cast<size_t>(r) * pp.Rp + w;
                for (int32_t a = 0; a < pp.n; ++a)
                    row[a] = tmp[static_cast<size_t>(pp.pos_of[a]) * pp.Wc + colw];
            }
        return PT2D_OK;
    }
    if (what == PT2D_F || what == PT2D_G) {
        const size_t esz = what == PT2D_F ? 8 : 4;
        std::vector<char> tmp(esz * pp.Wc);
        const void *src = what == PT2D_F ? static_cast<void *>(c->wk.f) : static_cast<void *>(c->wk.g);
        CK(c, cudaMemcpyAsync(tmp.data(), src, tmp.size(), cudaMemcpyDeviceToHost, s));
        CK(c, cudaStreamSynchronize(s));
        int64_t *o = static_cast<int64_t *>(dst);
        for (int32_t r = 0; r < pp.runs; ++r)
            for (int32_t w = 0; w < pp.R; ++w) {
                const size_t colw = static_cast<size_t>(r) * pp.Rp + w;
                if (esz == 8)
                    o[static_cast<size_t>(r) * pp.R + w] = reinterpret_cast<int64_t *>(tmp.data())[colw];
                else
                    o[static_cast<size_t>(r) * pp.R + w] = reinterpret_cast<int32_t *>(tmp.data())[colw];
            }
        return PT2D_OK;
    }
    return PT2D_ERR_INVALID_ARG;
}

int pt2d_read_walker(pt2d_ctx *c, int32_t run, int32_t walker, int8_t *dst) {
    if (!c || !dst) return PT2D_ERR_INVALID_ARG;
    const Prep &pp = c->pp;
    if (run < 0 || run >= pp.runs || walker < 0 || walker >= pp.R) return PT2D_ERR_INVALID_ARG;
    if (!c->inited) return PT2D_ERR_STATE;
    cudaSetDevice(c->device);
    std::vector<int8_t> tmp(pp.n);
    const int8_t *col = c->L.S + static_cast<int64_t>(run) * pp.Rp + walker;
    CK(c, cudaMemcpy2DAsync(tmp.data(), 1, col, static_cast<size_t>(pp.Wc), 1, pp.n,
                            cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    for (int32_t a = 0; a < pp.n; ++a) dst[a] = tmp[pp.pos_of[a]];
    return PT2D_OK;
}

int pt2d_write(pt2d_ctx *c, int32_t what, const void *src, size_t bytes) {
    if (!c || !src) return PT2D_ERR_INVALID_ARG;
    const size_t need = pt2d_array_bytes(c, what);
    if (need == 0 || bytes != need || what == PT2D_COLORS || what == PT2D_F || what == PT2D_G)
        return PT2D_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    cudaStream_t s = c->stream;
    const Prep &pp = c->pp;
    if (what == PT2D_COUNTERS) {
        const int64_t *v = static_cast<const int64_t *>(src);
        if (v[0] < 0 || v[1] < 0 || (v[2] != 1 && v[2] != -1) || v[0] > (int64_t(1) << 32))
            return PT2D_ERR_INVALID_ARG;
        CK(c, cudaStreamSynchronize(s));
        c->sweeps_done = v[0];
        c->events_done = v[1];
        c->dir = v[2];
        if (v[3] && !c->inited) {
            c->inited = 1;
            c->adopt_seed = true;
        }
        return PT2D_OK;
    }
    if (what == PT2D_WALKER_AT) {
        const int32_t *at = static_cast<const int32_t *>(src);
        std::vector<float> wb(pp.Wc, 0.0f);
        std::vector<int32_t> wp(pp.Wc, 0);
        for (int32_t r = 0; r < pp.runs; ++r) {
            std::vector<char> seen(pp.R, 0);
            for (int32_t sl = 0; sl < pp.R; ++sl) {
                const int32_t w = at[static_cast<size_t>(r) * pp.R + sl];
                if (w < 0 || w >= pp.R || seen[w]) return PT2D_ERR_INVALID_ARG;
                seen[w] = 1;
                const size_t colw = static_cast<size_t>(r) * pp.Rp + w;
                wb[colw] = c->beta[sl / pp.J];
                wp[colw] = c->P[sl % pp.J];
            }
        }
        CK(c, cudaMemcpyAsync(c->rs.walker_at, at, need, cudaMemcpyHostToDevice, s));
        CK(c, cudaMemcpyAsync(c->wk.wbeta, wb.data(), sizeof(float) * pp.Wc, cudaMemcpyHostToDevice, s));
        CK(c, cudaMemcpyAsync(c->wk.wP, wp.data(), sizeof(int32_t) * pp.Wc, cudaMemcpyHostToDevice, s));
        CK(c, cudaStreamSynchronize(s));
        return PT2D_OK;
    }
    if (void *dstp = direct_ptr(c, what)) {
        CK(c, cudaMemcpyAsync(dstp, src, need, cudaMemcpyHostToDevice, s));
        CK(c, cudaStreamSynchronize(s));
        return PT2D_OK;
    }
    if (what == PT2D_STATES) {
        const int8_t *in = static_cast<const int8_t *>(src);
        std::vector<int8_t> tmp(static_cast<size_t>(pp.n) * pp.Wc, 1);
        for (int32_t r = 0; r < pp.runs; ++r)
            for (int32_t w = 0; w < pp.R; ++w) {
                const int8_t *row = in + (static_cast<size_t>(r) * pp.R + w) * pp.n;
                const size_t colw = static_cast<size_t>(r) * pp.Rp + w;
                for (int32_t a = 0; a < pp.n; ++a) {
                    if (row[a] != 1 && row[a] != -1) return PT2D_ERR_INVALID_ARG;
                    tmp[static_cast<size_t>(pp.pos_of[a]) * pp.Wc + colw] = row[a];
                }
            }
        CK(c, cudaMemcpyAsync(c->L.S, tmp.data(), tmp.size(), cudaMemcpyHostToDevice, s));
        CK(c, cudaStreamSynchronize(s));
        return PT2D_OK;
    }
    return PT2D_ERR_INVALID_ARG;
}

// ---- host-side compiler helpers ------------------------------------------------
int pt2d_greedy_color(const pt2d_instance *inst, int32_t *color, int32_t *n_colors) {
    if (!inst || !color || !n_colors) return PT2D_ERR_INVALID_ARG;
    Prep pp;
    pt2d_instance tmp = *inst;
    tmp.color = nullptr;
    pt2d_options o;
    pt2d_default_options(&o);
    o.walkers_per_cta = 4;
    o.threads_per_cta = 32;
    int st = prepare(&tmp, 1, nullptr, 1, nullptr, 1, &o, pp, 0, false);
    if (st) return st;
    std::memcpy(color, pp.color.data(), sizeof(int32_t) * pp.n);
    *n_colors = pp.C;
    return PT2D_OK;
}

namespace {

// Penalty terms of g = sum_c (sum_{a in c} A_a x_a - b_c)^2, x_a = [s_a = +1],
// in the links form.  With y_a = [s_a = -1] = 1 - x_a and S = sum_a A_a, each
// constraint equals (sum_a A_a y_a - (S - b))^2; y^2 = y and
// 2 y_a y_b = y_a + y_b - [s_a != s_b] turn it into
//   (S - b)^2 + sum_a A_a (2b - S) y_a - sum_{a<b} A_a A_b [s_a != s_b],
// so g0 += (S - b)^2, k_a += A_a (2b - S), K_ab -= A_a A_b.  coef / rhs NULL
// mean all ones (one-hot groups).
int equality_penalty(int32_t n, int32_t n_cons, const int32_t *con_ptr, const int32_t *con_col,
                     const int32_t *coef, const int64_t *rhs, int32_t *lk_ptr, int32_t *lk_col,
                     int16_t *lk_w, int32_t cap, int32_t *nnz, int32_t *hk, int64_t *g0) {
    using i128 = __int128;
    if (n < 1 || n_cons < 0 || !con_ptr || !lk_ptr || !nnz || !hk || !g0) return PT2D_ERR_INVALID_ARG;
    if (con_ptr[0] != 0) return PT2D_ERR_INVALID_ARG;
    for (int32_t c = 0; c < n_cons; ++c)
        if (con_ptr[c + 1] < con_ptr[c]) return PT2D_ERR_INVALID_ARG;
    if (con_ptr[n_cons] > 0 && !con_col) return PT2D_ERR_INVALID_ARG;
    const i128 kLim = static_cast<i128>(1) << 62;
    std::vector<std::map<int32_t, i128>> K(n);
    std::vector<i128> k(n, 0);
    i128 c0 = 0;
    for (int32_t c = 0; c < n_cons; ++c) {
        const int32_t beg = con_ptr[c], m = con_ptr[c + 1] - beg;
        std::vector<std::pair<int32_t, int64_t>> mem(m);
        for (int32_t i = 0; i < m; ++i) mem[i] = {con_col[beg + i], coef ? coef[beg + i] : 1};
        std::sort(mem.begin(), mem.end());
        const i128 b = rhs ? rhs[c] : 1;
        i128 S = 0;
        for (int32_t i = 0; i < m; ++i) {
            if (mem[i].first < 0 || mem[i].first >= n || (i > 0 && mem[i].first == mem[i - 1].first))
                return PT2D_ERR_INVALID_ARG;
            S += mem[i].second;
        }
        if (b > kLim || b < -kLim) return PT2D_ERR_INVALID_ARG;
        for (int32_t i = 0; i < m; ++i) {
            const i128 A = mem[i].second;
            k[mem[i].first] += A * (2 * b - S);
            for (int32_t j = 0; j < m; ++j)
                if (j != i) K[mem[i].first][mem[j].first] -= A * mem[j].second;
            if (k[mem[i].first] > kLim || k[mem[i].first] < -kLim) return PT2D_ERR_INVALID_ARG;
        }
        c0 += (S - b) * (S - b);
        if (c0 > kLim) return PT2D_ERR_INVALID_ARG;
    }
    int64_t total = 0;
    for (int32_t a = 0; a < n; ++a)
        for (const auto &e : K[a])
            if (e.second != 0) ++total;
    if (total > INT32_MAX) return PT2D_ERR_INVALID_ARG;
    *nnz = static_cast<int32_t>(total);
    if (total > cap || (total > 0 && (!lk_col || !lk_w))) return PT2D_ERR_INVALID_ARG;
    int32_t pos = 0;
    lk_ptr[0] = 0;
    for (int32_t a = 0; a < n; ++a) {
        for (const auto &e : K[a]) {
            if (e.second == 0) continue;
            if (e.second < INT16_MIN || e.second > INT16_MAX) return PT2D_ERR_INVALID_ARG;
            lk_col[pos] = e.first;
            lk_w[pos] = static_cast<int16_t>(e.second);
            ++pos;
        }
        lk_ptr[a + 1] = pos;
        if (k[a] < INT32_MIN || k[a] > INT32_MAX) return PT2D_ERR_INVALID_ARG;
        hk[a] = static_cast<int32_t>(k[a]);
    }
    *g0 = static_cast<int64_t>(c0);
    return PT2D_OK;
}

}  // namespace

int pt2d_equality_penalty(int32_t n, int32_t n_cons, const int32_t *con_ptr, const int32_t *con_col,
                          const int32_t *coef, const int64_t *rhs, int32_t *lk_ptr, int32_t *lk_col,
                          int16_t *lk_w, int32_t cap, int32_t *nnz, int32_t *hk, int64_t *g0) {
    if (n_cons > 0 && con_ptr && con_ptr[n_cons] > 0 && !coef) return PT2D_ERR_INVALID_ARG;
    if (n_cons > 0 && !rhs) return PT2D_ERR_INVALID_ARG;
    return equality_penalty(n, n_cons, con_ptr, con_col, coef, rhs, lk_ptr, lk_col, lk_w, cap, nnz, hk, g0);
}

int pt2d_onehot_penalty(int32_t n, int32_t n_groups, const int32_t *grp_ptr, const int32_t *grp_col,
                        int32_t *lk_ptr, int32_t *lk_col, int16_t *lk_w, int32_t cap, int32_t *nnz,
                        int32_t *hk, int64_t *g0) {
    // (sum_{a in c} x_a - 1)^2: all coefficients 1, right-hand side 1
    return equality_penalty(n, n_groups, grp_ptr, grp_col, nullptr, nullptr, lk_ptr, lk_col, lk_w, cap, nnz,
                            hk, g0);
}

int pt2d_sparsify(int32_t N, const int16_t *Jq, int32_t rule, int32_t param, int32_t *n_out,
                  int64_t *nnz_cp, int64_t *nnz_lk, int32_t *cp_ptr, int32_t *cp_col, int16_t *cp_J,
                  int32_t *lk_ptr, int32_t *lk_col, int32_t *copy_of) {
    if (N < 1 || !Jq || !n_out || !nnz_cp || !nnz_lk) return PT2D_ERR_INVALID_ARG;
    for (int32_t i = 0; i < N; ++i) {
        if (Jq[static_cast<size_t>(i) * N + i] != 0) return PT2D_ERR_INVALID_ARG;
        for (int32_t j = 0; j < i; ++j)
            if (Jq[static_cast<size_t>(i) * N + j] != Jq[static_cast<size_t>(j) * N + i])
                return PT2D_ERR_INVALID_ARG;
    }
    // copies per logical node and the edge capacity of each copy (-1 = unbounded)
    std::vector<int32_t> K(N), off(N + 1, 0);
    std::vector<std::vector<int32_t>> nbrs(N);
    for (int32_t i = 0; i < N; ++i)
        for (int32_t j = 0; j < N; ++j)
            if (j != i && Jq[static_cast<size_t>(i) * N + j] != 0) nbrs[i].push_back(j);
    std::vector<std::vector<int32_t>> cap(N);
    for (int32_t i = 0; i < N; ++i) {
        const int32_t d = static_cast<int32_t>(nbrs[i].size());
        if (rule == PT2D_SPARSIFY_FIXED) {
            if (param < 1) return PT2D_ERR_INVALID_ARG;
            K[i] = param;
            cap[i].assign(K[i], -1);
        } else if (rule == PT2D_SPARSIFY_MAX_EDGES) {
            if (param < 1) return PT2D_ERR_INVALID_ARG;
            K[i] = std::max<int32_t>(1, (d + param - 1) / param);
            cap[i].assign(K[i], param);
        } else if (rule == PT2D_SPARSIFY_MAX_DEGREE) {
            if (param < 3) return PT2D_ERR_INVALID_ARG;
            if (d <= param) {
                K[i] = 1;
                cap[i].assign(1, param);
            } else {
                int32_t k = 2;
                while (2 * (param - 1) + (k - 2) * (param - 2) < d) ++k;
                K[i] = k;
                cap[i].assign(k, param - 2);
                cap[i][0] = param - 1;
                cap[i][k - 1] = param - 1;
            }
        } else {
            return PT2D_ERR_INVALID_ARG;
        }
        off[i + 1] = off[i] + K[i];
    }
    const int32_t n = off[N];
    // deal neighbours round-robin over copies, skipping full ones
    std::vector<std::vector<int32_t>> copy_for(N);
    for (int32_t i = 0; i < N; ++i) {
        copy_for[i].assign(N, -1);
        std::vector<int32_t> load(K[i], 0);
        int32_t c = 0;
        for (int32_t j : nbrs[i]) {
            int32_t tries = 0;
            while (cap[i][c] >= 0 && load[c] >= cap[i][c]) {
                c = (c + 1) % K[i];
                if (++tries > K[i]) return PT2D_ERR_INVALID_ARG;
            }
            copy_for[i][j] = c;
            load[c]++;
            c = (c + 1) % K[i];
        }
    }
    std::vector<std::vector<std::pair<int32_t, int16_t>>> adj(n);
    for (int32_t i = 0; i < N; ++i)
        for (int32_t j : nbrs[i]) {
            if (j <= i) continue;
            const int32_t a = off[i] + copy_for[i][j], b = off[j] + copy_for[j][i];
            const int16_t v = Jq[static_cast<size_t>(i) * N + j];
            adj[a].push_back({b, v});
            adj[b].push_back({a, v});
        }
    int64_t ncp = 0;
    for (auto &v : adj) {
        std::sort(v.begin(), v.end());
        ncp += static_cast<int64_t>(v.size());
    }
    const int64_t nlk = 2LL * (n - N);
    *n_out = n;
    *nnz_cp = ncp;
    *nnz_lk = nlk;
    if (!cp_ptr && !cp_col && !cp_J && !lk_ptr && !lk_col && !copy_of) return PT2D_OK;
    if (!cp_ptr || !cp_col || !cp_J || !lk_ptr || !lk_col || !copy_of) return PT2D_ERR_INVALID_ARG;
    cp_ptr[0] = 0;
    int64_t k = 0;
    for (int32_t a = 0; a < n; ++a) {
        for (const auto &e : adj[a]) {
            cp_col[k] = e.first;
            cp_J[k] = e.second;
            ++k;
        }
        cp_ptr[a + 1] = static_cast<int32_t>(k);
    }
    lk_ptr[0] = 0;
    k = 0;
    for (int32_t i = 0; i < N; ++i)
        for (int32_t c = 0; c < K[i]; ++c) {
            const int32_t a = off[i] + c;
            if (c > 0) lk_col[k++] = a - 1;
            if (c + 1 < K[i]) lk_col[k++] = a + 1;
            lk_ptr[a + 1] = static_cast<int32_t>(k);
            copy_of[a] = i;
        }
    return PT2D_OK;
}

// ---- diagnostics ------------------------------------------------------------------
int pt2d_diag_philox(const uint32_t *ctr, const uint32_t *key, uint32_t *out, int64_t count) {
    if (count < 0 || (count > 0 && (!ctr || !key || !out))) return PT2D_ERR_INVALID_ARG;
    if (int st = pt2d::check_device()) return st;
    return pt2d::diag_philox(ctr, key, out, count) == cudaSuccess ? PT2D_OK : PT2D_ERR_CUDA;
}

int pt2d_diag_pt_exp(const float *x, float *y, int64_t count) {
    if (count < 0 || (count > 0 && (!x || !y))) return PT2D_ERR_INVALID_ARG;
    if (int st = pt2d::check_device()) return st;
    return pt2d::diag_pt_exp(x, y, count) == cudaSuccess ? PT2D_OK : PT2D_ERR_CUDA;
}

int pt2d_diag_heatbath(const float *beta, const int32_t *H, const uint32_t *r, int8_t *spin,
                       int64_t count) {
    if (count < 0 || (count > 0 && (!beta || !H || !r || !spin))) return PT2D_ERR_INVALID_ARG;
    if (int st = pt2d::check_device()) return st;
    return pt2d::diag_heatbath(beta, H, r, spin, count) == cudaSuccess ? PT2D_OK : PT2D_ERR_CUDA;
}

int pt2d_diag_swap_accept(const float *x, const uint32_t *r, int8_t *accept, int64_t count) {
    if (count < 0 || (count > 0 && (!x || !r || !accept))) return PT2D_ERR_INVALID_ARG;
    if (int st = pt2d::check_device()) return st;
    return pt2d::diag_swap_accept(x, r, accept, count) == cudaSuccess ? PT2D_OK : PT2D_ERR_CUDA;
}

}  // extern "C"
