// Host side of the batched persistent 2D-PT API (include/pt2d.h, pt2d_batch_*):
// a device memory pool with a first-fit allocator, instances added and removed
// at any time, run descriptors ordered by decreasing work, launches replayed
// from a CUDA graph, per-instance reads, and an autotuner for the launch shape.
#include <algorithm>
#include <chrono>
#include <cstdint>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/pt2d.h"
#include "pt2d_batch.h"
#include "pt2d_prep.h"
#include "pt2d_trace.h"
#include "pt2d_wide.cuh"

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

// First-fit allocator over [base, base + size) with coalescing on free.
class Arena {
   public:
    void reset(size_t base, size_t size) {
        free_.clear();
        if (size) free_[base] = size;
    }
    bool alloc(size_t bytes, size_t *off) {
        bytes = align_up(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t next = it->first + bytes;
                free_.erase(it);
                if (rest) free_[next] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = align_up(bytes);
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t largest() const {
        size_t m = 0;
        for (const auto &kv : free_) m = std::max(m, kv.second);
        return m;
    }
    size_t total() const {
        size_t t = 0;
        for (const auto &kv : free_) t += kv.second;
        return t;
    }

   private:
    std::map<size_t, size_t> free_;
};

struct Inst {
    size_t off = 0, bytes = 0;
    int32_t n = 0, I = 0, J = 0, R = 0, Rp = 0, runs = 0, C = 0, rec_vec = 0;
    std::vector<int32_t> pos_of, color;
    std::vector<pt2d::BatchRun> desc;  // one per run
};

struct Layout1 {  // byte offsets within an instance block
    size_t rec, cofs, beta, P, total;
    size_t run0, run_stride;
    size_t state, walker_at, wparam, fg, stats, trace, best_state, scalars, counter;  // per run
};

Layout1 block_layout(int32_t n, int32_t C, int32_t rec_vec, int32_t I, int32_t J, int32_t R,
                     int32_t Rp, int32_t runs, int32_t trace_cap) {
    Layout1 l{};
    size_t o = 0;
    l.rec = o;
    o = align_up(o + static_cast<size_t>(n) * rec_vec * 16);
    l.cofs = o;
    o = align_up(o + static_cast<size_t>(C + 1) * 4);
    l.beta = o;
    o = align_up(o + static_cast<size_t>(I) * 4);
    l.P = o;
    o = align_up(o + static_cast<size_t>(J) * 4);
    l.run0 = o;
    size_t r = 0;
    l.state = r;
    r = align_up(r + static_cast<size_t>(n + 1) * Rp);
    l.walker_at = r;
    r = align_up(r + static_cast<size_t>(R) * 4);
    l.wparam = r;
    r = align_up(r + static_cast<size_t>(Rp) * 8);
    l.fg = r;
    r = align_up(r + static_cast<size_t>(Rp) * 12);
    l.stats = r;
    r = align_up(r + static_cast<size_t>(R) * 5 * 8);
    l.trace = r;
    r = align_up(r + static_cast<size_t>(trace_cap) * 16);
    l.best_state = r;
    r = align_up(r + static_cast<size_t>(n));
    l.scalars = r;
    r = align_up(r + pt2d::kScCount * 8);
    l.counter = r;
    r = align_up(r + 4);
    l.run_stride = r;
    l.total = o + r * static_cast<size_t>(runs);
    return l;
}

// Replicas per run padded to a power of two >= 16, so a run's spin rows are
// whole 16-byte vectors for the shared-memory copies.
int32_t pow2_at_least(int32_t x) {
    int32_t p = 16;
    while (p < x) p <<= 1;
    return p;
}

}  // namespace

struct pt2d_batch {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    bool own_pool = false;
    uint8_t *pool = nullptr;
    size_t pool_bytes = 0;
    int DC = 3;
    int32_t trace_cap = 0;
    int32_t max_runs = 0;
    int threads = 1024;
    int grid = 0;
    int smem_state = 0;
    int smem_state_max = 0;
    bool use_graph = true;
    Arena arena;
    std::map<int64_t, Inst> insts;
    int64_t next_id = 1;
    pt2d::BatchRun *d_runs = nullptr;
    pt2d::BatchItem *d_items = nullptr;               // [max_runs * kMaxSlabs]
    int32_t *d_queue = nullptr;
    int64_t *d_status = nullptr;                      // [max_runs][2]
    std::vector<std::pair<int64_t, int32_t>> order;  // run array order: (id, run)
    int32_t n_items = 0;                              // slabs for k_batch (d_items[0 .. n_items))
    int32_t n_items_bits8 = 0;                        // bit-packed slabs for k_batch_bits8, after them
    int state_int8 = 0, state_bits8 = 0;              // slab shared memory the two lists need
    int glob_sw = 32;                                 // slab width when spins stay in global memory
    int swap_mode = 0;                                // PT2D_SWAP_2D or PT2D_SWAP_JCOLUMN, all problems
    bool generic = false;                             // runtime-degree kernel
    int storage = 0;                                  // pt2d_batch_shape::storage
    int balance = 2;                                  // pt2d_batch_shape::balance
    bool int8 = true;                                 // int8 shared-memory slabs allowed
    bool bits = true;                                 // bit-packed shared-memory slabs allowed
    int32_t n_runs = 0;
    bool dirty = true;
    cudaGraphExec_t graph = nullptr;
    int graph_events = -1, graph_interval = -1, graph_threads = -1;
    static constexpr int kMaxSlabs = pt2d::kBatchMaxReplicas / 8;
    int64_t launches = 0;
    int last_cuda = 0;
};

namespace {

int fail(pt2d_batch *b, cudaError_t e) {
    if (b) b->last_cuda = static_cast<int>(e);
    cudaGetLastError();
    return PT2D_ERR_CUDA;
}

#define BK(b, expr)                                \
    do {                                           \
        cudaError_t _e = (expr);                   \
        if (_e != cudaSuccess) return fail(b, _e); \
    } while (0)

// A runtime-degree batch takes problems whose coupling degree is within the
// declared cap (its wide records pad the degree up to a multiple of 4).
bool degrees_fit(const pt2d_batch *b, const pt2d::Prep &pp) {
    return pp.dcmax <= std::max(b->DC, 6);
}

void drop_graph(pt2d_batch *b) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->graph_events = b->graph_interval = b->graph_threads = -1;
}

// Slab width and storage of a run: int8 spins in shared memory, the whole run
// when it fits in the shared memory reserved per CTA, else the widest power of
// two >= 8 that fits; else the same with bit-packed spins (widths >= 8); else
// int8 spins in global memory at the global-memory slab width.  Then the width
// is halved while a slab holds more than `cap` spin-walkers (0 = no cap).
void slab_shape(const pt2d_batch *b, pt2d::BatchRun &d, int64_t cap) {
    auto capped = [&](int32_t sw, int32_t narrowest) {
        while (cap > 0 && sw > narrowest && static_cast<int64_t>(d.n) * sw > cap) sw >>= 1;
        return sw;
    };
    for (int32_t sw = d.Rp; b->int8 && sw >= 8; sw >>= 1)
        if (static_cast<int64_t>(d.n + 1) * sw <= b->smem_state) {
            d.sw = capped(sw, 8);
            d.mode = 1;
            return;
        }
    if (b->smem_state > 0 && b->bits)
        for (int32_t sw = d.Rp; sw >= 8; sw >>= 1)
            if (pt2d::batch_bits_bytes(d.n, sw) <= b->smem_state) {
                d.sw = capped(sw, 8);
                d.mode = 2;
                return;
            }
    d.sw = capped(std::min<int32_t>(d.Rp, b->glob_sw), 16);
    d.mode = 0;
}

bool shape_valid(const pt2d_batch_shape &sh) {
    return sh.threads_per_cta >= 128 && sh.threads_per_cta <= 1024 && sh.threads_per_cta % 32 == 0 &&
           sh.storage >= 0 && sh.storage <= 3 && sh.global_width >= 16 &&
           sh.global_width <= pt2d::kBatchMaxReplicas && (sh.global_width & (sh.global_width - 1)) == 0 &&
           sh.balance >= 0 && sh.balance <= 1024;
}

// Install a launch shape; the run descriptors are rebuilt at the next launch
// when the slab layout changes.
bool apply_shape(pt2d_batch *b, const pt2d_batch_shape &sh) {
    if (!shape_valid(sh)) return false;
    b->threads = sh.threads_per_cta;
    const int smem_state = sh.storage == 1 ? 0 : b->smem_state_max;
    if (sh.storage != b->storage || smem_state != b->smem_state || sh.global_width != b->glob_sw ||
        sh.balance != b->balance)
        b->dirty = true;
    b->storage = sh.storage;
    b->smem_state = smem_state;
    b->int8 = sh.storage != 3;
    b->bits = sh.storage != 2;
    b->glob_sw = sh.global_width;
    b->balance = sh.balance;
    return true;
}

pt2d_batch_shape current_shape(const pt2d_batch *b) {
    return pt2d_batch_shape{b->threads, b->storage, b->glob_sw, b->balance};
}

int upload_descriptors(pt2d_batch *b) {
    std::vector<std::pair<pt2d::BatchRun, std::pair<int64_t, int32_t>>> tagged;
    int64_t total = 0;
    for (auto &kv : b->insts)
        for (auto &d : kv.second.desc) total += d.work;
    const int64_t cap = b->balance > 0 ? total / (static_cast<int64_t>(b->grid) * b->balance) : 0;
    for (auto &kv : b->insts)
        for (auto &d : kv.second.desc) {
            slab_shape(b, d, cap);
            d.nslab = d.Rp / d.sw;
            tagged.push_back({d, {kv.first, d.run}});
        }
    std::stable_sort(tagged.begin(), tagged.end(),
                     [](const auto &x, const auto &y) { return x.first.work > y.first.work; });
    if (static_cast<int32_t>(tagged.size()) > b->max_runs) return PT2D_ERR_OOM;
    std::vector<pt2d::BatchRun> all;
    std::vector<pt2d::BatchItem> items;
    std::vector<int64_t> item_work;
    b->order.clear();
    for (const auto &t : tagged) {
        const int32_t idx = static_cast<int32_t>(all.size());
        all.push_back(t.first);
        b->order.push_back(t.second);
        for (int32_t k = 0; k < t.first.nslab; ++k) {
            items.push_back({idx, k});
            item_work.push_back(static_cast<int64_t>(t.first.n) * t.first.sw);
        }
    }
    // largest slabs first, so the event ends on small ones; with specialised
    // records the bit-packed slabs form a second list (k_batch_bits8), after the
    // int8 ones (k_batch)
    std::vector<size_t> perm(items.size());
    for (size_t k = 0; k < perm.size(); ++k) perm[k] = k;
    auto bits8 = [&](size_t k) { return !b->generic && all[items[k].run].mode == 2; };
    std::stable_sort(perm.begin(), perm.end(), [&](size_t x, size_t y) {
        if (bits8(x) != bits8(y)) return !bits8(x);
        return item_work[x] > item_work[y];
    });
    std::vector<pt2d::BatchItem> sorted(items.size());
    int32_t n_bits8 = 0;
    for (size_t k = 0; k < perm.size(); ++k) {
        sorted[k] = items[perm[k]];
        n_bits8 += bits8(perm[k]) ? 1 : 0;
    }
    items.swap(sorted);
    // shared memory of the largest slab of each list: a batch of small problems
    // launches with less than the maximum, so several CTAs share an SM
    int64_t need_int8 = 0, need_bits8 = 0;
    for (size_t k = 0; k < items.size(); ++k) {
        const pt2d::BatchRun &r = all[items[k].run];
        if (k >= items.size() - n_bits8)
            need_bits8 = std::max(need_bits8, pt2d::batch_bits_bytes(r.n, r.sw));
        else if (r.mode == 1)
            need_int8 = std::max(need_int8, static_cast<int64_t>(r.n + 1) * r.sw);
        else if (r.mode == 2)
            need_int8 = std::max(need_int8, pt2d::batch_bits_bytes(r.n, r.sw));
    }
    b->state_int8 = static_cast<int>((need_int8 + 15) & ~int64_t{15});
    b->state_bits8 = static_cast<int>((need_bits8 + 15) & ~int64_t{15});
    if (!all.empty()) {
        BK(b, cudaMemcpyAsync(b->d_runs, all.data(), sizeof(pt2d::BatchRun) * all.size(),
                              cudaMemcpyHostToDevice, b->stream));
        BK(b, cudaMemcpyAsync(b->d_items, items.data(), sizeof(pt2d::BatchItem) * items.size(),
                              cudaMemcpyHostToDevice, b->stream));
    }
    b->n_runs = static_cast<int32_t>(all.size());
    b->n_items = static_cast<int32_t>(items.size()) - n_bits8;
    b->n_items_bits8 = n_bits8;
    b->dirty = false;
    drop_graph(b);
    return PT2D_OK;
}

int launch(pt2d_batch *b, int32_t events, int32_t interval) {
    if (b->dirty) {
        int st = upload_descriptors(b);
        if (st) return st;
    }
    if (b->n_runs == 0 || events == 0) return PT2D_OK;
    // k_batch takes the int8 slabs (all slabs of a runtime-degree batch),
    // k_batch_bits8 the bit-packed slabs of specialised records; each has its
    // own work counter
    pt2d::BatchArgs a{b->pool, b->d_runs, b->d_items, b->n_runs, b->n_items, b->d_queue, interval,
                      b->state_int8, b->d_status};
    pt2d::BatchArgs a8{b->pool, b->d_runs, b->d_items + b->n_items, b->n_runs, b->n_items_bits8,
                       b->d_queue + 1, interval, b->state_bits8, b->d_status};
    const int threads8 = std::min(b->threads, pt2d::kBatchBits8Threads);
    const int threads = std::min(b->threads, b->generic ? pt2d::kBatchGenericThreads : pt2d::kBatchInt8Threads);
    const int kdc = b->generic ? 0 : b->DC;
    // persistent CTAs: as many as fit on the SMs at once, no more than the slabs
    const int per_sm = b->n_items > 0 ? pt2d::batch_blocks_per_sm(kdc, 2, false, threads, b->state_int8) : 1;
    const int per_sm8 =
        b->n_items_bits8 > 0 ? pt2d::batch_blocks_per_sm(kdc, 2, true, threads8, b->state_bits8) : 1;
    const int grid = static_cast<int>(std::min<int64_t>(static_cast<int64_t>(b->grid) * per_sm, b->n_items));
    const int grid8 =
        static_cast<int>(std::min<int64_t>(static_cast<int64_t>(b->grid) * per_sm8, b->n_items_bits8));
    if (grid > 0) BK(b, pt2d::batch_kernel_attributes(kdc, 2, b->state_int8));
    // per event: the counters are cleared, then every slab of every run
    auto enqueue = [&]() -> cudaError_t {
        for (int32_t e = 0; e < events; ++e) {
            cudaError_t x = cudaMemsetAsync(b->d_queue, 0, 2 * sizeof(int32_t), b->stream);
            if (x != cudaSuccess) return x;
            if (grid8 > 0) {
                x = pt2d::launch_batch_bits8(a8, kdc, 2, grid8, threads8, b->stream);
                if (x != cudaSuccess) return x;
            }
            if (grid > 0) {
                x = pt2d::launch_batch(a, kdc, 2, grid, threads, b->stream);
                if (x != cudaSuccess) return x;
            }
        }
        return cudaSuccess;
    };
    if (!b->use_graph) {
        BK(b, enqueue());
    } else {
        if (!b->graph || b->graph_events != events || b->graph_interval != interval ||
            b->graph_threads != b->threads) {
            drop_graph(b);
            cudaGraph_t g = nullptr;
            BK(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
            cudaError_t e1 = enqueue();
            cudaError_t e3 = cudaStreamEndCapture(b->stream, &g);
            if (e1 != cudaSuccess) return fail(b, e1);
            if (e3 != cudaSuccess) return fail(b, e3);
            cudaError_t e4 = cudaGraphInstantiate(&b->graph, g, 0);
            cudaGraphDestroy(g);
            if (e4 != cudaSuccess) return fail(b, e4);
            b->graph_events = events;
            b->graph_interval = interval;
            b->graph_threads = b->threads;
        }
        BK(b, cudaGraphLaunch(b->graph, b->stream));
    }
    b->launches += static_cast<int64_t>(events) * ((grid > 0 ? 1 : 0) + (grid8 > 0 ? 1 : 0));
    return PT2D_OK;
}

}  // namespace

namespace pt2d {

int batch_instance_bytes_bounds(const pt2d_batch *b, const pt2d_instance *inst, int32_t I, int32_t J,
                                int32_t runs, size_t *lo, size_t *hi) {
    if (!b || !inst || !lo || !hi || inst->n < 1 || I < 1 || J < 1 || runs < 1 ||
        static_cast<int64_t>(I) * J > pt2d::kBatchMaxReplicas || !inst->cp_ptr || !inst->lk_ptr)
        return PT2D_ERR_INVALID_ARG;
    const int32_t n = inst->n;
    if (inst->cp_ptr[0] != 0 || inst->lk_ptr[0] != 0) return PT2D_ERR_INVALID_ARG;
    int32_t dcmax = 0, dlmax = 0, degmax = 0;
    for (int32_t a = 0; a < n; ++a) {
        const int32_t dc = inst->cp_ptr[a + 1] - inst->cp_ptr[a], dl = inst->lk_ptr[a + 1] - inst->lk_ptr[a];
        if (dc < 0 || dl < 0) return PT2D_ERR_INVALID_ARG;
        dcmax = std::max(dcmax, dc);
        dlmax = std::max(dlmax, dl);
        degmax = std::max(degmax, dc + dl);
    }
    if ((inst->cp_ptr[n] > 0 && (!inst->cp_col || !inst->cp_J)) || (inst->lk_ptr[n] > 0 && !inst->lk_col))
        return PT2D_ERR_INVALID_ARG;
    bool penalty = false;
    if (inst->lk_w)
        for (int32_t k = 0; k < inst->lk_ptr[n] && !penalty; ++k) penalty = inst->lk_w[k] != 1;
    if (inst->hk)
        for (int32_t a = 0; a < n && !penalty; ++a) penalty = inst->hk[a] != 0;
    int32_t rec_ints;
    if (b->generic) {  // the wide layout (prepare with force_dc < 0), within the declared degree
        if (dcmax > std::max(b->DC, 6)) return PT2D_ERR_INVALID_ARG;
        const int32_t DC = std::max<int32_t>(4, (dcmax + 3) / 4 * 4);
        rec_ints = pt2d::wide_record_ints(DC, dlmax, penalty);
    } else {  // the batch's specialised layout (prepare with force_dc = b->DC)
        if (penalty || inst->g0 != 0 || dlmax > 2 || dcmax > b->DC) return PT2D_ERR_INVALID_ARG;
        rec_ints = 2 * b->DC + 2 + 2;
    }
    const int32_t rec_vec = (rec_ints + 3) / 4;
    const int32_t R = I * J, Rp = pow2_at_least(R);
    // greedy colouring uses between 1 and degmax + 1 colours
    *lo = align_up(block_layout(n, 1, rec_vec, I, J, R, Rp, runs, b->trace_cap).total);
    *hi = align_up(block_layout(n, degmax + 1, rec_vec, I, J, R, Rp, runs, b->trace_cap).total);
    return PT2D_OK;
}

}  // namespace pt2d

extern "C" {

size_t pt2d_batch_instance_bytes(const pt2d_batch *b, const pt2d_instance *inst, int32_t I,
                                 int32_t J, int32_t runs) {
    if (!b || !inst || inst->n < 1 || I < 1 || J < 1 || runs < 1 ||
        static_cast<int64_t>(I) * J > pt2d::kBatchMaxReplicas)
        return 0;
    pt2d::Prep pp;
    pt2d_options o;
    pt2d_default_options(&o);
    o.sweep_kernel = 1;
    if (pt2d::prepare(inst, I, nullptr, J, nullptr, 1, &o, pp, b->generic ? -1 : b->DC, false)) return 0;
    if (b->generic && !degrees_fit(b, pp)) return 0;
    const int32_t R = I * J;
    return align_up(block_layout(inst->n, pp.C, pp.rec_vec, I, J, R, pow2_at_least(R), runs, b->trace_cap)
                        .total);
}

int pt2d_batch_create(pt2d_batch **out, size_t pool_bytes, int32_t max_coupling_degree,
                      int32_t max_runs, const pt2d_options *opt) {
    if (!out || pool_bytes == 0 || max_runs < 1 || max_coupling_degree < 0 || max_coupling_degree > (1 << 20))
        return PT2D_ERR_INVALID_ARG;
    *out = nullptr;
    pt2d_options dflt;
    pt2d_default_options(&dflt);
    if (!opt) opt = &dflt;
    if (opt->device >= 0 && cudaSetDevice(opt->device) != cudaSuccess) return PT2D_ERR_UNSUPPORTED;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return PT2D_ERR_UNSUPPORTED;
    }
    int major = 0, minor = 0, sms = 0, smem_optin = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (major != 10 || minor != 3) return PT2D_ERR_UNSUPPORTED;
    pt2d_batch *b = new (std::nothrow) pt2d_batch;
    if (!b) return PT2D_ERR_OOM;
    b->device = dev;
    // up to 6 coupling neighbours (and 2 links): the specialised kernels, records
    // padded to 3, 4 or 6; more: the runtime-degree kernel, any links and
    // general penalty terms (DC keeps the declared cap, launched as DC = 0)
    b->generic = max_coupling_degree > 6;
    b->DC = b->generic ? max_coupling_degree
                       : (max_coupling_degree <= 3 ? 3 : (max_coupling_degree <= 4 ? 4 : 6));
    b->trace_cap = std::max<int32_t>(opt->trace_capacity, 0);
    b->max_runs = max_runs;
    b->threads = opt->threads_per_cta > 0 ? opt->threads_per_cta : 1024;
    if (b->threads < 128 || b->threads > 1024 || b->threads % 32) {
        delete b;
        return PT2D_ERR_INVALID_ARG;
    }
    b->grid = sms > 0 ? sms : 152;
    b->smem_state_max = std::max(0, smem_optin - static_cast<int>(pt2d::batch_small_smem_bytes()) - 1024);
    b->smem_state_max &= ~15;
    if (opt->swap_mode != PT2D_SWAP_2D && opt->swap_mode != PT2D_SWAP_JCOLUMN) {
        delete b;
        return PT2D_ERR_INVALID_ARG;
    }
    b->swap_mode = opt->swap_mode;
    {
        const pt2d_batch_shape shape{b->threads, opt->sweep_kernel,
                                     opt->walkers_per_cta ? opt->walkers_per_cta : 32, 2};
        if (!apply_shape(b, shape)) {
            delete b;
            return PT2D_ERR_INVALID_ARG;
        }
    }
    if (opt->stream) {
        b->stream = static_cast<cudaStream_t>(opt->stream);
    } else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete b;
            return PT2D_ERR_CUDA;
        }
        b->own_stream = true;
    }
    const size_t head = align_up(sizeof(int32_t)) + align_up(sizeof(pt2d::BatchRun) * max_runs) +
                        align_up(sizeof(int64_t) * 2 * max_runs) +
                        align_up(sizeof(pt2d::BatchItem) * max_runs * pt2d_batch::kMaxSlabs);
    if (opt->workspace) {
        if (opt->workspace_bytes < head + 4096 || (reinterpret_cast<uintptr_t>(opt->workspace) & 255)) {
            pt2d_batch_destroy(b);
            return PT2D_ERR_INVALID_ARG;
        }
        b->pool = static_cast<uint8_t *>(opt->workspace);
        b->pool_bytes = opt->workspace_bytes;
    } else {
        if (pt2d::device_alloc(reinterpret_cast<void **>(&b->pool), pool_bytes + head) != cudaSuccess) {
            cudaGetLastError();
            pt2d_batch_destroy(b);
            return PT2D_ERR_OOM;
        }
        b->own_pool = true;
        b->pool_bytes = pool_bytes + head;
    }
    b->d_queue = reinterpret_cast<int32_t *>(b->pool);
    b->d_runs = reinterpret_cast<pt2d::BatchRun *>(b->pool + align_up(sizeof(int32_t)));
    b->d_status = reinterpret_cast<int64_t *>(b->pool + align_up(sizeof(int32_t)) +
                                              align_up(sizeof(pt2d::BatchRun) * max_runs));
    b->d_items = reinterpret_cast<pt2d::BatchItem *>(
        b->pool + align_up(sizeof(int32_t)) + align_up(sizeof(pt2d::BatchRun) * max_runs) +
        align_up(sizeof(int64_t) * 2 * max_runs));
    b->arena.reset(head, b->pool_bytes - head);
    *out = b;
    return PT2D_OK;
}

void pt2d_batch_destroy(pt2d_batch *b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    drop_graph(b);
    if (b->own_pool && b->pool) cudaFree(b->pool);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

int pt2d_batch_add(pt2d_batch *b, const pt2d_instance *inst, int32_t I, const float *beta, int32_t J,
                   const int32_t *P, int32_t runs, uint64_t seed, const int64_t *target,
                   int64_t *id_out) {
    if (!b || !inst || !beta || !P || !id_out || runs < 1 || I < 1 || J < 1) return PT2D_ERR_INVALID_ARG;
    if (static_cast<int64_t>(I) * J > pt2d::kBatchMaxReplicas) return PT2D_ERR_INVALID_ARG;
    if (runs >= (1 << 27)) return PT2D_ERR_INVALID_ARG;
    pt2d_options o;
    pt2d_default_options(&o);
    o.sweep_kernel = 1;
    Inst in;
    pt2d::Prep pp;
    int st = pt2d::prepare(inst, I, beta, J, P, 1, &o, pp, b->generic ? -1 : b->DC);
    if (st) return st;
    if (b->generic && !degrees_fit(b, pp)) return PT2D_ERR_INVALID_ARG;
    in.n = pp.n;
    in.I = I;
    in.J = J;
    in.R = I * J;
    in.Rp = pow2_at_least(in.R);
    in.runs = runs;
    in.C = pp.C;
    in.rec_vec = pp.rec_vec;
    in.pos_of = pp.pos_of;
    in.color = pp.color;
    const Layout1 l = block_layout(in.n, in.C, in.rec_vec, I, J, in.R, in.Rp, runs, b->trace_cap);
    if (!b->arena.alloc(l.total, &in.off)) return PT2D_ERR_OOM;
    in.bytes = l.total;
    cudaSetDevice(b->device);
    cudaStream_t s = b->stream;
    uint8_t *base = b->pool + in.off;
    auto undo = [&](cudaError_t e) {
        b->arena.release(in.off, in.bytes);
        return fail(b, e);
    };
    cudaError_t e = cudaMemsetAsync(base, 0, l.total, s);
    if (e != cudaSuccess) return undo(e);
    e = cudaMemcpyAsync(base + l.rec, pp.rec.data(), sizeof(int32_t) * pp.rec.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + l.cofs, pp.cofs.data(), sizeof(int32_t) * pp.cofs.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + l.beta, beta, sizeof(float) * I, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + l.P, P, sizeof(int32_t) * J, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return undo(e);
    std::vector<int64_t> scal(static_cast<size_t>(runs) * pt2d::kScCount, 0);
    for (int32_t r = 0; r < runs; ++r) {
        pt2d::BatchRun d{};
        d.swap_mode = b->swap_mode;
        const size_t rb = in.off + l.run0 + l.run_stride * r;
        d.state = static_cast<int64_t>(rb + l.state);
        d.rec = static_cast<int64_t>(in.off + l.rec);
        d.cofs = static_cast<int64_t>(in.off + l.cofs);
        d.beta = static_cast<int64_t>(in.off + l.beta);
        d.P = static_cast<int64_t>(in.off + l.P);
        d.walker_at = static_cast<int64_t>(rb + l.walker_at);
        d.wparam = static_cast<int64_t>(rb + l.wparam);
        d.counter = static_cast<int64_t>(rb + l.counter);
        d.fg = static_cast<int64_t>(rb + l.fg);
        d.stats = static_cast<int64_t>(rb + l.stats);
        d.trace = static_cast<int64_t>(rb + l.trace);
        d.best_state = static_cast<int64_t>(rb + l.best_state);
        d.scalars = static_cast<int64_t>(rb + l.scalars);
        d.k0 = static_cast<uint32_t>(seed);
        d.k1 = static_cast<uint32_t>(seed >> 32);
        d.n = in.n;
        d.C = in.C;
        d.I = I;
        d.J = J;
        d.R = in.R;
        d.Rp = in.Rp;
        d.run = r;
        d.trace_cap = b->trace_cap;
        d.rec_vec = in.rec_vec;
        d.dc = pp.DC;
        d.dl = pp.DL;
        d.penalty = pp.penalty ? 1 : 0;
        d.g0 = pp.g0;
        d.work = static_cast<int64_t>(in.n) * in.Rp;
        in.desc.push_back(d);
        scal[static_cast<size_t>(r) * pt2d::kScCount + pt2d::kScTarget] = target ? target[r] : INT64_MIN;
    }
    for (int32_t r = 0; r < runs; ++r) {
        e = cudaMemcpyAsync(b->pool + in.desc[r].scalars, scal.data() + static_cast<size_t>(r) * pt2d::kScCount,
                            pt2d::kScCount * 8, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return undo(e);
    }
    // host copies of pp's vectors must outlive the async copies
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return undo(e);
    const int64_t id = b->next_id++;
    b->insts.emplace(id, std::move(in));
    b->dirty = true;
    *id_out = id;
    return PT2D_OK;
}

int pt2d_batch_remove(pt2d_batch *b, int64_t id) {
    if (!b) return PT2D_ERR_INVALID_ARG;
    auto it = b->insts.find(id);
    if (it == b->insts.end()) return PT2D_ERR_INVALID_ARG;
    // later work on the stream may reuse the block; earlier launches finish first
    b->arena.release(it->second.off, it->second.bytes);
    b->insts.erase(it);
    b->dirty = true;
    return PT2D_OK;
}

int pt2d_batch_run(pt2d_batch *b, int32_t events, int32_t swap_interval) {
    pt2d::TraceRange trace("pt2d_batch_run");
    if (!b || events < 0 || swap_interval < 1) return PT2D_ERR_INVALID_ARG;
    cudaSetDevice(b->device);
    return launch(b, events, swap_interval);
}

int pt2d_batch_sync(pt2d_batch *b) {
    if (!b) return PT2D_ERR_INVALID_ARG;
    BK(b, cudaStreamSynchronize(b->stream));
    return PT2D_OK;
}

int pt2d_batch_get_shape(const pt2d_batch *b, pt2d_batch_shape *shape) {
    if (!b || !shape) return PT2D_ERR_INVALID_ARG;
    *shape = current_shape(b);
    return PT2D_OK;
}

int pt2d_batch_set_shape(pt2d_batch *b, const pt2d_batch_shape *shape) {
    if (!b || !shape) return PT2D_ERR_INVALID_ARG;
    return apply_shape(b, *shape) ? PT2D_OK : PT2D_ERR_INVALID_ARG;
}

int pt2d_batch_autotune(pt2d_batch *b, int32_t events, int32_t swap_interval, pt2d_batch_shape *chosen) {
    pt2d::TraceRange trace("pt2d_batch_autotune");
    if (!b || events < 1 || swap_interval < 1) return PT2D_ERR_INVALID_ARG;
    cudaSetDevice(b->device);
    struct Events {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        ~Events() {
            if (e0) cudaEventDestroy(e0);
            if (e1) cudaEventDestroy(e1);
        }
    } ev;
    BK(b, cudaEventCreate(&ev.e0));
    BK(b, cudaEventCreate(&ev.e1));
    const pt2d_batch_shape start = current_shape(b);
    float best_ms = -1.0f;
    pt2d_batch_shape best = start;
    // Every launch shape computes the same trajectories, so the trial launches are
    // ordinary progress of the chains.
    auto trial = [&](const pt2d_batch_shape &sh) -> int {
        apply_shape(b, sh);
        int st = launch(b, events, swap_interval);  // first launch per shape: not timed
        if (st) return st;
        BK(b, cudaEventRecord(ev.e0, b->stream));
        st = launch(b, events, swap_interval);
        if (st) return st;
        BK(b, cudaEventRecord(ev.e1, b->stream));
        BK(b, cudaEventSynchronize(ev.e1));
        float ms = 0.0f;
        BK(b, cudaEventElapsedTime(&ms, ev.e0, ev.e1));
        if (best_ms < 0.0f || ms < best_ms) {
            best_ms = ms;
            best = sh;
        }
        return PT2D_OK;
    };
    // balance 4 matters for batches of equal runs: 128 copies of one N = 200
    // instance are cut into 512 bit-packed slabs at balance 2 (3.4 per CTA: the
    // last wave a third full), 1024 at 4 (16.3 against 17.7 ms per event)
    for (int storage : {0, 1, 2})
        for (int balance : {0, 2, 4, 8}) {
            pt2d_batch_shape sh = start;
            sh.threads_per_cta = 1024;
            sh.storage = storage;
            sh.balance = balance;
            if (int st = trial(sh)) return st;
        }
    // fewer threads per CTA: batches of small problems then fit several CTAs
    // (several slabs at once) on an SM
    const pt2d_batch_shape wide = best;
    for (int threads : {512, 256, 128}) {
        pt2d_batch_shape sh = wide;
        sh.threads_per_cta = threads;
        if (int st = trial(sh)) return st;
    }
    apply_shape(b, best);
    if (chosen) *chosen = best;
    return PT2D_OK;
}

int pt2d_batch_poll(pt2d_batch *b, int64_t *ids, int64_t *solved_event, int64_t *events_done,
                    int32_t capacity, int32_t *count) {
    if (!b || !count || (capacity > 0 && (!ids || !solved_event || !events_done)))
        return PT2D_ERR_INVALID_ARG;
    cudaSetDevice(b->device);
    std::vector<int64_t> st(2 * b->order.size());
    if (!st.empty()) {
        BK(b, cudaMemcpyAsync(st.data(), b->d_status, sizeof(int64_t) * st.size(),
                              cudaMemcpyDeviceToHost, b->stream));
    }
    BK(b, cudaStreamSynchronize(b->stream));
    // aggregate over runs: solved at the earliest run's solving event
    std::map<int64_t, std::pair<int64_t, int64_t>> agg;
    for (size_t i = 0; i < b->order.size(); ++i) {
        const int64_t id = b->order[i].first;
        if (!b->insts.count(id)) continue;
        auto it = agg.find(id);
        const int64_t se = st[2 * i], ev = st[2 * i + 1];
        if (it == agg.end()) {
            agg[id] = {se, ev};
        } else {
            if (se >= 0 && (it->second.first < 0 || se < it->second.first)) it->second.first = se;
            it->second.second = std::min(it->second.second, ev);
        }
    }
    int32_t k = 0;
    for (const auto &kv : agg) {
        if (k < capacity) {
            ids[k] = kv.first;
            solved_event[k] = kv.second.first;
            events_done[k] = kv.second.second;
        }
        ++k;
    }
    *count = k;
    return PT2D_OK;
}

size_t pt2d_batch_free_bytes(const pt2d_batch *b) { return b ? b->arena.largest() : 0; }

int64_t pt2d_batch_launch_count(const pt2d_batch *b) { return b ? b->launches : 0; }

int pt2d_batch_cuda_error(const pt2d_batch *b) { return b ? b->last_cuda : 0; }

size_t pt2d_batch_array_bytes(const pt2d_batch *b, int64_t id, int32_t what) {
    if (!b) return 0;
    auto it = b->insts.find(id);
    if (it == b->insts.end()) return 0;
    const Inst &in = it->second;
    const size_t RR = static_cast<size_t>(in.runs) * in.R;
    switch (what) {
        case PT2D_STATES: return RR * in.n;
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
        case PT2D_TRACE_G: return static_cast<size_t>(in.runs) * b->trace_cap * 8;
        case PT2D_BEST_F:
        case PT2D_BEST_EVENT:
        case PT2D_SOLVED_EVENT:
        case PT2D_TARGET: return static_cast<size_t>(in.runs) * 8;
        case PT2D_BEST_STATE: return static_cast<size_t>(in.runs) * in.n;
        case PT2D_COLORS: return static_cast<size_t>(in.n) * 4;
        default: return 0;
    }
}

int pt2d_batch_read(pt2d_batch *b, int64_t id, int32_t what, void *dst, size_t bytes) {
    if (!b || !dst) return PT2D_ERR_INVALID_ARG;
    auto it = b->insts.find(id);
    if (it == b->insts.end()) return PT2D_ERR_INVALID_ARG;
    const size_t need = pt2d_batch_array_bytes(b, id, what);
    if (need == 0 || bytes != need) return PT2D_ERR_INVALID_ARG;
    const Inst &in = it->second;
    cudaSetDevice(b->device);
    BK(b, cudaStreamSynchronize(b->stream));
    if (what == PT2D_COLORS) {
        std::memcpy(dst, in.color.data(), need);
        return PT2D_OK;
    }
    auto copy = [&](void *h, int64_t off, size_t nbytes) -> cudaError_t {
        return cudaMemcpy(h, b->pool + off, nbytes, cudaMemcpyDeviceToHost);
    };
    const int32_t R = in.R, n = in.n;
    for (int32_t r = 0; r < in.runs; ++r) {
        const pt2d::BatchRun &d = in.desc[r];
        int64_t sc[pt2d::kScCount];
        BK(b, copy(sc, d.scalars, sizeof sc));
        switch (what) {
            case PT2D_STATES: {
                if (!sc[pt2d::kScInited]) return PT2D_ERR_STATE;
                std::vector<int8_t> tmp(static_cast<size_t>(n + 1) * in.Rp);
                BK(b, copy(tmp.data(), d.state, tmp.size()));
                int8_t *o = static_cast<int8_t *>(dst) + static_cast<size_t>(r) * R * n;
                for (int32_t w = 0; w < R; ++w)
                    for (int32_t a = 0; a < n; ++a)
                        o[static_cast<size_t>(w) * n + a] = tmp[static_cast<size_t>(in.pos_of[a]) * in.Rp + w];
                break;
            }
            case PT2D_WALKER_AT:
                BK(b, copy(static_cast<int32_t *>(dst) + static_cast<size_t>(r) * R, d.walker_at, 4 * R));
                break;
            case PT2D_F:
            case PT2D_G: {
                std::vector<int64_t> f(in.Rp);
                std::vector<int32_t> g(in.Rp);
                BK(b, copy(f.data(), d.fg, 8 * in.Rp));
                BK(b, copy(g.data(), d.fg + 8 * in.Rp, 4 * in.Rp));
                int64_t *o = static_cast<int64_t *>(dst) + static_cast<size_t>(r) * R;
                for (int32_t w = 0; w < R; ++w) o[w] = what == PT2D_F ? f[w] : g[w];
                break;
            }
            case PT2D_COUNTERS: {
                if (r == 0) {
                    const int64_t ev = sc[pt2d::kScEvents];
                    const int64_t dir = b->swap_mode ? -1 : (((ev / 2) % 2 == 0) ? 1 : -1);
                    int64_t v[4] = {sc[pt2d::kScSweeps], ev, dir, sc[pt2d::kScInited]};
                    std::memcpy(dst, v, sizeof v);
                }
                break;
            }
            case PT2D_TRACE_F:
            case PT2D_TRACE_G:
                if (b->trace_cap)
                    BK(b, copy(static_cast<int64_t *>(dst) + static_cast<size_t>(r) * b->trace_cap,
                               d.trace + (what == PT2D_TRACE_G ? 8 * b->trace_cap : 0), 8 * b->trace_cap));
                break;
            case PT2D_BEST_F: static_cast<int64_t *>(dst)[r] = sc[pt2d::kScInited] ? sc[pt2d::kScBestF] : INT64_MAX; break;
            case PT2D_BEST_EVENT: static_cast<int64_t *>(dst)[r] = sc[pt2d::kScInited] ? sc[pt2d::kScBestEvent] : -1; break;
            case PT2D_SOLVED_EVENT: static_cast<int64_t *>(dst)[r] = sc[pt2d::kScInited] ? sc[pt2d::kScSolvedEvent] : -1; break;
            case PT2D_TARGET: static_cast<int64_t *>(dst)[r] = sc[pt2d::kScTarget]; break;
            case PT2D_BEST_STATE:
                BK(b, copy(static_cast<int8_t *>(dst) + static_cast<size_t>(r) * n, d.best_state, n));
                break;
            case PT2D_ACC_P:
            case PT2D_ACC_B:
            case PT2D_SUM_F:
            case PT2D_SUM_G:
            case PT2D_N_FEASIBLE: {
                const int k = what == PT2D_ACC_P ? 0 : what == PT2D_ACC_B ? 1 : what == PT2D_SUM_F ? 2 : what == PT2D_SUM_G ? 3 : 4;
                BK(b, copy(static_cast<int64_t *>(dst) + static_cast<size_t>(r) * R, d.stats + 8LL * R * k, 8 * R));
                break;
            }
            default:
                return PT2D_ERR_INVALID_ARG;
        }
    }
    return PT2D_OK;
}

}  // extern "C"
