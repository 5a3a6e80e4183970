// Continuous-batching server for constrained Ising problems (include/pt2d.h,
// pt2d_server_*), built on the batched persistent kernel.
//
// Requests wait in a FIFO queue with a host copy of their problem.  Each step
// admits queued requests in order while the device pool has room (a request
// that does not fit blocks the ones behind it, so large requests are not
// starved), runs one batched launch of `events_per_step` events over every
// resident request, then evicts the requests that are solved (bottom-right
// g = 0 and f <= target) or out of sweeps, keeping their lowest-energy
// feasible state.  A request's trajectory depends only on its own problem,
// seed and events, never on what else is resident, and eviction happens at a
// whole number of steps after its admission, so its result is the same alone
// and in any mix.
#include <chrono>
#include <cstdint>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <vector>

#include "../../include/pt2d.h"
#include "pt2d_batch.h"
#include "pt2d_trace.h"

namespace {

struct Request {
    int32_t n = 0, I = 0, J = 0;
    std::vector<int32_t> cp_ptr, cp_col, lk_ptr, lk_col, h, color, hk;
    std::vector<int16_t> cp_J, lk_w;
    bool has_h = false, has_color = false, has_lk_w = false, has_hk = false;
    int64_t g0 = 0;
    std::vector<float> beta;
    std::vector<int32_t> P;
    uint64_t seed = 0;
    int64_t target = 0, max_sweeps = 0;
    int32_t state = PT2D_REQUEST_QUEUED;
    int32_t error = 0;
    int64_t batch_id = -1;
    double t_submit = 0, t_admit = -1, t_done = -1;
    int64_t best_f = INT64_MAX, best_event = -1, solved_event = -1, sweeps_done = 0;
    std::vector<int8_t> best_state;

    pt2d_instance view() const {
        pt2d_instance v{};
        v.n = n;
        v.cp_ptr = cp_ptr.data();
        v.cp_col = cp_col.data();
        v.cp_J = cp_J.data();
        v.lk_ptr = lk_ptr.data();
        v.lk_col = lk_col.data();
        v.h = has_h ? h.data() : nullptr;
        v.color = has_color ? color.data() : nullptr;
        v.lk_w = has_lk_w ? lk_w.data() : nullptr;
        v.hk = has_hk ? hk.data() : nullptr;
        v.g0 = g0;
        return v;
    }
};

}  // namespace

struct pt2d_server {
    pt2d_batch *b = nullptr;
    int32_t interval = 50;
    int32_t events_per_step = 10;
    int32_t max_runs = 0;
    size_t capacity = 0;  // pool bytes when empty: a request needing more can never be admitted
    std::deque<int64_t> queue;
    std::map<int64_t, Request> reqs;
    std::map<int64_t, int64_t> by_batch;  // batch id -> request id
    int64_t next_id = 1;
    int64_t steps = 0;
    std::chrono::steady_clock::time_point t0;
};

namespace {

double now_s(const pt2d_server *s) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - s->t0).count();
}

int finish(pt2d_server *s, Request &r) {
    int st = pt2d_batch_read(s->b, r.batch_id, PT2D_BEST_F, &r.best_f, sizeof(int64_t));
    if (!st) st = pt2d_batch_read(s->b, r.batch_id, PT2D_BEST_EVENT, &r.best_event, sizeof(int64_t));
    if (!st) st = pt2d_batch_read(s->b, r.batch_id, PT2D_SOLVED_EVENT, &r.solved_event, sizeof(int64_t));
    int64_t counters[4] = {0, 0, 0, 0};
    if (!st) st = pt2d_batch_read(s->b, r.batch_id, PT2D_COUNTERS, counters, sizeof counters);
    r.best_state.assign(r.n, 0);
    if (!st) st = pt2d_batch_read(s->b, r.batch_id, PT2D_BEST_STATE, r.best_state.data(), r.n);
    if (st) return st;
    r.sweeps_done = counters[0];
    pt2d_batch_remove(s->b, r.batch_id);
    s->by_batch.erase(r.batch_id);
    r.batch_id = -1;
    r.state = PT2D_REQUEST_DONE;
    r.t_done = now_s(s);
    return PT2D_OK;
}

}  // namespace

extern "C" {

int pt2d_server_create(pt2d_server **out, size_t pool_bytes, int32_t max_coupling_degree,
                       int32_t max_requests, int32_t swap_interval, int32_t events_per_step,
                       const pt2d_options *opt) {
    if (!out || swap_interval < 1 || events_per_step < 1 || max_requests < 1) return PT2D_ERR_INVALID_ARG;
    *out = nullptr;
    pt2d_server *s = new (std::nothrow) pt2d_server;
    if (!s) return PT2D_ERR_OOM;
    pt2d_options o;
    if (opt) {
        o = *opt;
    } else {
        pt2d_default_options(&o);
    }
    o.trace_capacity = 0;
    int st = pt2d_batch_create(&s->b, pool_bytes, max_coupling_degree, max_requests, &o);
    if (st) {
        delete s;
        return st;
    }
    s->capacity = pt2d_batch_free_bytes(s->b);
    s->interval = swap_interval;
    s->events_per_step = events_per_step;
    s->max_runs = max_requests;
    s->t0 = std::chrono::steady_clock::now();
    *out = s;
    return PT2D_OK;
}

void pt2d_server_destroy(pt2d_server *s) {
    if (!s) return;
    pt2d_batch_destroy(s->b);
    delete s;
}

int pt2d_server_submit(pt2d_server *s, const pt2d_instance *inst, int32_t I, const float *beta,
                       int32_t J, const int32_t *P, uint64_t seed, int64_t target,
                       int64_t max_sweeps, int64_t *request_id) {
    if (!s || !inst || !beta || !P || !request_id || inst->n < 1 || I < 1 || J < 1 || max_sweeps < 1 ||
        !inst->cp_ptr || !inst->lk_ptr)
        return PT2D_ERR_INVALID_ARG;
    // Size from the degrees alone (no colouring, no CSR check: a submission
    // costs O(n) here, so a stream of submissions does not starve the step
    // loop); the exact size only when the bounds straddle the pool.  A problem
    // larger than the pool would block the FIFO head for ever.
    size_t lo = 0, hi = 0;
    if (int st = pt2d::batch_instance_bytes_bounds(s->b, inst, I, J, 1, &lo, &hi)) return st;
    if (lo > s->capacity) return PT2D_ERR_OOM;
    if (hi > s->capacity) {
        const size_t need = pt2d_batch_instance_bytes(s->b, inst, I, J, 1);
        if (need == 0) return PT2D_ERR_INVALID_ARG;
        if (need > s->capacity) return PT2D_ERR_OOM;
    }
    Request r;
    const int32_t n = inst->n;
    r.n = n;
    r.I = I;
    r.J = J;
    r.cp_ptr.assign(inst->cp_ptr, inst->cp_ptr + n + 1);
    r.cp_col.assign(inst->cp_col, inst->cp_col + r.cp_ptr[n]);
    r.cp_J.assign(inst->cp_J, inst->cp_J + r.cp_ptr[n]);
    r.lk_ptr.assign(inst->lk_ptr, inst->lk_ptr + n + 1);
    r.lk_col.assign(inst->lk_col, inst->lk_col + r.lk_ptr[n]);
    if (inst->h) {
        r.h.assign(inst->h, inst->h + n);
        r.has_h = true;
    }
    if (inst->color) {
        r.color.assign(inst->color, inst->color + n);
        r.has_color = true;
    }
    if (inst->lk_w) {
        r.lk_w.assign(inst->lk_w, inst->lk_w + r.lk_ptr[n]);
        r.has_lk_w = true;
    }
    if (inst->hk) {
        r.hk.assign(inst->hk, inst->hk + n);
        r.has_hk = true;
    }
    r.g0 = inst->g0;
    r.beta.assign(beta, beta + I);
    r.P.assign(P, P + J);
    r.seed = seed;
    r.target = target;
    r.max_sweeps = max_sweeps;
    r.t_submit = now_s(s);
    const int64_t id = s->next_id++;
    s->reqs.emplace(id, std::move(r));
    s->queue.push_back(id);
    *request_id = id;
    return PT2D_OK;
}

int pt2d_server_step(pt2d_server *s, int32_t *active, int32_t *queued, int32_t *finished) {
    pt2d::TraceRange trace("pt2d_server_step");
    if (!s) return PT2D_ERR_INVALID_ARG;
    // admit in arrival order while the pool has room
    while (!s->queue.empty() && static_cast<int32_t>(s->by_batch.size()) < s->max_runs) {
        const int64_t rid = s->queue.front();
        Request &r = s->reqs[rid];
        if (r.state == PT2D_REQUEST_CANCELLED) {
            s->queue.pop_front();
            continue;
        }
        const pt2d_instance v = r.view();
        int64_t bid = -1;
        const int st = pt2d_batch_add(s->b, &v, r.I, r.beta.data(), r.J, r.P.data(), 1, r.seed,
                                      &r.target, &bid);
        if (st == PT2D_ERR_OOM) break;
        s->queue.pop_front();
        if (st) {
            r.state = PT2D_REQUEST_FAILED;
            r.error = st;
            r.t_done = now_s(s);
            continue;
        }
        r.batch_id = bid;
        r.state = PT2D_REQUEST_RUNNING;
        r.t_admit = now_s(s);
        s->by_batch[bid] = rid;
    }
    int32_t done = 0;
    if (!s->by_batch.empty()) {
        int st = pt2d_batch_run(s->b, s->events_per_step, s->interval);
        if (st) return st;
        s->steps += 1;
        const int32_t cap = static_cast<int32_t>(s->by_batch.size());
        std::vector<int64_t> ids(cap), se(cap), ev(cap);
        int32_t cnt = 0;
        st = pt2d_batch_poll(s->b, ids.data(), se.data(), ev.data(), cap, &cnt);
        if (st) return st;
        for (int32_t k = 0; k < std::min(cnt, cap); ++k) {
            auto it = s->by_batch.find(ids[k]);
            if (it == s->by_batch.end()) continue;
            Request &r = s->reqs[it->second];
            r.sweeps_done = ev[k] * s->interval;
            if (se[k] >= 0 || r.sweeps_done >= r.max_sweeps) {
                st = finish(s, r);
                if (st) return st;
                ++done;
            }
        }
    }
    if (active) *active = static_cast<int32_t>(s->by_batch.size());
    if (queued) *queued = static_cast<int32_t>(s->queue.size());
    if (finished) *finished = done;
    return PT2D_OK;
}

int pt2d_server_status(pt2d_server *s, int64_t request_id, pt2d_request_status *out,
                       int8_t *best_state) {
    if (!s || !out) return PT2D_ERR_INVALID_ARG;
    auto it = s->reqs.find(request_id);
    if (it == s->reqs.end()) return PT2D_ERR_INVALID_ARG;
    const Request &r = it->second;
    out->state = r.state;
    out->error = r.error;
    out->n = r.n;
    out->best_f = r.best_f;
    out->best_event = r.best_event;
    out->solved_event = r.solved_event;
    out->sweeps_done = r.sweeps_done;
    out->t_submit = r.t_submit;
    out->t_admit = r.t_admit;
    out->t_done = r.t_done;
    if (best_state && r.state == PT2D_REQUEST_DONE) std::memcpy(best_state, r.best_state.data(), r.n);
    return PT2D_OK;
}

int pt2d_server_cancel(pt2d_server *s, int64_t request_id) {
    if (!s) return PT2D_ERR_INVALID_ARG;
    auto it = s->reqs.find(request_id);
    if (it == s->reqs.end()) return PT2D_ERR_INVALID_ARG;
    Request &r = it->second;
    if (r.state == PT2D_REQUEST_RUNNING) {
        pt2d_batch_remove(s->b, r.batch_id);
        s->by_batch.erase(r.batch_id);
        r.batch_id = -1;
    }
    if (r.state == PT2D_REQUEST_QUEUED || r.state == PT2D_REQUEST_RUNNING) {
        r.state = PT2D_REQUEST_CANCELLED;
        r.t_done = now_s(s);
    }
    return PT2D_OK;
}

int pt2d_server_forget(pt2d_server *s, int64_t request_id) {
    if (!s) return PT2D_ERR_INVALID_ARG;
    auto it = s->reqs.find(request_id);
    if (it == s->reqs.end()) return PT2D_ERR_INVALID_ARG;
    if (it->second.state == PT2D_REQUEST_QUEUED || it->second.state == PT2D_REQUEST_RUNNING)
        return PT2D_ERR_STATE;
    s->reqs.erase(it);
    return PT2D_OK;
}

size_t pt2d_server_free_bytes(const pt2d_server *s) { return s ? pt2d_batch_free_bytes(s->b) : 0; }

}  // extern "C"
