// Adaptive ladder schedule for 2D-PT (include/pt2d.h, pt2d_adaptive_schedule):
// the paper's Algorithm 2 as a host driver over the library's contexts.
//
// The first column (penalty P0) grows rows: each new inverse temperature is one
// step alpha_beta / sigma_E above the last, until the energy spread of a row's
// population falls to sigma_min or the row cap is reached.  Every row that
// steps also proposes the next column's penalty, alpha_P / (beta sigma_g)
// above its own; the next column takes the median proposal.  Later columns
// repeat the row walk from beta0 at their penalty and stop once the coldest
// row's population is feasible on average (mean g < 1/2) or the column cap is
// reached.  The final beta ladder is the median over the columns of each row.
//
// A population sample at (beta, P) is n_chain runs of a 1 x 1 grid: mcs
// heat-bath sweeps from the initial state (one event, so no swap happens),
// then E = f + P g and g of each chain.  Sample k uses seed + k.  Statistics
// come from exact integer sums, rounded once to double; everything after that
// is IEEE double in a fixed order, so the ladders are reproducible bit for bit.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/pt2d.h"
#include "pt2d_trace.h"

namespace {

using i128 = __int128;
using u128 = unsigned __int128;

// Nearest double to an exact integer (ties to even).
double to_double(i128 v) {
    const bool neg = v < 0;
    u128 m = neg ? static_cast<u128>(-(v + 1)) + 1 : static_cast<u128>(v);
    if (m < (static_cast<u128>(1) << 53)) {
        const double d = static_cast<double>(static_cast<uint64_t>(m));
        return neg ? -d : d;
    }
    int bits = 0;
    for (u128 t = m; t; t >>= 1) ++bits;
    int shift = bits - 53;
    u128 q = m >> shift;
    const u128 rem = m & ((static_cast<u128>(1) << shift) - 1);
    const u128 half = static_cast<u128>(1) << (shift - 1);
    if (rem > half || (rem == half && (q & 1))) ++q;
    if (q == (static_cast<u128>(1) << 53)) {
        q >>= 1;
        ++shift;
    }
    const double d = std::ldexp(static_cast<double>(static_cast<uint64_t>(q)), shift);
    return neg ? -d : d;
}

struct Stats {
    double sig_E, sig_g, mean_g;
};

Stats population_stats(const std::vector<int64_t> &E, const std::vector<int64_t> &g) {
    const i128 n = static_cast<i128>(E.size());
    i128 s1 = 0, s2 = 0, t1 = 0, t2 = 0;
    for (size_t c = 0; c < E.size(); ++c) {
        s1 += E[c];
        s2 += static_cast<i128>(E[c]) * E[c];
        t1 += g[c];
        t2 += static_cast<i128>(g[c]) * g[c];
    }
    const double nn = to_double(n * n);
    Stats st;
    st.sig_E = std::sqrt(to_double(n * s2 - s1 * s1) / nn);
    st.sig_g = std::sqrt(to_double(n * t2 - t1 * t1) / nn);
    st.mean_g = to_double(t1) / to_double(n);
    return st;
}

double median(std::vector<double> v) {
    std::sort(v.begin(), v.end());
    const size_t m = v.size();
    if (m % 2) return v[m / 2];
    return (v[m / 2 - 1] + v[m / 2]) / 2;
}

struct Sampler {
    const pt2d_instance *inst;
    const pt2d_schedule_params *prm;
    pt2d_options opt;
    int64_t k = 0;
    std::vector<int64_t> f, g, E;

    int operator()(double beta, int32_t P, Stats *out) {
        const float bf = static_cast<float>(beta);
        pt2d_ctx *ctx = nullptr;
        int st = pt2d_create(&ctx, inst, 1, &bf, 1, &P, prm->n_chain, &opt);
        if (st) return st;
        st = pt2d_run(ctx, prm->mcs, prm->mcs, prm->seed + static_cast<uint64_t>(k));
        const size_t bytes = sizeof(int64_t) * static_cast<size_t>(prm->n_chain);
        if (!st) st = pt2d_read(ctx, PT2D_F, f.data(), bytes);
        if (!st) st = pt2d_read(ctx, PT2D_G, g.data(), bytes);
        pt2d_destroy(ctx);
        if (st) return st;
        for (int32_t c = 0; c < prm->n_chain; ++c) E[c] = f[c] + static_cast<int64_t>(P) * g[c];
        *out = population_stats(E, g);
        ++k;
        return PT2D_OK;
    }
};

bool valid(const pt2d_schedule_params *p) {
    return p->beta0 > 0 && std::isfinite(p->beta0) && p->P0 >= 0 && p->max_rows >= 1 &&
           p->max_cols >= 1 && p->sigma_min > 0 && p->alpha_beta > 0 && p->alpha_P > 0 &&
           std::isfinite(p->sigma_min) && std::isfinite(p->alpha_beta) && std::isfinite(p->alpha_P) &&
           p->n_chain >= 2 && p->mcs >= 1;
}

}  // namespace

extern "C" int pt2d_adaptive_schedule(const pt2d_instance *inst, const pt2d_schedule_params *prm,
                                      const pt2d_options *opt, float *beta_out, int32_t *I_out,
                                      int32_t *P_out, int32_t *J_out, int64_t *samples_out) {
    if (!inst || !prm || !beta_out || !I_out || !P_out || !J_out || !valid(prm)) return PT2D_ERR_INVALID_ARG;
    Sampler s{inst, prm, {}};
    if (opt) {
        s.opt = *opt;
    } else {
        pt2d_default_options(&s.opt);
    }
    s.opt.trace_capacity = 0;
    s.opt.profile = 0;
    // Every population sample is a 1 x 1 context of n_chain runs: one device
    // workspace, allocated here and reused by each of them (a context on caller
    // memory clears what it carves at creation), saves a cudaMalloc / cudaFree
    // pair per sample.
    struct Workspace {
        void *p = nullptr;
        ~Workspace() {
            if (p) cudaFree(p);
        }
    } ws;
    if (!s.opt.workspace) {
        size_t need = 0;
        if (int e = pt2d_workspace_size(inst, 1, 1, prm->n_chain, &s.opt, &need)) return e;
        if (s.opt.device >= 0 && cudaSetDevice(s.opt.device) != cudaSuccess) return PT2D_ERR_UNSUPPORTED;
        if (int e = pt2d::check_device()) return e;
        if (pt2d::device_alloc(&ws.p, need) != cudaSuccess) {
            cudaGetLastError();
            ws.p = nullptr;
            return PT2D_ERR_OOM;
        }
        s.opt.workspace = ws.p;
        s.opt.workspace_bytes = need;
    }
    s.f.resize(prm->n_chain);
    s.g.resize(prm->n_chain);
    s.E.resize(prm->n_chain);

    // first column, penalty P0
    std::vector<std::vector<double>> cols;
    std::vector<double> col{prm->beta0};
    std::vector<double> proposals;
    for (int32_t i = 0; i < prm->max_rows; ++i) {
        const double b = col[i];
        Stats st;
        if (int e = s(b, prm->P0, &st)) return e;
        if (!(st.sig_E > prm->sigma_min)) break;
        if (i + 1 < prm->max_rows) col.push_back(b + prm->alpha_beta / st.sig_E);
        if (st.sig_g > 0) proposals.push_back(prm->P0 + prm->alpha_P / (b * st.sig_g));
    }
    const int32_t I = static_cast<int32_t>(col.size());
    cols.push_back(col);
    std::vector<int32_t> P{prm->P0};
    // remaining columns
    while (static_cast<int32_t>(P.size()) < prm->max_cols && !proposals.empty()) {
        const double next = std::nearbyint(median(proposals));
        if (!(next >= 0 && next <= 2147483647.0)) return PT2D_ERR_INVALID_ARG;
        const int32_t Pj = static_cast<int32_t>(next);
        P.push_back(Pj);
        col.assign(1, prm->beta0);
        proposals.clear();
        double mean_g = 0.0;
        for (int32_t i = 0; i < I; ++i) {
            const double b = col[i];
            Stats st;
            if (int e = s(b, Pj, &st)) return e;
            mean_g = st.mean_g;
            if (i + 1 < I) col.push_back(b + prm->alpha_beta / std::max(st.sig_E, prm->sigma_min));
            if (st.sig_g > 0) proposals.push_back(Pj + prm->alpha_P / (b * st.sig_g));
        }
        cols.push_back(col);
        if (mean_g < 0.5) break;  // the coldest row of this column is feasible on average
    }
    for (int32_t i = 0; i < I; ++i) {
        std::vector<double> row;
        for (const auto &c : cols) row.push_back(c[i]);
        beta_out[i] = static_cast<float>(median(row));
    }
    std::memcpy(P_out, P.data(), sizeof(int32_t) * P.size());
    *I_out = I;
    *J_out = static_cast<int32_t>(P.size());
    if (samples_out) *samples_out = s.k;
    return PT2D_OK;
}
