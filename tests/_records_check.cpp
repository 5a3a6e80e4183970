// Host-side check of the packed neighbour records that pt2d::prepare builds
// (test helper, compiled by tests/test_records.py against libpt2d.so; no GPU).
//
// For random instances it decodes every record with the documented layouts
// (specialised, penalty-specialised, wide) and compares the result with the
// instance it came from: the spin id, 2h, every coupling (neighbour and J,
// padding entries pointing at the zero row with J = 0; for coupling width 3 also
// the packed J bytes), every copy link, and with penalty terms the link
// weights K and the field k.  Prints "ok" or the
// first mismatch and exits non-zero.
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <map>
#include <random>
#include <vector>

#include "pt2d_prep.h"
#include "pt2d_wide.cuh"

namespace {

struct Inst {
    int n = 0;
    std::vector<int32_t> cp_ptr, cp_col, lk_ptr, lk_col, h, hk;
    std::vector<int16_t> cp_J, lk_w;
    std::vector<std::map<int, int>> cadj, ladj;  // neighbour -> J / K
};

Inst make(std::mt19937 &rng, int n, int max_deg, int link_deg, bool penalty) {
    Inst in;
    in.n = n;
    in.cadj.resize(n);
    in.ladj.resize(n);
    std::vector<int> deg(n, 0);
    for (int tries = 0; tries < n * max_deg * 4; ++tries) {
        const int a = static_cast<int>(rng() % n), b = static_cast<int>(rng() % n);
        if (a == b || deg[a] >= max_deg || deg[b] >= max_deg || in.cadj[a].count(b)) continue;
        int J = static_cast<int>(rng() % 65535) - 32767;
        if (J == 0) J = -32768;
        in.cadj[a][b] = J;
        in.cadj[b][a] = J;
        ++deg[a];
        ++deg[b];
    }
    std::vector<int> ldeg(n, 0);
    for (int tries = 0; tries < n * link_deg * 4; ++tries) {
        const int a = static_cast<int>(rng() % n), b = static_cast<int>(rng() % n);
        if (a == b || ldeg[a] >= link_deg || ldeg[b] >= link_deg || in.ladj[a].count(b)) continue;
        const int K = penalty ? static_cast<int>(rng() % 7) - 3 : 1;
        if (K == 0) continue;
        in.ladj[a][b] = K;
        in.ladj[b][a] = K;
        ++ldeg[a];
        ++ldeg[b];
    }
    in.cp_ptr.assign(n + 1, 0);
    in.lk_ptr.assign(n + 1, 0);
    for (int a = 0; a < n; ++a) {
        for (const auto &e : in.cadj[a]) {
            in.cp_col.push_back(e.first);
            in.cp_J.push_back(static_cast<int16_t>(e.second));
        }
        for (const auto &e : in.ladj[a]) {
            in.lk_col.push_back(e.first);
            in.lk_w.push_back(static_cast<int16_t>(e.second));
        }
        in.cp_ptr[a + 1] = static_cast<int32_t>(in.cp_col.size());
        in.lk_ptr[a + 1] = static_cast<int32_t>(in.lk_col.size());
        in.h.push_back(static_cast<int32_t>(rng() % 201) - 100);
        in.hk.push_back(penalty ? static_cast<int32_t>(rng() % 9) - 4 : 0);
    }
    return in;
}

int fail(const char *what, int p, int k) {
    std::printf("mismatch: %s at position %d entry %d\n", what, p, k);
    return 1;
}

// Decode every record of pp and compare with the instance.
int check(const Inst &in, const pt2d::Prep &pp, bool penalty) {
    const int n = in.n, DC = pp.DC, DL = pp.DL;
    const int scale = pp.pad_ref / n;
    const int ri = pp.rec_vec * 4;
    const int jo = pt2d::wide_jpack_offset(DC, DL);
    for (int p = 0; p < n; ++p) {
        const int32_t *r = pp.rec.data() + static_cast<size_t>(p) * ri;
        const int a = r[DC + DL];
        if (a < 0 || a >= n || pp.pos_of[a] != p) return fail("spin id", p, 0);
        if (r[DC + DL + 1] != 2 * in.h[a]) return fail("2h", p, 0);
        std::map<int, int> got;
        for (int k = 0; k < DC; ++k) {
            if (r[k] % scale) return fail("coupling reference scale", p, k);
            const int row = r[k] / scale;
            int J;
            if (pp.wide) {
                const uint32_t lo = static_cast<uint32_t>(r[jo + 2 * (k / 4)]) >> (8 * (k % 4)) & 0xFFu;
                const uint32_t hi = static_cast<uint32_t>(r[jo + 2 * (k / 4) + 1]) >> (8 * (k % 4)) & 0xFFu;
                J = 256 * static_cast<int8_t>(hi) + static_cast<int>(lo);
            } else {
                if (r[DC + DL + 2 + k] % 2) return fail("2J parity", p, k);
                J = r[DC + DL + 2 + k] / 2;
                if (!pp.pen_kernel && DC == 3 && DL == 2) {  // packed bytes in the two spare ints
                    const uint32_t lo = static_cast<uint32_t>(r[10]) >> (8 * k) & 0xFFu;
                    const uint32_t hi = static_cast<uint32_t>(r[11]) >> (8 * k) & 0xFFu;
                    if (256 * static_cast<int8_t>(hi) + static_cast<int>(lo) != J) return fail("packed J bytes", p, k);
                    if ((static_cast<uint32_t>(r[10]) | static_cast<uint32_t>(r[11])) >> 24)
                        return fail("packed J byte 3", p, k);
                }
            }
            if (row == n) {
                if (J != 0) return fail("padding coupling with J != 0", p, k);
                continue;
            }
            if (row < 0 || row > n || got.count(pp.pid[row])) return fail("coupling reference", p, k);
            got[pp.pid[row]] = J;
        }
        if (got != in.cadj[a]) return fail("coupling set", p, 0);
        const int ko = pp.wide ? jo + DC / 2 : 2 * DC + DL + 2;
        std::map<int, int> links;
        for (int k = 0; k < DL; ++k) {
            if (r[DC + k] % scale) return fail("link reference scale", p, k);
            const int row = r[DC + k] / scale;
            const int K = penalty ? r[ko + k] : 1;
            if (row == n) {
                if (penalty && K != 0) return fail("padding link with K != 0", p, k);
                continue;
            }
            if (row < 0 || row > n || links.count(pp.pid[row])) return fail("link reference", p, k);
            links[pp.pid[row]] = K;
        }
        if (links != in.ladj[a]) return fail("link set", p, 0);
        if (penalty && r[ko + DL] != in.hk[a]) return fail("penalty field", p, 0);
        if (pp.wide && static_cast<int>(pp.rec_vec) * 4 < pt2d::wide_record_ints(DC, DL, penalty))
            return fail("record size", p, 0);
    }
    return 0;
}

}  // namespace

int main() {
    std::mt19937 rng(20260);
    const float beta[2] = {0.1f, 0.3f};
    const int32_t P[2] = {1, 4};
    int cases = 0;
    // (max coupling degree, link degree, penalty terms, force_dc, sweep kernel, expected layout)
    struct Case {
        int max_deg, link_deg;
        bool penalty;
        int force_dc, mode;
        int layout;  // 0 specialised, 1 penalty-specialised, 2 wide
    } cs[] = {
        {3, 2, false, 0, 0, 0},  {6, 2, false, 0, 2, 0},  {4, 2, false, 0, 1, 0},  {3, 2, false, 4, 1, 0},
        {3, 2, true, 0, 0, 1},   {5, 3, true, 0, 0, 1},   {6, 2, true, 0, 2, 1},   {9, 2, false, 0, 0, 2},
        {3, 4, false, 0, 0, 2},  {13, 3, true, 0, 0, 2},  {3, 2, true, 0, 1, 2},   {3, 2, false, -1, 1, 2},
        {21, 5, true, -1, 1, 2}, {1, 1, false, -1, 1, 2}, {7, 0, false, 0, 2, 2},
        {3, 2, true, 0, 3, 1},   {6, 3, true, 0, 3, 1},   {3, 2, false, 0, 3, 0},
    };
    for (const Case &c : cs) {
        for (int rep = 0; rep < 3; ++rep) {
            const int n = 40 + static_cast<int>(rng() % 200);
            Inst in = make(rng, n, c.max_deg, c.link_deg, c.penalty);
            pt2d_instance pi{};
            pi.n = n;
            pi.cp_ptr = in.cp_ptr.data();
            pi.cp_col = in.cp_col.data();
            pi.cp_J = in.cp_J.data();
            pi.lk_ptr = in.lk_ptr.data();
            pi.lk_col = in.lk_col.data();
            pi.h = in.h.data();
            if (c.penalty) {
                pi.lk_w = in.lk_w.data();
                pi.hk = in.hk.data();
                pi.g0 = 3;
            }
            pt2d_options o;
            pt2d_default_options(&o);
            o.sweep_kernel = c.mode;
            pt2d::Prep pp;
            const int st = pt2d::prepare(&pi, 2, beta, 2, P, 3, &o, pp, c.force_dc);
            if (st) {
                std::printf("prepare failed (%d) in case %d\n", st, cases);
                return 1;
            }
            const int layout = pp.wide ? 2 : (pp.pen_kernel ? 1 : 0);
            if (layout != c.layout) {
                std::printf("layout %d, expected %d, in case %d\n", layout, c.layout, cases);
                return 1;
            }
            if (pp.wide && pp.DC % 4) {
                std::printf("wide coupling width %d not a multiple of 4\n", pp.DC);
                return 1;
            }
            if (check(in, pp, c.penalty)) {
                std::printf("in case %d (layout %d, DC %d, DL %d)\n", cases, layout, pp.DC, pp.DL);
                return 1;
            }
        }
        ++cases;
    }
    std::printf("ok %d cases\n", cases);
    return 0;
}
