/*
 * Plain CPU oracle for two-dimensional parallel tempering (2D-PT).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * restatement of the method that the GPU library is checked against.  Only the
 * test suite, the smoke check and the CPU-baseline leg of the benchmark may
 * load it; the product path never does.  It shares no code with the GPU
 * library: every routine below is written from the paper (or, for the random
 * number generator, from its published definition).
 *
 * Must be compiled with -ffp-contract=off and without -ffast-math: every
 * single-precision operation is rounded to nearest-even on its own, which is
 * what makes the results bit-reproducible on another implementation.
 *
 * Definitions followed:
 *  - penalised energy E_j = f + P_j g                       (Eq. 1)
 *  - P-swap acceptance  min(1, exp(beta dP dg))             (Eq. 2)
 *  - beta-swap acceptance min(1, exp(dbeta dE))             (Eq. 3)
 *  - the 2D-PT loop: sweeps, E and g on the final sweep, alternating
 *    odd/even pairs and P/beta directions                   (Algorithm 1)
 *  - copy constraint g = number of broken copy links, equivalent to a
 *    ferromagnetic coupling between copies   (Section "Graph sparsification")
 * Readings where the paper is silent (heat-bath rule, RNG keys, the fixed
 * float sequences) are stated at each function.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#if !defined(FLT_EVAL_METHOD) || FLT_EVAL_METHOD != 0
#error "the oracle needs single-precision evaluation (FLT_EVAL_METHOD == 0)"
#endif

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel Random Numbers: As   */
/* Easy as 1, 2, 3", SC'11).  Ten rounds of the 4x32 S-box; the key is      */
/* bumped by the two Weyl constants (golden ratio, sqrt(3)-1) between        */
/* rounds.                                                                   */
/* ------------------------------------------------------------------------ */
#define ORC_PHILOX_M0 0xD2511F53u
#define ORC_PHILOX_M1 0xCD9E8D57u
#define ORC_PHILOX_W0 0x9E3779B9u
#define ORC_PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod0 = (uint64_t)ORC_PHILOX_M0 * (uint64_t)x0;
        uint64_t prod1 = (uint64_t)ORC_PHILOX_M1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += ORC_PHILOX_W0;
        k1 += ORC_PHILOX_W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Stream tags: the low 4 bits of counter word 3 (the run index fills the rest). */
enum { ORC_TAG_INIT = 0, ORC_TAG_SWEEP = 1, ORC_TAG_SWAP = 2 };

/* One 32-bit word of the keyed stream: key = seed, counter = (c0,c1,c2,
 * (run << 4) | tag), word index `word` in 0..3. */
static uint32_t orc_word(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2,
                         uint32_t run, uint32_t tag, int word)
{
    uint32_t ctr[4] = {c0, c1, c2, (run << 4) | tag};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[word];
}

/* Uniform on the 2^23-point grid of (0,1]: (top 23 bits of the word + 1)
 * times 2^-23, exact.  Never zero, so u * d is never 0 * inf. */
static float orc_uniform(uint32_t r)
{
    return (float)((r >> 9) + 1u) * 0x1p-23f;
}

/* ------------------------------------------------------------------------ */
/* pt_exp: single-precision exponential, written from the textbook method    */
/* (Cody & Waite additive range reduction x = k ln2 + r, |r| <= ln2/2, then  */
/* the degree-7 Taylor polynomial of e^r in Horner form, then scaling by     */
/* 2^k through the exponent field).  Every operation is a separately rounded */
/* float operation.  Constants:                                              */
/*   L2E    = RN(log2 e)                                                     */
/*   LN2_HI = ln 2 rounded to float, then its low 12 significand bits        */
/*            cleared, so k*LN2_HI is exact for |k| < 2^12                    */
/*   LN2_LO = RN(ln 2 - LN2_HI)                                              */
/*   C_n    = RN(1/n!)                                                       */
/* ------------------------------------------------------------------------ */
static const float ORC_L2E = 0x1.715476p+0f;     /* 1.44269502 */
static const float ORC_LN2_HI = 0x1.62ep-1f;     /* 0.693115234 */
static const float ORC_LN2_LO = 0x1.0bfbe8p-15f; /* 3.19461833e-5 */
static const float ORC_C[8] = {
    0x1p+0f,          /* 1/0! */
    0x1p+0f,          /* 1/1! */
    0x1p-1f,          /* 1/2! */
    0x1.555556p-3f,   /* 1/3! */
    0x1.555556p-5f,   /* 1/4! */
    0x1.111112p-7f,   /* 1/5! */
    0x1.6c16c2p-10f,  /* 1/6! */
    0x1.a01a02p-13f,  /* 1/7! */
};

static float orc_pow2i(int m) /* 2^m for -126 <= m <= 127 */
{
    uint32_t bits = (uint32_t)(m + 127) << 23;
    float f;
    memcpy(&f, &bits, sizeof f);
    return f;
}

float orc_pt_exp(float x)
{
    if (x != x) return x;
    if (x > 88.75f) return INFINITY;
    if (x < -104.0f) return 0.0f;
    float kf = rintf(x * ORC_L2E);
    int k = (int)kf;
    float r = (x - kf * ORC_LN2_HI) - kf * ORC_LN2_LO;
    float p = ORC_C[7];
    for (int i = 6; i >= 0; --i) {
        p = p * r;
        p = p + ORC_C[i];
    }
    if (k > 127) return (p * orc_pow2i(k - 64)) * orc_pow2i(64);
    if (k < -126) return (p * orc_pow2i(k + 64)) * orc_pow2i(-64);
    return p * orc_pow2i(k);
}

/* ------------------------------------------------------------------------ */
/* Heat-bath (Gibbs) update.  Algorithm 1 asks for sweeps but leaves the     */
/* single-spin rule open; this is the standard heat bath for                 */
/* E = f + P g: with the local field H = E(s_a=-1) - E(s_a=+1),              */
/* P(s_a = +1) = 1 / (1 + exp(-beta H)).  Fixed float sequence:               */
/*   t = beta * float(H); e = pt_exp(-t); d = 1 + e; v = u * d;              */
/*   new spin = +1 iff v < 1  (the division-free form of u < 1/(1+e)).      */
/* ------------------------------------------------------------------------ */
int orc_heatbath(float beta, int32_t H, uint32_t r)
{
    float Hf = (float)H;
    float t = beta * Hf;
    float e = orc_pt_exp(-t);
    float d = 1.0f + e;
    float v = orc_uniform(r) * d;
    return (v < 1.0f) ? 1 : -1;
}

/* Metropolis swap test "rand <= min(1, exp(x))" (Algorithm 1). */
int orc_swap_accept(float x, uint32_t r)
{
    if (x >= 0.0f) return 1;
    return orc_uniform(r) <= orc_pt_exp(x);
}

/* ------------------------------------------------------------------------ */
/* Physical instance: symmetric coupling CSR (int16 J), symmetric link CSR   */
/* (copy constraints), optional integer field h, and a proper colouring.     */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t n;
    const int32_t *cp_ptr;
    const int32_t *cp_col;
    const int16_t *cp_J;
    const int32_t *lk_ptr;
    const int32_t *lk_col;
    const int32_t *h; /* may be NULL */
    const int32_t *color;
    int32_t n_colors;
    const int16_t *lk_w;  /* penalty weight K of each link entry; NULL = all 1        */
    const int32_t *hk;    /* penalty field k of each spin; NULL = all 0               */
    int64_t g0;           /* constant term of g                                       */
} orc_inst;

/* Ising cost f(s) = -sum_{a<b} J_ab s_a s_b - sum_a h_a s_a  (the "f" of Eq. 1). */
int64_t orc_cost_f(const orc_inst *in, const int8_t *s)
{
    int64_t f = 0;
    for (int32_t a = 0; a < in->n; ++a) {
        for (int32_t k = in->cp_ptr[a]; k < in->cp_ptr[a + 1]; ++k) {
            int32_t b = in->cp_col[k];
            if (b > a) f -= (int64_t)in->cp_J[k] * s[a] * s[b];
        }
        if (in->h) f -= (int64_t)in->h[a] * s[a];
    }
    return f;
}

/* Constraint function g(s) = g0 + sum_{links a<b} K_ab [s_a != s_b] + sum_a k_a [s_a = -1].
 * Copy constraints (K = 1, k = 0, g0 = 0): the number of links with s_a != s_b,
 * i.e. sum (s_a - s_b)^2 / 4; g >= 0 and g = 0 iff all copies agree.  Any
 * quadratic penalty of binary variables (one-hot, slack) has this form. */
int64_t orc_constraint_g(const orc_inst *in, const int8_t *s)
{
    int64_t g = in->g0;
    for (int32_t a = 0; a < in->n; ++a) {
        for (int32_t k = in->lk_ptr[a]; k < in->lk_ptr[a + 1]; ++k) {
            int32_t b = in->lk_col[k];
            if (b > a && s[a] != s[b]) g += in->lk_w ? in->lk_w[k] : 1;
        }
        if (in->hk && s[a] < 0) g += in->hk[a];
    }
    return g;
}

/* H_a = E(s_a=-1) - E(s_a=+1) = 2 sum_b J_ab s_b + 2 h_a + P (sum_{links} K_al s_l + k_a)
 * (g(s_a=-1) - g(s_a=+1) = sum_l K_al s_l + k_a). */
int32_t orc_local_field(const orc_inst *in, const int8_t *s, int32_t a, int32_t P)
{
    int64_t H = 0;
    for (int32_t k = in->cp_ptr[a]; k < in->cp_ptr[a + 1]; ++k)
        H += 2 * (int64_t)in->cp_J[k] * s[in->cp_col[k]];
    if (in->h) H += 2 * (int64_t)in->h[a];
    int64_t L = in->hk ? in->hk[a] : 0;
    for (int32_t k = in->lk_ptr[a]; k < in->lk_ptr[a + 1]; ++k)
        L += (int64_t)(in->lk_w ? in->lk_w[k] : 1) * s[in->lk_col[k]];
    H += (int64_t)P * L;
    return (int32_t)H;
}

/* Initial state S0 (Algorithm 1 input): uniform +-1 from the INIT stream,
 * counter (spin, 0, walker/4, run<<4|INIT), word walker%4; +1 iff r < 2^31. */
void orc_init_walker(const orc_inst *in, uint64_t seed, int32_t run, int32_t walker, int8_t *s)
{
    for (int32_t a = 0; a < in->n; ++a) {
        uint32_t r = orc_word(seed, (uint32_t)a, 0u, (uint32_t)walker >> 2, (uint32_t)run,
                              ORC_TAG_INIT, walker & 3);
        s[a] = (r < 0x80000000u) ? 1 : -1;
    }
}

/* One Monte Carlo sweep of one walker at (beta, P): every spin once, colour
 * class by colour class (spins of one colour share no edge, so their order
 * within the class does not matter; ascending id is used).  The uniform for
 * spin a in global sweep t is word walker%4 of the SWEEP stream at counter
 * (a, t, walker/4, run<<4|SWEEP). */
void orc_sweep_walker(const orc_inst *in, uint64_t seed, int32_t run, int32_t walker,
                      int64_t sweep_index, float beta, int32_t P, int8_t *s)
{
    for (int32_t c = 0; c < in->n_colors; ++c)
        for (int32_t a = 0; a < in->n; ++a) {
            if (in->color[a] != c) continue;
            int32_t H = orc_local_field(in, s, a, P);
            uint32_t r = orc_word(seed, (uint32_t)a, (uint32_t)sweep_index,
                                  (uint32_t)walker >> 2, (uint32_t)run, ORC_TAG_SWEEP, walker & 3);
            s[a] = (int8_t)orc_heatbath(beta, H, r);
        }
}

/* ------------------------------------------------------------------------ */
/* Full 2D-PT (Algorithm 1) for a set of independent runs.                   */
/* ------------------------------------------------------------------------ */
typedef struct {
    int8_t *spins;        /* [n_runs][I*J][n]   state of each walker          */
    int32_t *walker_at;   /* [n_runs][I*J]      slot (i*J+j) -> walker         */
    int64_t *f;           /* [n_runs][I*J]      per walker, final sweep        */
    int64_t *g;           /* [n_runs][I*J]                                     */
    int64_t *counters;    /* [4]: sweeps done, events done, direction, inited  */
    int64_t trace_cap;    /* events kept in the trace                          */
    int64_t *trace_f;     /* [n_runs][trace_cap] bottom-right f after event n  */
    int64_t *trace_g;     /* [n_runs][trace_cap]                               */
    int64_t *best_f;      /* [n_runs] lowest bottom-right f with g == 0        */
    int64_t *best_event;  /* [n_runs] event index of best_f (-1 if none)       */
    int8_t *best_state;   /* [n_runs][n]                                       */
    const int64_t *target;/* [n_runs] or NULL: solved iff g == 0, f <= target  */
    int64_t *solved_event;/* [n_runs] first solving event (-1 if none)         */
    int64_t *acc_P;       /* [n_runs][I*J] accepted P-swaps by lower slot      */
    int64_t *acc_B;       /* [n_runs][I*J] accepted beta-swaps by lower slot   */
    uint32_t *hist;       /* slot-state counts after each event, or NULL:      */
                          /* [n_runs][I*J][2^n] if hist_slot < 0, else         */
                          /* [n_runs][2^n] for slot hist_slot only             */
    int64_t hist_slot;
    int64_t *sum_f;       /* [n_runs][I*J] per slot: sum of f after events     */
    int64_t *sum_g;       /* [n_runs][I*J] per slot: sum of g                   */
    int64_t *n_feasible;  /* [n_runs][I*J] per slot: count of g == 0            */
    int64_t mode;         /* 0: 2D-PT (Algorithm 1); 1: J-column PT baseline    */
} orc_state;

/* The slot an event records.  2D-PT: the bottom-right replica (beta_I, P_J).
 * J-column PT (standard PT repeated over J columns, the paper's comparison
 * baseline, whose best feasible energy is picked among the J columns): the
 * replica of the last row with the lowest g, then the lowest f, then the
 * lowest column. */
static int32_t orc_record_slot(int32_t I, int32_t J, const int32_t *at, const int64_t *fw,
                               const int64_t *gw, int64_t mode)
{
    if (mode == 0) return I * J - 1;
    int32_t best = (I - 1) * J;
    for (int32_t j = 1; j < J; ++j) {
        const int32_t s = (I - 1) * J + j;
        const int64_t g = gw[at[s]], gb = gw[at[best]];
        if (g < gb || (g == gb && fw[at[s]] < fw[at[best]])) best = s;
    }
    return best;
}

static void orc_swap_slots(int32_t *walker_at, int32_t sa, int32_t sb)
{
    int32_t t = walker_at[sa];
    walker_at[sa] = walker_at[sb];
    walker_at[sb] = t;
}

/* One swap event of Algorithm 1 for one run, given f and g of every walker
 * (indexed by walker) after the final sweep.  Event n (1-based) uses the pairs
 * starting at the first replica when n is odd and at the second when n is
 * even; direction +1 swaps along P inside every row (Eq. 2), -1 along beta
 * inside every column (Eq. 3).  `at` maps slot -> walker and is permuted in
 * place; acc_P / acc_B count accepted swaps by the lower slot of the pair. */
void orc_swap_event(int32_t I, const float *beta, int32_t J, const int32_t *P, const int64_t *fw,
                    const int64_t *gw, int32_t *at, uint64_t seed, uint32_t run, int64_t nev,
                    int direction, int64_t *acc_P, int64_t *acc_B)
{
    const int even = (nev % 2 == 0);
    if (direction == 1) {
        /* swaps along P: each row, pairs (p, p+1) for p = even, even+2, ... */
        for (int32_t i = 0; i < I; ++i)
            for (int32_t p = even; p + 1 < J; p += 2) {
                const int32_t sa = i * J + p, sb = i * J + p + 1;
                const int64_t dP = (int64_t)P[p + 1] - (int64_t)P[p];
                const int64_t dg = gw[at[sb]] - gw[at[sa]];
                const float x = beta[i] * (float)(dP * dg);
                const uint32_t r = orc_word(seed, (uint32_t)sa, (uint32_t)nev, 0u, run,
                                            ORC_TAG_SWAP, 0);
                if (orc_swap_accept(x, r)) {
                    orc_swap_slots(at, sa, sb);
                    acc_P[sa] += 1;
                }
            }
    } else {
        /* swaps along beta: each column, pairs (b, b+1) for b = even, even+2, ... */
        for (int32_t j = 0; j < J; ++j)
            for (int32_t b = even; b + 1 < I; b += 2) {
                const int32_t sa = b * J + j, sb = (b + 1) * J + j;
                const float dbeta = beta[b + 1] - beta[b];
                const int64_t Ea = fw[at[sa]] + (int64_t)P[j] * gw[at[sa]];
                const int64_t Eb = fw[at[sb]] + (int64_t)P[j] * gw[at[sb]];
                const float x = dbeta * (float)(Eb - Ea);
                const uint32_t r = orc_word(seed, (uint32_t)sa, (uint32_t)nev, 0u, run,
                                            ORC_TAG_SWAP, 0);
                if (orc_swap_accept(x, r)) {
                    orc_swap_slots(at, sa, sb);
                    acc_B[sa] += 1;
                }
            }
    }
}

int orc_pt2d_run(const orc_inst *in, int32_t I, const float *beta, int32_t J, const int32_t *P,
                 int32_t n_runs, const int32_t *run_ids, uint64_t seed, int64_t sweeps,
                 int32_t interval, orc_state *st)
{
    const int32_t n = in->n;
    const int32_t R = I * J;
    if (interval < 1 || sweeps < 0 || I < 1 || J < 1) return -1;

    if (!st->counters[3]) {
        for (int32_t q = 0; q < n_runs; ++q) {
            for (int32_t w = 0; w < R; ++w) {
                orc_init_walker(in, seed, run_ids[q], w, st->spins + ((int64_t)q * R + w) * n);
                st->walker_at[(int64_t)q * R + w] = w; /* walker w starts at slot w */
            }
            st->best_f[q] = INT64_MAX;
            st->best_event[q] = -1;
            st->solved_event[q] = -1;
        }
        st->counters[0] = 0;
        st->counters[1] = 0;
        st->counters[2] = st->mode ? -1 : 1; /* swap_direction <- 1 (J-column PT: beta-swaps only) */
        st->counters[3] = 1;
    }

    const int64_t n_swap = sweeps / interval; /* N_swap = floor(MCS / MCS_per_swap) */
    for (int64_t e = 0; e < n_swap; ++e) {
        const int64_t nev = st->counters[1] + 1; /* global event index n (1-based) */
        const int even = (nev % 2 == 0);
        const int64_t t0 = st->counters[0];
        for (int32_t q = 0; q < n_runs; ++q) {
            const uint32_t run = (uint32_t)run_ids[q];
            int32_t *at = st->walker_at + (int64_t)q * R;
            int8_t *S = st->spins + (int64_t)q * R * n;
            /* for each replica: MCS_per_swap sweeps, then E and g of the final sweep */
            for (int32_t slot = 0; slot < R; ++slot) {
                const int32_t w = at[slot];
                const int32_t i = slot / J, j = slot % J;
                int8_t *s = S + (int64_t)w * n;
                for (int32_t k = 0; k < interval; ++k)
                    orc_sweep_walker(in, seed, (int32_t)run, w, t0 + k, beta[i], P[j], s);
                st->f[(int64_t)q * R + w] = orc_cost_f(in, s);
                st->g[(int64_t)q * R + w] = orc_constraint_g(in, s);
            }
            const int64_t *fw = st->f + (int64_t)q * R;
            const int64_t *gw = st->g + (int64_t)q * R;
            orc_swap_event(I, beta, J, P, fw, gw, at, seed, run, nev, (int)st->counters[2],
                           st->acc_P + (int64_t)q * R, st->acc_B + (int64_t)q * R);
            /* store spins from the last replica (bottom-right slot; J-column PT: best of the last row) */
            const int32_t wl = at[orc_record_slot(I, J, at, fw, gw, st->mode)];
            const int64_t fl = fw[wl], gl = gw[wl];
            if (st->trace_f && nev - 1 < st->trace_cap) {
                st->trace_f[(int64_t)q * st->trace_cap + nev - 1] = fl;
                st->trace_g[(int64_t)q * st->trace_cap + nev - 1] = gl;
            }
            if (gl == 0 && fl < st->best_f[q]) {
                st->best_f[q] = fl;
                st->best_event[q] = nev;
                memcpy(st->best_state + (int64_t)q * n, S + (int64_t)wl * n, (size_t)n);
            }
            if (st->target && st->solved_event[q] < 0 && gl == 0 && fl <= st->target[q])
                st->solved_event[q] = nev;
            for (int32_t slot = 0; slot < R; ++slot) {
                const int32_t w = at[slot];
                st->sum_f[(int64_t)q * R + slot] += fw[w];
                st->sum_g[(int64_t)q * R + slot] += gw[w];
                st->n_feasible[(int64_t)q * R + slot] += (gw[w] == 0);
                if (st->hist && (st->hist_slot < 0 || st->hist_slot == slot)) {
                    const int8_t *s = S + (int64_t)w * n;
                    uint64_t idx = 0;
                    for (int32_t a = 0; a < n; ++a)
                        if (s[a] > 0) idx |= (uint64_t)1 << a;
                    const int64_t row = st->hist_slot < 0 ? (int64_t)q * R + slot : (int64_t)q;
                    st->hist[row * ((int64_t)1 << n) + (int64_t)idx] += 1;
                }
            }
        }
        st->counters[0] = t0 + interval;
        st->counters[1] = nev;
        if (even && !st->mode) st->counters[2] = -st->counters[2];
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Helpers for pinning the decisions against their closed forms.            */
/* ------------------------------------------------------------------------ */

/* Number of the 2^23 distinct uniforms u = m 2^-23 for which the heat-bath
 * decision gives +1; divided by 2^23 it is the realised P(s = +1). */
int64_t orc_heatbath_count(float beta, int32_t H)
{
    int64_t c = 0;
    for (uint32_t m = 0; m < (1u << 23); ++m)
        c += orc_heatbath(beta, H, m << 9) > 0;
    return c;
}

/* Number of uniforms for which the swap test accepts at exponent x. */
int64_t orc_swap_count(float x)
{
    int64_t c = 0;
    for (uint32_t m = 0; m < (1u << 23); ++m)
        c += orc_swap_accept(x, m << 9);
    return c;
}

/* The float constants pt_exp uses: L2E, LN2_HI, LN2_LO, C_0..C_7. */
void orc_pt_exp_constants(float out[11])
{
    out[0] = ORC_L2E;
    out[1] = ORC_LN2_HI;
    out[2] = ORC_LN2_LO;
    for (int i = 0; i < 8; ++i) out[3 + i] = ORC_C[i];
}

/* Element-wise forms for comparing long input lists with another implementation. */
void orc_pt_exp_array(const float *x, float *y, int64_t count)
{
    for (int64_t i = 0; i < count; ++i) y[i] = orc_pt_exp(x[i]);
}

void orc_heatbath_array(const float *beta, const int32_t *H, const uint32_t *r, int8_t *s,
                        int64_t count)
{
    for (int64_t i = 0; i < count; ++i) s[i] = (int8_t)orc_heatbath(beta[i], H[i], r[i]);
}

void orc_swap_accept_array(const float *x, const uint32_t *r, int8_t *a, int64_t count)
{
    for (int64_t i = 0; i < count; ++i) a[i] = (int8_t)orc_swap_accept(x[i], r[i]);
}

void orc_philox_array(const uint32_t *ctr, const uint32_t *key, uint32_t *out, int64_t count)
{
    for (int64_t i = 0; i < count; ++i) orc_philox4x32_10(ctr + 4 * i, key + 2 * i, out + 4 * i);
}
