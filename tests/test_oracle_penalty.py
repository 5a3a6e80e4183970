"""Pins of the oracle's general constraint functions (penalty terms).

Eq. 1 allows any constraint function g >= 0.  One-hot groups are expanded into
link weights K, penalty fields k and a constant g0; the oracle evaluates that
form.  Pinned here against the definition g = sum_c (sum_{a in c} x_a - 1)^2
itself (brute force over every state), the local field against E(s_a = -1) -
E(s_a = +1) with E = f + P g, and 2D-PT sampling against the exact Boltzmann
distribution of f + P g.  The library's expansion must equal the oracle's.
"""
import itertools

import numpy as np
import pytest

import oracle
from oracle.penalties import onehot
from oracle.sparsify import PhysInstance


def _instance(n, groups, seed, h=True):
    rng = np.random.default_rng(seed)
    A = np.zeros((n, n), np.int16)
    for a in range(n):
        for b in range(a + 1, n):
            if rng.random() < 0.5:
                A[a, b] = A[b, a] = rng.integers(-5, 6)
    cp_ptr = np.concatenate([[0], np.cumsum((A != 0).sum(1))]).astype(np.int32)
    cp_col = np.concatenate([np.nonzero(A[a])[0] for a in range(n)]).astype(np.int32)
    cp_J = np.concatenate([A[a][A[a] != 0] for a in range(n)]).astype(np.int16)
    lk_ptr, lk_col, lk_w, hk, g0 = onehot(n, groups)
    hf = rng.integers(-3, 4, n).astype(np.int32) if h else None
    return PhysInstance(n, cp_ptr, cp_col, cp_J, lk_ptr, lk_col, hf, n, np.arange(n, dtype=np.int32),
                        np.arange(n + 1, dtype=np.int32), lk_w=lk_w, hk=hk, g0=g0)


def _g_definition(S, groups):
    x = (S > 0).astype(np.int64)
    return sum((x[:, list(c)].sum(1) - 1) ** 2 for c in groups)


def _f_definition(inst, S):
    S64 = S.astype(np.int64)
    f = np.zeros(S.shape[0], np.int64)
    for a in range(inst.n):
        for k in range(inst.cp_ptr[a], inst.cp_ptr[a + 1]):
            b = int(inst.cp_col[k])
            if b > a:
                f -= int(inst.cp_J[k]) * S64[:, a] * S64[:, b]
        if inst.h is not None:
            f -= int(inst.h[a]) * S64[:, a]
    return f


def _all_states(n):
    return np.array(list(itertools.product([1, -1], repeat=n)), dtype=np.int8)


GROUPS = [[0, 1, 2, 3], [4, 5, 6], [7, 8], [2, 9, 10, 11, 5]]  # overlapping groups included


def test_expanded_g_equals_the_definition_on_every_state():
    inst = _instance(12, GROUPS, 1)
    oi = oracle.OracleInstance(inst)
    S = _all_states(12)
    g_def = _g_definition(S, GROUPS)
    g_orc = np.array([oi.constraint_g(s) for s in S])
    assert np.array_equal(g_orc, g_def)
    assert g_def.min() == 0 and (g_def == 0).sum() > 0


def test_local_field_is_the_energy_difference_with_penalties():
    inst = _instance(12, GROUPS, 2)
    oi = oracle.OracleInstance(inst)
    rng = np.random.default_rng(5)
    for _ in range(200):
        s = rng.choice(np.array([-1, 1], np.int8), 12)
        a = int(rng.integers(12))
        P = int(rng.integers(0, 50))
        up, down = s.copy(), s.copy()
        up[a], down[a] = 1, -1
        E = lambda t: _f_definition(inst, t[None])[0] + P * _g_definition(t[None], GROUPS)[0]
        assert oi.local_field(s, a, P) == E(down) - E(up)


def test_copy_links_are_the_unit_weight_case():
    """K = 1, k = 0, g0 = 0 gives the copy constraint's broken-link count."""
    inst = oracle.sparsify(np.array([[0, 3, -2], [3, 0, 1], [-2, 1, 0]], np.int16), "fixed", 2)
    w = PhysInstance(inst.n, inst.cp_ptr, inst.cp_col, inst.cp_J, inst.lk_ptr, inst.lk_col, None,
                     inst.N, inst.copy_of, inst.offset, lk_w=np.ones(inst.lk_col.size, np.int16),
                     hk=np.zeros(inst.n, np.int32), g0=0)
    a, b = oracle.OracleInstance(inst), oracle.OracleInstance(w)
    for s in _all_states(inst.n):
        assert a.constraint_g(s) == b.constraint_g(s)
        for k in range(inst.n):
            assert a.local_field(s, k, 7) == b.local_field(s, k, 7)


def test_sampling_with_penalties_is_stationary():
    groups = [[0, 1, 2, 3], [4, 5, 6, 7]]
    inst = _instance(8, groups, 3)
    S = _all_states(8)
    f = _f_definition(inst, S)
    g = _g_definition(S, groups)
    beta = np.array([0.05, 0.15, 0.4], np.float32)
    P = np.array([1, 4, 10], np.int32)
    runs = 24
    run = oracle.OracleRun(oracle.OracleInstance(inst), beta, P, list(range(runs)), seed=8)
    run.run(300, 1)
    for arr in (run.sum_f, run.sum_g, run.n_feasible):
        arr[...] = 0
    run.run(3000, 1)
    T = 3000
    zmax = 0.0
    for i, b in enumerate(beta):
        for j, p in enumerate(P):
            E = f + int(p) * g
            w = np.exp(-float(b) * (E - E.min()))
            pi = w / w.sum()
            s = i * len(P) + j
            for per_run, ex in ((run.sum_f[:, s] / T, pi @ f), (run.sum_g[:, s] / T, pi @ g),
                                (run.n_feasible[:, s] / T, pi[g == 0].sum())):
                se = per_run.std(ddof=1) / np.sqrt(runs)
                zmax = max(zmax, abs(per_run.mean() - ex) / max(se, 1e-9 * max(abs(ex), 1.0)))
    assert zmax < 5.0, zmax


def test_library_expansion_equals_the_oracle():
    import paper_2506_14781_gb300 as pt

    for groups, n in ((GROUPS, 12), ([[0, 1], [1, 2], [0, 2]], 3), ([[3, 1, 4, 0]], 6), ([], 4)):
        mine = pt.onehot_penalty(n, groups)
        ref = onehot(n, groups)
        for x, y in zip(mine[:4], ref[:4]):
            assert np.array_equal(x, y)
        assert mine[4] == ref[4]


@pytest.mark.parametrize("old,new", [
    ("L += (int64_t)(in->lk_w ? in->lk_w[k] : 1) * s[in->lk_col[k]];",
     "L += (int64_t)1 * s[in->lk_col[k]];"),                      # weights dropped from the field
    ("int64_t L = in->hk ? in->hk[a] : 0;", "int64_t L = 0;"),      # penalty field dropped
])
def test_planted_penalty_mistake_fails_stationarity(tmp_path, old, new):
    from oracle import _build, core

    src = open(_build.SRC).read()
    assert src.count(old) == 1
    path = _build.compile_variant(src.replace(old, new), str(tmp_path / "liboracle_pen.so"))
    groups = [[0, 1, 2, 3], [4, 5, 6, 7]]
    inst = _instance(8, groups, 3)
    S = _all_states(8)
    f, g = _f_definition(inst, S), _g_definition(S, groups)
    beta = np.array([0.05, 0.15, 0.4], np.float32)
    P = np.array([1, 4, 10], np.int32)
    with core.use_library(path):
        run = oracle.OracleRun(oracle.OracleInstance(inst), beta, P, list(range(8)), seed=8)
        run.run(2000, 1)
    zmax = 0.0
    for i, b in enumerate(beta):
        for j, p in enumerate(P):
            E = f + int(p) * g
            w = np.exp(-float(b) * (E - E.min()))
            pi = w / w.sum()
            s = i * len(P) + j
            per_run = run.sum_g[:, s] / 2000
            se = per_run.std(ddof=1) / np.sqrt(8)
            zmax = max(zmax, abs(per_run.mean() - pi @ g) / max(se, 1e-9))
    assert zmax > 8.0, zmax


# ---- linear equality constraints (one-hot generalised, slack-encoded inequalities) ----
def _residual_definition(S, constraints):
    x = (S > 0).astype(np.int64)
    g = np.zeros(S.shape[0], np.int64)
    for ids, coef, b in constraints:
        g += (x[:, list(ids)] @ np.asarray(coef, np.int64) - int(b)) ** 2
    return g


def _equality_sets():
    import synth

    rng = np.random.default_rng(17)
    sets = [
        (10, [([0, 1, 2, 3], [1, 1, 1, 1], 1)]),                               # one-hot
        (10, [([0, 1, 2, 3], [2, -1, 3, 1], 2), ([3, 4, 5], [1, 1, 1], 0),    # mixed signs, b = 0
              ([1, 6, 7, 8, 9], [-2, 1, 4, -3, 1], -1)]),                      # negative rhs
        (12, [([int(a) for a in rng.choice(12, 6, replace=False)],
               [int(c) for c in rng.integers(-4, 5, 6)], int(rng.integers(-3, 6))) for _ in range(4)]),
    ]
    # inequality 2 x0 + 3 x1 + x2 + 2 x3 <= 4 with slack spins 4.. (coefficients 1, 2, 1)
    sl = synth.slack_coefficients(4)
    ids = [0, 1, 2, 3] + list(range(4, 4 + len(sl)))
    sets.append((4 + len(sl) + 2, [(ids, [2, 3, 1, 2] + sl, 4), ([4 + len(sl), 4 + len(sl) + 1], [1, 1], 1)]))
    return sets


def test_equality_expansion_equals_the_definition_on_every_state():
    """g of the expanded links form equals sum_c (sum A x - b)^2 on all 2^n
    states, for one-hot, mixed-sign, negative right-hand-side, overlapping and
    slack-encoded constraints."""
    from oracle.penalties import equality

    for n, cons in _equality_sets():
        lk_ptr, lk_col, lk_w, hk, g0 = equality(n, cons)
        inst = PhysInstance(n, np.zeros(n + 1, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int16),
                            lk_ptr, lk_col, None, n, np.arange(n, dtype=np.int32),
                            np.arange(n + 1, dtype=np.int32), lk_w=lk_w, hk=hk, g0=g0)
        oi = oracle.OracleInstance(inst)
        S = _all_states(n)
        g_orc = np.array([oi.constraint_g(s) for s in S])
        assert np.array_equal(g_orc, _residual_definition(S, cons)), cons


def test_equality_with_unit_coefficients_is_the_onehot_expansion():
    from oracle.penalties import equality

    for groups, n in ((GROUPS, 12), ([[0, 1], [1, 2], [0, 2]], 3), ([], 4)):
        a = equality(n, [(g, [1] * len(g), 1) for g in groups])
        b = onehot(n, groups)
        for x, y in zip(a[:4], b[:4]):
            assert np.array_equal(x, y)
        assert a[4] == b[4]


def test_slack_coefficients_cover_exactly_zero_to_b():
    import synth

    for b in range(0, 70):
        c = synth.slack_coefficients(b)
        sums = {sum(x * y for x, y in zip(bits, c)) for bits in itertools.product([0, 1], repeat=len(c))}
        assert sums == set(range(b + 1)), (b, c)
        assert len(c) == (b + 1).bit_length() - 1 + (0 if (b + 1) & b == 0 else 1)


def test_library_equality_expansion_equals_the_oracle():
    import paper_2506_14781_gb300 as pt
    from oracle.penalties import equality

    for n, cons in _equality_sets():
        mine = pt.equality_penalty(n, cons)
        ref = equality(n, cons)
        for x, y in zip(mine[:4], ref[:4]):
            assert np.array_equal(x, y)
        assert mine[4] == ref[4]
    # a pair weight outside int16 is refused by both
    big = [([0, 1], [300, 200], 100)]
    with pytest.raises(ValueError):
        equality(2, big)
    with pytest.raises(pt.Pt2dError):
        pt.equality_penalty(2, big)
    # repeated spin inside a constraint
    with pytest.raises(pt.Pt2dError):
        pt.equality_penalty(3, [([0, 1, 0], [1, 1, 1], 1)])


def test_colouring_problem_cost_is_four_times_the_same_colour_weight():
    """The colouring input's Ising cost f equals 4 F - k W (F the weight of
    monochromatic edges) on every feasible state of a small graph, and a
    proper colouring has f = -k W."""
    import synth

    prob = synth.colouring(6, 3, 4, w_max=3)
    deg = np.bincount(prob.edges.ravel(), minlength=prob.V)
    assert np.all(deg == 3)
    inst = PhysInstance(prob.n, prob.cp_ptr, prob.cp_col, prob.cp_J, np.zeros(prob.n + 1, np.int32),
                        np.zeros(0, np.int32), prob.h, prob.n, np.arange(prob.n, dtype=np.int32),
                        np.arange(prob.n + 1, dtype=np.int32))
    for col in itertools.product(range(3), repeat=prob.V):
        s = -np.ones(prob.n, np.int8)
        s[np.arange(prob.V) * 3 + np.array(col)] = 1
        f = _f_definition(inst, s[None])[0]
        F = sum(int(w) for (u, v), w in zip(prob.edges.tolist(), prob.w.tolist()) if col[u] == col[v])
        assert f == 4 * F - 3 * prob.W
        assert prob.same_colour_weight(f) == F


def test_local_field_with_weighted_equality_constraints():
    """With general integer coefficients (link weights other than -1, fields of
    both signs) the oracle's heat-bath field is still E(s_a = -1) - E(s_a = +1)
    for E = f + P g, g the squared residuals."""
    from oracle.penalties import equality

    for n, cons in _equality_sets():
        lk_ptr, lk_col, lk_w, hk, g0 = equality(n, cons)
        rng = np.random.default_rng(n)
        A = np.zeros((n, n), np.int16)
        for a in range(n):
            for b in range(a + 1, n):
                if rng.random() < 0.3:
                    A[a, b] = A[b, a] = rng.integers(-9, 10)
        cp_ptr = np.concatenate([[0], np.cumsum((A != 0).sum(1))]).astype(np.int32)
        cp_col = np.concatenate([np.nonzero(A[a])[0] for a in range(n)]).astype(np.int32)
        cp_J = np.concatenate([A[a][A[a] != 0] for a in range(n)]).astype(np.int16)
        h = rng.integers(-4, 5, n).astype(np.int32)
        inst = PhysInstance(n, cp_ptr, cp_col, cp_J, lk_ptr, lk_col, h, n, np.arange(n, dtype=np.int32),
                            np.arange(n + 1, dtype=np.int32), lk_w=lk_w, hk=hk, g0=g0)
        oi = oracle.OracleInstance(inst)
        for _ in range(100):
            s = rng.choice(np.array([-1, 1], np.int8), n)
            a = int(rng.integers(n))
            P = int(rng.integers(0, 30))
            up, down = s.copy(), s.copy()
            up[a], down[a] = 1, -1
            E = lambda t: _f_definition(inst, t[None])[0] + P * _residual_definition(t[None], cons)[0]
            assert oi.local_field(s, a, P) == E(down) - E(up)
