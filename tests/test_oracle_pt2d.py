"""Pins of the oracle's 2D-PT loop (Algorithm 1, Eqs. 1-3).

* Stationarity: at the tiny configuration (20 physical spins, every state
  enumerated) the per-slot means of f, g and of the feasible indicator agree
  with the exact Boltzmann values at (beta_i, P_j) (Appendix A: swaps that obey
  detailed balance keep each slot at its own Boltzmann distribution).
* KL decay: the empirical distribution of the last replica converges to the
  target with D_KL ~ O(1/t) (Fig. 2c, Appendix B); without P-swaps the
  high-penalty replica mixes far more slowly (Fig. 2c).
* Event order of Algorithm 1 (odd/even pairs, P then beta) from the golden
  facts file; resume invariance run(a); run(b) == run(a+b).
* Planted mistakes: copies of the oracle with a flipped swap sign, a flipped
  heat-bath field, a flipped beta difference or a dropped copy-link term are
  compiled and must fail the stationarity pin.
"""
import json
import os

import numpy as np
import pytest

import oracle
import synth
from oracle import _build, boltzmann, core

HERE = os.path.dirname(os.path.abspath(__file__))
FACTS = json.load(open(os.path.join(HERE, "golden", "paper_facts.json")))


def _exact_slot_stats(phys, beta, P):
    S = boltzmann.all_states(phys.n)
    f, g = boltzmann.energies(phys, S)
    out = {}
    for i, b in enumerate(beta):
        for j, p in enumerate(P):
            pi = boltzmann.boltzmann(f, g, float(b), int(p))
            out[(i, j)] = (float(pi @ f), float(pi @ g), float(pi[g == 0].sum()))
    return out


def _stationarity_z(phys, beta, P, runs=24, sweeps=4000, burn_in=500, seed=7, mode=0):
    """Largest |z| over slots of (mean f, mean g, feasible fraction), with the
    standard error taken from the spread over independent runs (after a
    burn-in whose samples are discarded)."""
    oi = oracle.OracleInstance(phys)
    run = oracle.OracleRun(oi, beta, P, list(range(runs)), seed=seed, mode=mode)
    run.run(burn_in, 1)
    for a in (run.sum_f, run.sum_g, run.n_feasible):
        a[...] = 0
    run.run(sweeps, 1)
    T = run.events_done - burn_in
    exact = _exact_slot_stats(phys, beta, P)
    J = len(P)
    zmax = 0.0
    for (i, j), (ef, eg, ep) in exact.items():
        s = i * J + j
        for per_run, ex in ((run.sum_f[:, s] / T, ef), (run.sum_g[:, s] / T, eg),
                            (run.n_feasible[:, s] / T, ep)):
            se = per_run.std(ddof=1) / np.sqrt(runs)
            scale = max(abs(ex), 1.0)
            z = abs(per_run.mean() - ex) / max(se, 1e-9 * scale)
            zmax = max(zmax, z)
    return zmax


def test_stationarity_tiny_config(tiny_config):
    z = _stationarity_z(tiny_config["phys"], tiny_config["beta"], tiny_config["P"])
    assert z < 5.0, z


MUTATIONS = {
    "pswap_sign": ("const int64_t dg = gw[at[sb]] - gw[at[sa]];",
                   "const int64_t dg = gw[at[sa]] - gw[at[sb]];"),
    "heatbath_sign": ("float t = beta * Hf;", "float t = -(beta * Hf);"),
    "bswap_sign": ("const float dbeta = beta[b + 1] - beta[b];",
                   "const float dbeta = beta[b] - beta[b + 1];"),
    "drop_link_field": ("H += (int64_t)P * L;", "H += 0;"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_fails_stationarity(tiny_config, tmp_path, name):
    old, new = MUTATIONS[name]
    src = open(_build.SRC).read()
    assert src.count(old) == 1
    path = _build.compile_variant(src.replace(old, new), str(tmp_path / f"liboracle_{name}.so"))
    with core.use_library(path):
        z = _stationarity_z(tiny_config["phys"], tiny_config["beta"], tiny_config["P"],
                            runs=8, sweeps=2000, burn_in=200)
    assert z > 8.0, (name, z)


def _fig2_instance(seed=3):
    """5-node all-to-all integer instance, two copies per node (Fig. 2a shape;
    the paper's Full Adder coefficients are not given, so couplings are drawn
    from {+-1, +-2, +-3})."""
    rng = np.random.default_rng(seed)
    A = rng.integers(1, 4, size=(5, 5)) * rng.choice([-1, 1], size=(5, 5))
    Jq = np.triu(A, 1)
    Jq = (Jq + Jq.T).astype(np.int16)
    return Jq, oracle.sparsify(Jq, "fixed", 2)


def _logical_kl_curve(Jq, phys, beta, P, checkpoints, seed=11):
    oi = oracle.OracleInstance(phys)
    R = len(beta) * len(P)
    run = oracle.OracleRun(oi, beta, P, [0], seed=seed, hist=True, hist_slot=R - 1)
    fl = boltzmann.logical_energies(Jq)
    p = boltzmann.boltzmann(fl, np.zeros_like(fl), float(beta[-1]), 0)
    # physical index -> logical index through the first copy of each chain
    idx = np.arange(1 << phys.n)
    first = phys.offset[:-1]
    logical_idx = np.zeros_like(idx)
    for i, a in enumerate(first):
        logical_idx |= ((idx >> a) & 1) << i
    S = boltzmann.all_states(phys.n)
    _, g = boltzmann.energies(phys, S)
    feas = g == 0
    out = []
    done = 0
    for t in checkpoints:
        run.run(t - done, 1)
        done = t
        h = run.hist[0].astype(np.float64)
        counts = np.bincount(logical_idx[feas], weights=h[feas], minlength=1 << Jq.shape[0])
        out.append(boltzmann.kl(counts / counts.sum(), p))
    return np.array(out)


def test_kl_decays_like_one_over_t():
    Jq, phys = _fig2_instance()
    beta = np.array([1.0], dtype=np.float32)
    P = np.array([2, 4, 6, 8], dtype=np.int32)
    ts = np.array([2000, 8000, 32000, 128000])
    kl = _logical_kl_curve(Jq, phys, beta, P, ts)
    slope = np.polyfit(np.log(ts), np.log(kl), 1)[0]
    assert -1.4 < slope < -0.6, (slope, kl)
    # Appendix B: for near-independent samples KL * t -> (k-1) tau / 2 with k = 2^5
    k = 2**Jq.shape[0]
    assert kl[-1] * ts[-1] < 20 * (k - 1) / 2


def test_pswaps_speed_up_the_rigid_replica():
    Jq, phys = _fig2_instance()
    beta = np.array([1.0], dtype=np.float32)
    t = [20000]
    kl_swaps = _logical_kl_curve(Jq, phys, beta, np.array([2, 4, 6, 8], dtype=np.int32), t)[0]
    kl_alone = _logical_kl_curve(Jq, phys, beta, np.array([8], dtype=np.int32), t)[0]
    assert kl_alone > 5 * kl_swaps, (kl_alone, kl_swaps)


def test_alg1_event_order(tiny_config):
    phys = tiny_config["phys"]
    oi = oracle.OracleInstance(phys)
    I = J = 4
    beta = np.full(I, 1e-9, dtype=np.float32)  # hot: nearly every swap accepted
    beta = np.cumsum(beta).astype(np.float32)
    P = np.array([1, 2, 3, 4], dtype=np.int32)
    run = oracle.OracleRun(oi, beta, P, [0], seed=3)
    expected = [tuple(e) for e in FACTS["alg1_event_order"]["events"]]
    for kind, parity in expected:
        accP0, accB0 = run.acc_P.copy(), run.acc_B.copy()
        run.run(1, 1)
        dP = (run.acc_P - accP0).reshape(I, J)
        dB = (run.acc_B - accB0).reshape(I, J)
        if kind == "P":
            assert dB.sum() == 0
            cols = np.nonzero(dP.sum(0))[0]
            assert len(cols) > 0 and all(c % 2 == parity and c + 1 < J for c in cols)
        else:
            assert dP.sum() == 0
            rows = np.nonzero(dB.sum(1))[0]
            assert len(rows) > 0 and all(r % 2 == parity and r + 1 < I for r in rows)


def test_resume_is_bit_identical(tiny_config):
    oi = oracle.OracleInstance(tiny_config["phys"])
    args = (tiny_config["beta"], tiny_config["P"], [0, 5], 99)
    a = oracle.OracleRun(oi, *args, trace_cap=200, target=tiny_config["inst"].E_planted)
    a.run(60, 3)
    a.run(90, 3)
    b = oracle.OracleRun(oi, *args, trace_cap=200, target=tiny_config["inst"].E_planted)
    b.run(150, 3)
    for name in ("spins", "walker_at", "f", "g", "counters", "trace_f", "trace_g", "best_f",
                 "best_event", "best_state", "solved_event", "acc_P", "acc_B"):
        assert np.array_equal(getattr(a, name), getattr(b, name)), name


def test_stats_match_definitions(tiny_config):
    phys = tiny_config["phys"]
    oi = oracle.OracleInstance(phys)
    run = oracle.OracleRun(oi, tiny_config["beta"], tiny_config["P"], [2], seed=5)
    run.run(40, 4)
    for w in range(run.R):
        s = run.spins[0, w]
        assert run.f[0, w] == oi.cost_f(s)
        assert run.g[0, w] == oi.constraint_g(s)
    # local field = E(s_a = -1) - E(s_a = +1) at every spin and a few penalties
    rng = np.random.default_rng(1)
    for _ in range(20):
        s = np.where(rng.random(phys.n) < 0.5, -1, 1).astype(np.int8)
        a = int(rng.integers(phys.n))
        for Pj in (0, 7, 131068):
            sp, sm = s.copy(), s.copy()
            sp[a], sm[a] = 1, -1
            Ep = oi.cost_f(sp) + Pj * oi.constraint_g(sp)
            Em = oi.cost_f(sm) + Pj * oi.constraint_g(sm)
            assert oi.local_field(s, a, Pj) == Em - Ep


# ---- J-column PT baseline (mode 1): standard PT in every column --------------------
def test_jcolumn_stationarity(tiny_config):
    """Beta-swaps alone inside each column keep every slot's Boltzmann
    distribution at its (beta_i, P_j)."""
    z = _stationarity_z(tiny_config["phys"], tiny_config["beta"], tiny_config["P"], mode=1)
    assert z < 5.0, z


def test_jcolumn_mistake_fails_stationarity(tiny_config, tmp_path):
    old, new = MUTATIONS["bswap_sign"]
    src = open(_build.SRC).read()
    path = _build.compile_variant(src.replace(old, new), str(tmp_path / "liboracle_jc.so"))
    with core.use_library(path):
        z = _stationarity_z(tiny_config["phys"], tiny_config["beta"], tiny_config["P"],
                            runs=8, sweeps=2000, burn_in=200, mode=1)
    assert z > 8.0, z


def test_jcolumn_invariants_and_record(tiny_config):
    """Replicas never leave their column, no P-swap is ever made, every event
    swaps along beta with alternating pair parity, and each event records the
    last-row replica of lowest (g, f), first column on ties."""
    phys = tiny_config["phys"]
    oi = oracle.OracleInstance(phys)
    I = J = 4
    beta = np.cumsum(np.full(I, 1e-9, dtype=np.float32)).astype(np.float32)  # hot: swaps accepted
    P = np.array([1, 2, 3, 4], dtype=np.int32)
    run = oracle.OracleRun(oi, beta, P, [0, 1], seed=3, trace_cap=64, mode=1)
    for ev in range(1, 41):
        accB0 = run.acc_B.copy()
        run.run(1, 1)
        assert run.counters[2] == -1 and run.acc_P.sum() == 0
        dB = (run.acc_B - accB0).reshape(2, I, J).sum(axis=(0, 2))
        rows = np.nonzero(dB)[0]
        assert len(rows) > 0 and all(r % 2 == (ev + 1) % 2 for r in rows)
        assert np.all(run.walker_at % J == np.arange(I * J) % J)
        for q in range(2):
            last = run.walker_at[q, (I - 1) * J:]
            keys = [(run.g[q, w], run.f[q, w], j) for j, w in enumerate(last)]
            g, f, _ = min(keys)
            assert (run.trace_f[q, ev - 1], run.trace_g[q, ev - 1]) == (f, g)
