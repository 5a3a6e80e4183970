"""Pins of the instance pipeline: planted Wishart generator, copy-chain
sparsifier and greedy colouring.

* Wishart: W^T t = 0, symmetric zero-diagonal J, the closed-form planted cost
  -sum W^2 / (2N), and brute force over all 2^N states (the planted state is a
  ground state of the real couplings; for the quantised ones the brute-force
  minimum is recorded and compared with the planted cost).
* Sparsifier: every logical state lifts to a physical state with g = 0 and the
  same cost, g = 0 physical states are exactly the 2^N lifts, degree caps hold,
  and the text's own counts (Fig. 2a; three-copy chains with 2N constraint
  terms and 600 physical spins at N = 200) are reproduced.
* Colouring: proper, and greedy (every smaller colour is blocked by an earlier
  neighbour).
"""
import json
import os

import numpy as np
import pytest

import oracle
import synth
from oracle import boltzmann

HERE = os.path.dirname(os.path.abspath(__file__))
FACTS = json.load(open(os.path.join(HERE, "golden", "paper_facts.json")))


@pytest.mark.parametrize("N,alpha,seed", [(10, 0.5, 1), (12, 0.25, 3), (16, 0.75, 4)])
def test_wishart_planted_structure(N, alpha, seed):
    inst = synth.wishart_planted(N, alpha, seed)
    t = inst.t.astype(np.float64)
    assert np.abs(inst.W.T @ t).max() < 1e-9
    assert np.array_equal(inst.J, inst.J.T)
    assert np.all(np.diag(inst.J) == 0)
    assert np.array_equal(inst.Jq, inst.Jq.T)
    assert np.abs(inst.Jq).max() == 32767
    # closed form of the real-valued planted cost
    f_t = -0.5 * t @ inst.J @ t
    assert abs(f_t - inst.E_planted_real) < 1e-9 * max(1.0, abs(f_t))
    # brute force on the real couplings: t (and -t) are ground states
    S = boltzmann.all_states(N).astype(np.float64)
    f_all = -0.5 * np.einsum("si,ij,sj->s", S, inst.J, S)
    assert f_all.min() >= inst.E_planted_real - 1e-9
    # quantised couplings: the planted cost is exact and (typically) minimal
    fq = boltzmann.logical_energies(inst.Jq)
    ti = inst.t.astype(np.int64)
    assert -(ti @ np.triu(inst.Jq.astype(np.int64), 1) @ ti) == inst.E_planted
    # quantisation can move the ground state; it can only do so by a small margin
    assert fq.min() <= inst.E_planted
    assert inst.E_planted - fq.min() <= 4 * N * N


def test_tiny_instance_planted_is_ground_state(tiny_config):
    inst = tiny_config["inst"]
    fq = boltzmann.logical_energies(inst.Jq)
    assert fq.min() == inst.E_planted


def test_sparsifier_lift_bijection(tiny_config):
    inst, phys = tiny_config["inst"], tiny_config["phys"]
    assert phys.n == 20 and phys.n_links == 10
    oi = oracle.OracleInstance(phys)
    fl = boltzmann.logical_energies(inst.Jq)
    L = boltzmann.all_states(inst.N)
    for k in range(L.shape[0]):
        s = oracle.lift(phys, L[k])
        assert oi.constraint_g(s) == 0
        assert oi.cost_f(s) == fl[k]
        assert np.array_equal(oracle.project(phys, s), L[k])
    # every g = 0 physical state is a lift: exactly 2^N of the 2^n states
    S = boltzmann.all_states(phys.n)
    f, g = boltzmann.energies(phys, S)
    assert int((g == 0).sum()) == 2**inst.N
    # the enumerating energy routine agrees with the C one on random states
    rng = np.random.default_rng(0)
    for k in rng.integers(0, S.shape[0], 64):
        assert oi.cost_f(S[k]) == f[k] and oi.constraint_g(S[k]) == g[k]


def test_fig2a_two_copies_give_degree_three():
    fact = FACTS["fig2a_sparsification"]
    rng = np.random.default_rng(11)
    N = fact["N_logical"]
    A = rng.integers(1, 4, size=(N, N)) * rng.choice([-1, 1], size=(N, N))
    Jq = np.triu(A, 1)
    Jq = (Jq + Jq.T).astype(np.int16)
    phys = oracle.sparsify(Jq, "fixed", fact["copies_per_node"])
    assert phys.n == fact["n_physical"]
    deg = np.diff(phys.cp_ptr) + np.diff(phys.lk_ptr)
    assert deg.max() == fact["max_physical_degree"]


def test_three_copy_chains_match_text():
    fact = FACTS["three_copy_chains"]
    inst = synth.wishart_planted(30, 0.75, 9)
    phys = oracle.sparsify(inst.Jq, "fixed", fact["copies_per_node"])
    assert phys.n_links == fact["links_per_logical_node"] * inst.N
    assert phys.n == fact["copies_per_node"] * inst.N
    assert fact["example_n_physical"] == fact["copies_per_node"] * fact["example_N"]


def _check_edge_preservation(Jq, phys):
    N = Jq.shape[0]
    seen = {}
    for a in range(phys.n):
        for k in range(phys.cp_ptr[a], phys.cp_ptr[a + 1]):
            b = phys.cp_col[k]
            i, j = int(phys.copy_of[a]), int(phys.copy_of[b])
            assert i != j
            assert phys.cp_J[k] == Jq[i, j]
            if a < b:
                key = (min(i, j), max(i, j))
                assert key not in seen
                seen[key] = True
    expected = {(i, j) for i in range(N) for j in range(i + 1, N) if Jq[i, j] != 0}
    assert set(seen) == expected
    # links only join consecutive copies of one logical node
    for a in range(phys.n):
        for k in range(phys.lk_ptr[a], phys.lk_ptr[a + 1]):
            b = phys.lk_col[k]
            assert phys.copy_of[a] == phys.copy_of[b] and abs(a - b) == 1
    assert phys.n_links == phys.n - N


def test_sparsifier_max_edges_rule():
    inst = synth.wishart_planted(40, 0.5, 2)
    phys = oracle.sparsify(inst.Jq, "max_edges", 3)
    deg_c = np.diff(phys.cp_ptr)
    assert deg_c.max() <= 3
    d = (inst.Jq != 0).sum(1)
    assert phys.n == int(np.ceil(d / 3).sum())
    _check_edge_preservation(inst.Jq, phys)


def test_sparsifier_max_degree_rule():
    inst = synth.wishart_planted(30, 0.25, 6)
    phys = oracle.sparsify(inst.Jq, "max_degree", 4)
    deg = np.diff(phys.cp_ptr) + np.diff(phys.lk_ptr)
    assert deg.max() <= 4
    _check_edge_preservation(inst.Jq, phys)


@pytest.mark.parametrize("rule,param,N", [("fixed", 2, 10), ("max_edges", 3, 40), ("max_degree", 4, 30)])
def test_greedy_colouring(rule, param, N):
    inst = synth.wishart_planted(N, 0.5, 8)
    phys = oracle.sparsify(inst.Jq, rule, param)
    color, C = oracle.greedy_color(phys.n, phys.cp_ptr, phys.cp_col, phys.lk_ptr, phys.lk_col)
    assert oracle.is_proper(color, phys.cp_ptr, phys.cp_col, phys.lk_ptr, phys.lk_col)
    maxdeg = int((np.diff(phys.cp_ptr) + np.diff(phys.lk_ptr)).max())
    assert C <= maxdeg + 1
    # greedy property: each smaller colour is taken by an earlier neighbour
    for a in range(phys.n):
        earlier = set()
        for k in list(range(phys.cp_ptr[a], phys.cp_ptr[a + 1])):
            if phys.cp_col[k] < a:
                earlier.add(int(color[phys.cp_col[k]]))
        for k in list(range(phys.lk_ptr[a], phys.lk_ptr[a + 1])):
            if phys.lk_col[k] < a:
                earlier.add(int(color[phys.lk_col[k]]))
        assert all(c in earlier for c in range(color[a]))
        assert color[a] not in earlier
