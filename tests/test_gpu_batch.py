"""Batched persistent form vs the plain contexts and the oracle (tolerance zero).

Every problem in a batch must follow exactly the trajectory a plain context
with the same instance, ladders, seed and run count follows: spins, slot maps,
f, g, swap counts, traces, best states and counters, whatever the launch
shape, the placement of the spins (shared or global memory), the chunking of
the events into launches, and the other problems sharing the batch.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pt():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2506_14781_gb300 import build as b

    b.build()
    import paper_2506_14781_gb300 as m

    return m


WHATS = ["STATES", "WALKER_AT", "F", "G", "COUNTERS", "TRACE_F", "TRACE_G", "BEST_F", "BEST_EVENT",
         "BEST_STATE", "SOLVED_EVENT", "ACC_P", "ACC_B", "SUM_F", "SUM_G", "N_FEASIBLE", "COLORS"]


def _problem(pt, N, alpha, seed, rule, I, J, runs):
    inst = synth.wishart_planted(N, alpha, seed)
    phys = pt.sparsify(inst.Jq, *rule)
    beta = synth.beta_ladder(I, 0.1, 2.0, inst.scale)
    P = synth.penalty_ladder(J, 0.5, 4.0, 32767)
    return dict(inst=inst, phys=phys, beta=beta, P=P, runs=runs, seed=1000 + seed,
                target=inst.E_planted)


def _plain(pt, pr, sweeps, interval, trace, swap_mode="2d"):
    ctx = pt.PT2D(pr["phys"], pr["beta"], pr["P"], pr["runs"], trace_capacity=trace,
                  swap_mode=swap_mode)
    ctx.write(pt.TARGET, np.full(pr["runs"], pr["target"], np.int64))
    ctx.run(sweeps, interval, pr["seed"])
    return ctx


def _assert_same(pt, batch, bid, ctx):
    for w in WHATS:
        a = batch.read(bid, getattr(pt, w))
        b = ctx.read(getattr(pt, w))
        if not np.array_equal(a, b):
            bad = np.argwhere(a != b)
            raise AssertionError(f"{w} differs at {bad[:5].tolist()} ({len(bad)} entries)")


def _mixed(pt):
    return [
        _problem(pt, 12, 0.5, 1, ("max_degree", 4), 4, 4, 2),     # R = 16
        _problem(pt, 30, 0.25, 2, ("max_degree", 4), 5, 3, 1),    # R = 15 (ragged)
        _problem(pt, 57, 0.75, 3, ("max_degree", 4), 16, 8, 1),   # R = 128, n ~ 1.5k
        _problem(pt, 90, 0.5, 4, ("max_degree", 4), 12, 8, 1),    # R = 96 (padded to 128)
        _problem(pt, 40, 0.5, 5, ("max_edges", 3), 8, 8, 3),      # R = 64
        _problem(pt, 160, 0.5, 6, ("max_degree", 4), 16, 8, 1),   # n ~ 12.6k: global memory
    ]


@pytest.mark.parametrize("kernel,threads", [("auto", 0), ("global", 0), ("auto", 256),
                                            ("bits", 0), ("bits", 128), ("smem", 512)])
def test_batch_matches_plain_contexts(pt, kernel, threads):
    probs = _mixed(pt)
    trace = 16
    batch = pt.Batch(1 << 30, max_coupling_degree=3, max_runs=64, trace_capacity=trace,
                     threads_per_cta=threads, sweep_kernel=kernel)
    ids = [batch.add(p["phys"], p["beta"], p["P"], p["runs"], p["seed"], p["target"]) for p in probs]
    # 7 events of 5 sweeps, in three launches
    batch.run(2, 5)
    batch.run(4, 5)
    batch.run(1, 5)
    for pr, bid in zip(probs, ids):
        ctx = _plain(pt, pr, 35, 5, trace)
        _assert_same(pt, batch, bid, ctx)
        ctx.close()
    batch.close()


def test_batch_slab_storage_by_size(pt):
    """Runs whose int8 slab of 8 walkers does not fit in shared memory go to
    bit-packed slabs (widths 8 and 32 walkers), next to int8 shared-memory slabs
    of 8, 16 and 128 walkers, in one launch; each matches its plain context."""
    probs = [
        _problem(pt, 600, 0.5, 31, ("max_edges", 3), 16, 8, 1),   # n ~ 120k: bits, 8 walkers
        _problem(pt, 300, 0.5, 32, ("max_edges", 3), 16, 8, 1),   # n ~ 30k: bits, 32 walkers
        _problem(pt, 240, 0.5, 35, ("max_edges", 3), 16, 8, 1),   # n ~ 19k: int8, 8 walkers
        _problem(pt, 150, 0.5, 33, ("max_edges", 3), 16, 8, 2),   # n ~ 7.5k: int8, 16 walkers
        _problem(pt, 40, 0.5, 34, ("max_edges", 3), 4, 8, 1),     # int8, whole run
    ]
    assert probs[0]["phys"].n > 110000
    batch = pt.Batch(1 << 28, max_coupling_degree=3, max_runs=16, trace_capacity=8)
    ids = [batch.add(p["phys"], p["beta"], p["P"], p["runs"], p["seed"], p["target"]) for p in probs]
    batch.run(3, 4)
    batch.run(2, 4)
    for pr, bid in zip(probs, ids):
        ctx = _plain(pt, pr, 20, 4, 8)
        _assert_same(pt, batch, bid, ctx)
        ctx.close()
    batch.close()


def test_batch_shape_changes_between_launches(pt):
    """Switching storage, slab widths, balance and threads between launches
    leaves every trajectory unchanged."""
    probs = _mixed(pt)[:5]
    batch = pt.Batch(1 << 29, max_coupling_degree=3, max_runs=64, trace_capacity=8)
    ids = [batch.add(p["phys"], p["beta"], p["P"], p["runs"], p["seed"], p["target"]) for p in probs]
    shapes = [dict(storage="global", global_width=16, balance=0, threads_per_cta=256),
              dict(storage="bits", balance=64, threads_per_cta=1024),
              dict(storage="smem", balance=1, threads_per_cta=640),
              dict(storage="auto", global_width=128, balance=8, threads_per_cta=128)]
    for sh in shapes:
        batch.shape = sh
        assert all(batch.shape[k] == v for k, v in sh.items())
        batch.run(2, 3)
    with pytest.raises(pt.Pt2dError):
        batch.shape = dict(global_width=24)
    for pr, bid in zip(probs, ids):
        ctx = _plain(pt, pr, 24, 3, 8)
        _assert_same(pt, batch, bid, ctx)
        ctx.close()
    batch.close()


@pytest.mark.parametrize("kernel", ["auto", "global"])
def test_batch_jcolumn_baseline_matches_plain(pt, kernel):
    probs = _mixed(pt)[:5]
    batch = pt.Batch(1 << 29, max_coupling_degree=3, max_runs=64, trace_capacity=16,
                     sweep_kernel=kernel, swap_mode="jcolumn")
    ids = [batch.add(p["phys"], p["beta"], p["P"], p["runs"], p["seed"], p["target"]) for p in probs]
    batch.run(3, 5)
    batch.run(4, 5)
    for pr, bid in zip(probs, ids):
        ctx = _plain(pt, pr, 35, 5, 16, swap_mode="jcolumn")
        _assert_same(pt, batch, bid, ctx)
        assert batch.read(bid, pt.ACC_P).sum() == 0
        ctx.close()
    batch.close()


def test_batch_add_remove_between_launches(pt):
    a = _problem(pt, 20, 0.5, 11, ("max_degree", 4), 4, 4, 1)
    b = _problem(pt, 45, 0.75, 12, ("max_degree", 4), 8, 4, 2)
    c = _problem(pt, 33, 0.25, 13, ("max_degree", 4), 6, 5, 1)
    batch = pt.Batch(1 << 28, max_coupling_degree=3, trace_capacity=8)
    ia = batch.add(a["phys"], a["beta"], a["P"], a["runs"], a["seed"], a["target"])
    ib = batch.add(b["phys"], b["beta"], b["P"], b["runs"], b["seed"], b["target"])
    batch.run(3, 4)
    batch.remove(ia)
    ic = batch.add(c["phys"], c["beta"], c["P"], c["runs"], c["seed"], c["target"])
    batch.run(4, 4)
    _assert_same(pt, batch, ib, _plain(pt, b, 28, 4, 8))
    _assert_same(pt, batch, ic, _plain(pt, c, 16, 4, 8))


def test_batch_pool_full_and_autotune(pt):
    a = _problem(pt, 60, 0.5, 21, ("max_degree", 4), 16, 8, 1)
    probe = pt.Batch(1 << 26, max_coupling_degree=3, trace_capacity=4)
    need = probe.instance_bytes(a["phys"], 16, 8, 1)
    probe.close()
    assert need > 0
    batch = pt.Batch(2 * need + need // 2, max_coupling_degree=3, trace_capacity=4)
    i1 = batch.add(a["phys"], a["beta"], a["P"], 1, a["seed"], a["target"])
    i2 = batch.add(a["phys"], a["beta"], a["P"], 1, a["seed"] + 1, a["target"])
    with pytest.raises(pt.PoolFull):
        batch.add(a["phys"], a["beta"], a["P"], 1, a["seed"] + 2, a["target"])
    shape = batch.autotune(2, 3)  # every trial launch advances the chains
    assert shape["threads_per_cta"] in (128, 256, 512, 1024) and shape == batch.shape
    batch.run(2, 3)
    sweeps = int(batch.read(i1, pt.COUNTERS)[0])
    assert sweeps % 6 == 0 and sweeps >= 5 * 2 * 3
    _assert_same(pt, batch, i1, _plain(pt, a, sweeps, 3, 4))
    a2 = dict(a, seed=a["seed"] + 1)
    _assert_same(pt, batch, i2, _plain(pt, a2, sweeps, 3, 4))


def test_batch_matches_oracle_on_tiny_config(pt, tiny_config):
    cfg = tiny_config
    phys_p = pt.sparsify(cfg["inst"].Jq, "fixed", 2)
    batch = pt.Batch(1 << 24, max_coupling_degree=6, trace_capacity=64)
    bid = batch.add(phys_p, cfg["beta"], cfg["P"], 2, 7, cfg["inst"].E_planted)
    batch.run(50, 2)
    orc = oracle.OracleRun(oracle.OracleInstance(oracle.sparsify(cfg["inst"].Jq, "fixed", 2)),
                           cfg["beta"], cfg["P"], [0, 1], 7, trace_cap=64,
                           target=cfg["inst"].E_planted)
    orc.run(100, 2)
    for w, attr in (("STATES", "spins"), ("WALKER_AT", "walker_at"), ("F", "f"), ("G", "g"),
                    ("TRACE_F", "trace_f"), ("TRACE_G", "trace_g"), ("BEST_F", "best_f"),
                    ("BEST_STATE", "best_state"), ("ACC_P", "acc_P"), ("ACC_B", "acc_B"),
                    ("SUM_F", "sum_f"), ("N_FEASIBLE", "n_feasible")):
        assert np.array_equal(batch.read(bid, getattr(pt, w)), getattr(orc, attr)), w


def test_full_size_uneven_batch_sampled_runs(pt):
    """The 1024-instance uneven workload at full size in the benchmark's launch
    configuration (default shape, one event of 50 sweeps): the smallest, a
    middle and the largest instance are checked in full against the oracle."""
    I, J, interval = 16, 8, 50
    specs = synth.batch_specs(1024, 1000)
    probs = []
    for N, alpha, seed in specs:
        inst = synth.wishart_planted(N, alpha, seed)
        probs.append((inst, pt.sparsify(inst.Jq, "max_degree", 4),
                      synth.beta_ladder(I, 0.1, 5.0, inst.scale), synth.penalty_ladder(J, 0.5, 64.0, 32767),
                      seed))
    probe = pt.Batch(1 << 22, 3, 8, trace_capacity=4)
    need = sum(probe.instance_bytes(p[1], I, J, 1) for p in probs)
    probe.close()
    batch = pt.Batch(int(need * 1.02) + (64 << 20), 3, len(probs), trace_capacity=4)
    ids = [batch.add(p[1], p[2], p[3], 1, p[4], p[0].E_planted) for p in probs]
    batch.run(1, interval)
    order = np.argsort([p[1].n for p in probs])
    for k in (order[0], order[len(order) // 2], order[-1]):
        inst, phys, beta, P, seed = probs[k]
        orc = oracle.OracleRun(oracle.OracleInstance(oracle.sparsify(inst.Jq, "max_degree", 4)), beta, P,
                               [0], seed, trace_cap=4, target=inst.E_planted)
        orc.run(interval, interval)
        for w, attr in (("STATES", "spins"), ("WALKER_AT", "walker_at"), ("F", "f"), ("G", "g"),
                        ("TRACE_F", "trace_f"), ("TRACE_G", "trace_g"), ("BEST_F", "best_f"),
                        ("ACC_P", "acc_P"), ("ACC_B", "acc_B"), ("SUM_F", "sum_f")):
            assert np.array_equal(batch.read(ids[k], getattr(pt, w)), getattr(orc, attr)), (k, w)
    batch.close()


def _penalty_problem(pt, n, groups, seed, I, J):
    """A one-hot constrained problem (general penalty terms) with random couplings."""
    rng = np.random.default_rng(seed)
    A = np.zeros((n, n), np.int16)
    for a in range(n):
        for b in range(a + 1, n):
            if rng.random() < 0.3:
                A[a, b] = A[b, a] = rng.integers(-300, 301)
    cp_ptr = np.concatenate([[0], np.cumsum((A != 0).sum(1))]).astype(np.int32)
    cp_col = np.concatenate([np.nonzero(A[a])[0] for a in range(n)]).astype(np.int32)
    cp_J = np.concatenate([A[a][A[a] != 0] for a in range(n)]).astype(np.int16)
    lk_ptr, lk_col, lk_w, hk, g0 = pt.onehot_penalty(n, groups)
    phys = pt.PhysicalInstance(n, cp_ptr, cp_col, cp_J, lk_ptr, lk_col, h=rng.integers(-50, 51, n).astype(np.int32),
                               lk_w=lk_w, hk=hk, g0=g0)
    beta = np.geomspace(2e-4, 4e-3, I).astype(np.float32)
    P = np.linspace(40, 400, J).astype(np.int32)
    return dict(phys=phys, beta=beta, P=P, runs=1, seed=seed, target=-10 ** 6)


@pytest.mark.parametrize("kernel,threads", [("auto", 0), ("global", 0), ("bits", 0), ("auto", 128)])
def test_runtime_degree_batch_matches_plain(pt, kernel, threads):
    """A batch declared with a coupling degree above 6 runs every problem on the
    runtime-degree kernel: three copies per node (~N/3 couplings per copy),
    one-hot penalty terms and ordinary <= 3-edge chains together, each equal to
    its plain context (at 128 threads per CTA several CTAs share an SM)."""
    probs = [
        _problem(pt, 30, 0.75, 41, ("fixed", 3), 8, 4, 2),
        _problem(pt, 45, 0.5, 42, ("fixed", 3), 16, 8, 1),
        _problem(pt, 60, 0.5, 43, ("max_edges", 3), 8, 8, 1),
        _penalty_problem(pt, 40, [list(range(k, k + 5)) for k in range(0, 40, 5)], 44, 8, 4),
        _penalty_problem(pt, 24, [[0, 1, 2], [3, 4, 5], [2, 6, 9, 12]], 45, 4, 4),
    ]
    batch = pt.Batch(1 << 28, max_coupling_degree=64, max_runs=16, trace_capacity=16, sweep_kernel=kernel,
                     threads_per_cta=threads)
    ids = [batch.add(p["phys"], p["beta"], p["P"], p["runs"], p["seed"], p["target"]) for p in probs]
    batch.run(3, 5)
    batch.run(4, 5)
    for pr, bid in zip(probs, ids):
        ctx = _plain(pt, pr, 35, 5, 16)
        _assert_same(pt, batch, bid, ctx)
        ctx.close()
    batch.close()


def _colouring_problem(pt, V, k, seed, capacity, I, J):
    """k-colouring of a random cubic graph: one-hot groups plus per-colour
    capacity inequalities through slack spins (library expansion)."""
    prob = synth.colouring(V, k, seed, w_max=2)
    n = prob.n
    cons = [(g, [1] * len(g), 1) for g in prob.groups]
    sl = synth.slack_coefficients(capacity)
    for c in range(k):
        cons.append(([v * k + c for v in range(V)] + list(range(n, n + len(sl))), [1] * V + sl, capacity))
        n += len(sl)
    pad = n - prob.n
    lk_ptr, lk_col, lk_w, hk, g0 = pt.equality_penalty(n, cons)
    phys = pt.PhysicalInstance(n, np.concatenate([prob.cp_ptr, np.full(pad, prob.cp_ptr[-1], np.int32)]),
                               prob.cp_col, prob.cp_J, lk_ptr, lk_col,
                               h=np.concatenate([prob.h, np.zeros(pad, np.int32)]), lk_w=lk_w, hk=hk, g0=g0)
    beta = np.geomspace(0.02, 1.5, I).astype(np.float32)
    P = np.linspace(1, 10, J).astype(np.int32)
    return dict(phys=phys, beta=beta, P=P, runs=1, seed=seed, target=prob.f_proper)


@pytest.mark.parametrize("kernel", ["auto", "global"])
def test_runtime_degree_batch_runs_equality_constraints(pt, kernel):
    """Colouring problems with one-hot and slack-encoded capacity constraints
    (link degree ~V/k) in the runtime-degree batch, each equal to its plain
    context."""
    probs = [_colouring_problem(pt, 18, 3, 51, 7, 8, 4), _colouring_problem(pt, 30, 4, 52, 9, 4, 4)]
    batch = pt.Batch(1 << 28, max_coupling_degree=64, max_runs=8, trace_capacity=16, sweep_kernel=kernel)
    ids = [batch.add(p["phys"], p["beta"], p["P"], p["runs"], p["seed"], p["target"]) for p in probs]
    batch.run(5, 6)
    for pr, bid in zip(probs, ids):
        ctx = _plain(pt, pr, 30, 6, 16)
        _assert_same(pt, batch, bid, ctx)
        ctx.close()
    batch.close()


def test_runtime_degree_server_takes_penalty_requests(pt):
    pr = _penalty_problem(pt, 30, [list(range(k, k + 3)) for k in range(0, 30, 3)], 46, 8, 4)
    srv = pt.Server(1 << 26, 64, 8, 5, 4)
    rid = srv.submit(pr["phys"], pr["beta"], pr["P"], pr["seed"], pr["target"], 60)
    for _ in range(100):
        srv.step()
        if srv.status(rid)["state"] == "done":
            break
    got = srv.status(rid, with_state=True)
    assert got["state"] == "done" and got["sweeps_done"] == 60
    ctx = _plain(pt, dict(pr, runs=1), 60, 5, 4)
    assert ctx.read(pt.BEST_F)[0] == got["best_f"]
    assert ctx.read(pt.BEST_EVENT)[0] == got["best_event"]
    if got["best_event"] >= 0:
        assert np.array_equal(ctx.read(pt.BEST_STATE)[0], got["best_state"])
    ctx.close()
    srv.close()


def test_runtime_degree_batch_penalty_problem_matches_oracle(pt):
    """A problem with general penalty terms (one-hot groups, expanded by the
    oracle's own code) in the runtime-degree batch, next to a three-copy
    problem: the batch's record equals the oracle's for the same seed."""
    from oracle.penalties import onehot

    groups = [list(range(k, k + 5)) for k in range(0, 40, 5)]
    pr = _penalty_problem(pt, 40, groups, 44, 8, 4)
    other = _problem(pt, 45, 0.5, 42, ("fixed", 3), 16, 8, 1)
    batch = pt.Batch(1 << 28, max_coupling_degree=64, max_runs=8, trace_capacity=16)
    bid = batch.add(pr["phys"], pr["beta"], pr["P"], 1, pr["seed"], pr["target"])
    batch.add(other["phys"], other["beta"], other["P"], 1, other["seed"], other["target"])
    batch.run(6, 5)
    ph = pr["phys"]
    p2, c2, w2, k2, g2 = onehot(ph.n, groups)
    phys_o = oracle.PhysInstance(ph.n, ph.cp_ptr, ph.cp_col, ph.cp_J, p2, c2, ph.h, ph.n,
                                 np.arange(ph.n, dtype=np.int32), np.arange(ph.n + 1, dtype=np.int32),
                                 lk_w=w2, hk=k2, g0=g2)
    orc = oracle.OracleRun(oracle.OracleInstance(phys_o), pr["beta"], pr["P"], [0], pr["seed"], trace_cap=16,
                           target=pr["target"])
    orc.run(30, 5)
    for w, attr in (("STATES", "spins"), ("WALKER_AT", "walker_at"), ("F", "f"), ("G", "g"),
                    ("TRACE_F", "trace_f"), ("TRACE_G", "trace_g"), ("BEST_F", "best_f"),
                    ("BEST_STATE", "best_state"), ("SOLVED_EVENT", "solved_event"), ("ACC_P", "acc_P"),
                    ("ACC_B", "acc_B"), ("SUM_F", "sum_f"), ("SUM_G", "sum_g")):
        assert np.array_equal(batch.read(bid, getattr(pt, w)), getattr(orc, attr)), w
    batch.close()
