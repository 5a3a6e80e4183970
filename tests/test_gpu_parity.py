"""GPU library vs the CPU oracle, through the C ABI.

Tolerance: zero.  Couplings, fields and energies are integers and the float
decisions follow one fixed single-precision sequence on both sides, so spins,
walker <-> slot maps, f, g, swap counts, traces and best states must match
bit for bit.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import core as ocore

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


ARRAYS = [
    ("STATES", "spins"), ("WALKER_AT", "walker_at"), ("F", "f"), ("G", "g"),
    ("TRACE_F", "trace_f"), ("TRACE_G", "trace_g"), ("BEST_F", "best_f"),
    ("BEST_EVENT", "best_event"), ("BEST_STATE", "best_state"), ("SOLVED_EVENT", "solved_event"),
    ("ACC_P", "acc_P"), ("ACC_B", "acc_B"), ("SUM_F", "sum_f"), ("SUM_G", "sum_g"),
    ("N_FEASIBLE", "n_feasible"),
]


def assert_same(pt, ctx, orc, runs_sel=None, trace=True):
    for what, attr in ARRAYS:
        if not trace and what.startswith("TRACE"):
            continue
        got = ctx.read(getattr(pt, what))
        if runs_sel is not None:
            got = got[runs_sel]
        exp = getattr(orc, attr)
        assert got.shape == exp.shape, what
        if not np.array_equal(got, exp):
            bad = np.argwhere(got != exp)
            raise AssertionError(f"{what} differs at {bad[:5].tolist()} ({len(bad)} entries)")
    c = ctx.read(pt.COUNTERS)
    assert list(c) == list(orc.counters), (c, orc.counters)


def both(pt, inst_q, Jrule, beta, P, runs, seed, schedule, *, target=None, trace=64, wpc=0,
         threads=0, phys=None, kernel="auto", wpt=0, swap_mode="2d"):
    if phys is None:
        phys_p = pt.sparsify(inst_q.Jq, *Jrule)
        phys_o = oracle.sparsify(inst_q.Jq, *Jrule)
    else:
        phys_p, phys_o = phys
    ctx = pt.PT2D(phys_p, beta, P, runs, trace_capacity=trace, walkers_per_cta=wpc,
                  threads_per_cta=threads, sweep_kernel=kernel, walkers_per_thread=wpt,
                  swap_mode=swap_mode)
    orc = oracle.OracleRun(oracle.OracleInstance(phys_o), beta, P, list(range(runs)), seed,
                           trace_cap=trace, target=target, mode=pt.SWAP_MODES[swap_mode])
    if target is not None:
        ctx.write(pt.TARGET, np.full(runs, target, np.int64))
    for sweeps, interval in schedule:
        ctx.run(sweeps, interval, seed)
        orc.run(sweeps, interval)
    return ctx, orc


# ---- element-wise device arithmetic -------------------------------------------------
def test_philox_matches_oracle(pt):
    rng = np.random.default_rng(1)
    ctr = rng.integers(0, 2**32, size=(200000, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2**32, size=(200000, 2), dtype=np.uint64).astype(np.uint32)
    assert np.array_equal(pt.diag_philox(ctr, key), ocore.philox_array(ctr, key))


def test_philox_matches_curand(pt, tmp_path):
    """cuRAND's device Philox4_32_10 (a library run on the GPU) gives the same
    blocks as the library's generator at random counters and 64-bit keys, and
    so as the oracle's."""
    import ctypes
    import os
    import subprocess

    src = os.path.join(os.path.dirname(__file__), "_curand_philox.cu")
    lib = str(tmp_path / "libcurand_philox.so")
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared",
                    "-Xcompiler", "-fPIC", src, "-o", lib], check=True, capture_output=True)
    L = ctypes.CDLL(lib)
    L.curand_philox.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_longlong]
    rng = np.random.default_rng(2)
    n = 50000
    ctr = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:, 1] &= 0x3FFFFFFF  # cuRAND's offset is 4 x the low 64 counter bits, a 64-bit value
    key = rng.integers(0, 2**32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    out = np.zeros((n, 4), np.uint32)
    assert L.curand_philox(ctr.ctypes.data, key.ctypes.data, out.ctypes.data, n) == 0
    assert np.array_equal(pt.diag_philox(ctr, key), out)
    assert np.array_equal(ocore.philox_array(ctr[:2000], key[:2000]), out[:2000])


def test_pt_exp_bit_exact_dense(pt):
    lo = np.float32(-104.5).view(np.uint32)  # negative floats: larger bit pattern = more negative
    neg = np.arange(np.uint32(0x80000000), lo + np.uint32(1), 53, dtype=np.uint64).astype(np.uint32)
    pos = np.arange(0, np.float32(89.5).view(np.uint32), 53, dtype=np.uint32)
    x = np.concatenate([neg, pos]).view(np.float32)
    x = np.concatenate([x, np.array([0.0, -0.0, 88.72, 88.75, 88.7228, -103.97, -104.0, -87.3,
                                     np.inf, -np.inf], np.float32)])
    got = pt.diag_pt_exp(x)
    exp = ocore.pt_exp_array(x)
    assert np.array_equal(got.view(np.uint32), exp.view(np.uint32))


def _boundary_cases(rng, count):
    beta = rng.choice(np.array([1.1e-6, 7.3e-6, 3.1e-5, 0.01, 0.5, 2.0], np.float32), count)
    H = rng.integers(-400000, 400001, count).astype(np.int32)
    small = beta >= 0.01
    H[small] = rng.integers(-60, 61, small.sum())
    z = beta.astype(np.float64) * H
    sig = np.where(z >= 0, 1 / (1 + np.exp(-np.minimum(z, 700))), np.exp(np.maximum(z, -700)) /
                   (1 + np.exp(np.maximum(z, -700))))
    m = np.clip(np.floor(sig * 2**23).astype(np.int64) + rng.integers(-3000, 3001, count), 0,
                2**23 - 1)
    r = (m.astype(np.uint64) << np.uint64(9)) | rng.integers(0, 512, count).astype(np.uint64)
    return beta, H, r.astype(np.uint32)


def test_heatbath_matches_oracle(pt):
    rng = np.random.default_rng(2)
    # uniform random triples
    n = 2_000_000
    beta = rng.choice(np.array([0.0, 1e-6, 1e-5, 3e-5, 1e-4, 0.1, 1.0, 30.0], np.float32), n)
    H = rng.integers(-2**23, 2**23, n).astype(np.int32)
    r = rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)
    assert np.array_equal(pt.diag_heatbath(beta, H, r), ocore.heatbath_array(beta, H, r))
    # triples straddling the decision boundary (exercise the exact path)
    beta, H, r = _boundary_cases(rng, 2_000_000)
    assert np.array_equal(pt.diag_heatbath(beta, H, r), ocore.heatbath_array(beta, H, r))
    # u = 0 with saturated exponentials
    H = np.array([-2**23 + 1, 2**23 - 1, -500000, 500000, 0], np.int32)
    for b in (np.float32(1.0), np.float32(1e-4), np.float32(2.1e-5)):
        bb = np.full(H.size, b, np.float32)
        for rv in (0, 1, 511, 512):
            rr = np.full(H.size, rv, np.uint32)
            assert np.array_equal(pt.diag_heatbath(bb, H, rr), ocore.heatbath_array(bb, H, rr))


@pytest.mark.parametrize("beta,H", [(1e-5, 30000), (3.2e-5, -131068), (2.0, 3), (7.3e-6, 0)])
def test_heatbath_exhaustive_over_uniforms(pt, beta, H):
    r = (np.arange(2**23, dtype=np.uint64) << np.uint64(9)).astype(np.uint32)
    b = np.full(r.size, beta, np.float32)
    h = np.full(r.size, H, np.int32)
    got = pt.diag_heatbath(b, h, r)
    assert np.array_equal(got, ocore.heatbath_array(b, h, r))
    assert int((got > 0).sum()) == oracle.heatbath_count(beta, H)


def test_swap_accept_matches_oracle(pt):
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.uniform(-120, 5, 1_000_000), -rng.exponential(1.0, 1_000_000)])
    x = x.astype(np.float32)
    r = rng.integers(0, 2**32, x.size, dtype=np.uint64).astype(np.uint32)
    assert np.array_equal(pt.diag_swap_accept(x, r), ocore.swap_accept_array(x, r))


# ---- whole trajectories ----------------------------------------------------------------
def test_tiny_config_bit_exact_full_length(pt, tiny_config):
    """Tiny configuration as specified: 20 physical spins, I=4 x J=4, swaps every
    sweep, 10^5 sweeps, one run."""
    cfg = tiny_config
    ctx, orc = both(pt, cfg["inst"], ("fixed", 2), cfg["beta"], cfg["P"], 1, 7,
                    [(100000, 1)], target=cfg["inst"].E_planted, trace=1 << 17)
    assert_same(pt, ctx, orc)
    assert orc.best_f[0] == cfg["inst"].E_planted  # the planted ground state is reached


@pytest.mark.parametrize("kernel,wpc,threads,wpt", [
    ("global", 4, 32, 0), ("global", 16, 64, 0), ("global", 32, 256, 0), ("global", 128, 256, 0),
    ("smem", 16, 32, 4), ("smem", 32, 64, 4), ("smem", 64, 1024, 4), ("smem", 128, 128, 4),
    ("smem", 16, 64, 8), ("smem", 64, 512, 8), ("smem", 128, 32, 8), ("smem", 16, 768, 8),
    ("smem", 32, 768, 0), ("bits", 8, 32, 0),
    ("bits", 16, 64, 0), ("bits", 64, 1024, 0), ("bits", 128, 96, 0), ("bits", 8, 64, 4),
    ("bits", 16, 64, 4), ("bits", 64, 512, 8), ("bits", 128, 512, 8), ("bits", 8, 640, 8),
    ("bits", 8, 896, 8), ("bits", 16, 832, 0),
    ("auto", 0, 0, 0)])
def test_ragged_tiles_and_resume(pt, kernel, wpc, threads, wpt):
    inst = synth.wishart_planted(30, 0.5, 21)
    beta = synth.beta_ladder(5, 0.2, 3.0, inst.scale)
    P = synth.penalty_ladder(3, 0.5, 4.0, 32767)
    # R = 15 (not a multiple of 4), 7 runs, interval 7, resumed once, a trailing partial block
    ctx, orc = both(pt, inst, ("max_edges", 3), beta, P, 7, 0xDEADBEEF12345,
                    [(35, 7), (20, 7), (7, 7)], target=inst.E_planted, wpc=wpc, threads=threads,
                    kernel=kernel, wpt=wpt)
    if kernel != "auto":
        assert ctx.tiling["kernel"] == kernel and ctx.tiling["walkers_per_cta"] == wpc
    assert_same(pt, ctx, orc)


@pytest.mark.parametrize("kernel,wpc,threads", [("smem", 16, 64), ("smem", 32, 128), ("smem", 128, 512),
                                                ("bits", 8, 64), ("bits", 16, 96), ("bits", 64, 512)])
def test_eight_walkers_per_thread_across_runs(pt, kernel, wpc, threads):
    """Eight walkers a thread with runs of 5 x 4 = 20 replicas (5 quads): a
    thread's second quad starts the next run at every odd run boundary, and
    must draw that run's random numbers."""
    inst = synth.wishart_planted(24, 0.5, 33)
    beta = synth.beta_ladder(5, 0.2, 3.0, inst.scale)
    P = synth.penalty_ladder(4, 0.5, 4.0, 32767)
    ctx, orc = both(pt, inst, ("max_edges", 3), beta, P, 7, 4321, [(30, 6), (12, 6)],
                    target=inst.E_planted, wpc=wpc, threads=threads, kernel=kernel, wpt=8)
    assert ctx.tiling["walkers_per_thread"] == 8 and ctx.tiling["kernel"] == kernel
    assert_same(pt, ctx, orc)


@pytest.mark.parametrize("kernel,wpt", [("global", 0), ("smem", 4), ("smem", 8), ("bits", 0), ("bits", 4)])
def test_degree_layouts_both_kernels(pt, kernel, wpt):
    """Specialised neighbour layouts DC = 4 and 6 (max-degree and fixed-copy
    sparsifications), on both sweep kernels."""
    for N, rule, seed in ((40, ("max_degree", 4), 3), (12, ("fixed", 2), 5), (13, ("fixed", 3), 6)):
        inst = synth.wishart_planted(N, 0.5, seed)
        beta = synth.beta_ladder(4, 0.2, 2.0, inst.scale)
        P = synth.penalty_ladder(4, 0.5, 4.0, 32767)
        ctx, orc = both(pt, inst, rule, beta, P, 3, 77, [(24, 3)], kernel=kernel,
                        wpc={"smem": 16, "bits": 8}.get(kernel, 0), wpt=wpt)
        assert_same(pt, ctx, orc)


@pytest.mark.parametrize("kernel,wpc", [("auto", 0), ("smem", 16), ("smem", 128), ("global", 0)])
def test_generic_degree_kernel_with_fields(pt, kernel, wpc):
    """Irregular instance with fields and degrees beyond the specialised kernels,
    on the generic kernel with the slab in shared memory and in global memory."""
    rng = np.random.default_rng(9)
    n = 90
    A = np.zeros((n, n), np.int16)
    for a in range(n):
        for b in rng.choice(n, 8, replace=False):
            if b != a:
                v = np.int16(rng.integers(-900, 901))
                A[a, b] = A[b, a] = v
    links = [(a, a + 1) for a in range(0, n - 1, 3)] + [(a, a + 2) for a in range(0, n - 2, 5)]
    L = np.zeros((n, n), bool)
    for a, b in links:
        L[a, b] = L[b, a] = True
    cp_ptr = np.concatenate([[0], np.cumsum((A != 0).sum(1))]).astype(np.int32)
    cp_col = np.concatenate([np.nonzero(A[a])[0] for a in range(n)]).astype(np.int32)
    cp_J = np.concatenate([A[a][A[a] != 0] for a in range(n)]).astype(np.int16)
    lk_ptr = np.concatenate([[0], np.cumsum(L.sum(1))]).astype(np.int32)
    lk_col = np.concatenate([np.nonzero(L[a])[0] for a in range(n)]).astype(np.int32)
    h = rng.integers(-500, 501, n).astype(np.int32)
    phys_p = pt.PhysicalInstance(n, cp_ptr, cp_col, cp_J, lk_ptr, lk_col, h=h)
    phys_o = oracle.PhysInstance(n, cp_ptr, cp_col, cp_J, lk_ptr, lk_col, h, n, np.arange(n),
                                 np.arange(n + 1))
    beta = np.array([1e-4, 4e-4, 1e-3], np.float32)
    P = np.array([0, 300, 900, 2000], np.int32)
    ctx, orc = both(pt, None, None, beta, P, 3, 5, [(24, 4)], phys=(phys_p, phys_o), trace=8,
                    kernel=kernel, wpc=wpc)
    assert ctx.tiling["kernel"] == ("generic" if kernel == "global" else "generic_smem")
    assert ctx.num_colors == orc.oinst.n_colors
    assert np.array_equal(ctx.read(pt.COLORS), orc.oinst.color)
    assert_same(pt, ctx, orc)


def test_single_row_single_column_single_spin(pt):
    inst = synth.wishart_planted(8, 0.5, 4)
    # one row (P-swaps only) and one column (beta-swaps only)
    for beta, P in ((synth.beta_ladder(1, 1.0, 1.0, inst.scale), synth.penalty_ladder(5, 0.5, 4, 32767)),
                    (synth.beta_ladder(6, 0.1, 2.0, inst.scale), synth.penalty_ladder(1, 2, 2, 32767))):
        ctx, orc = both(pt, inst, ("fixed", 2), beta, P, 2, 11, [(40, 2), (3, 2)])
        assert_same(pt, ctx, orc)
    # one spin, no edges, a field
    one_p = pt.PhysicalInstance(1, [0, 0], [], [], [0, 0], [], h=np.array([3], np.int32))
    one_o = oracle.PhysInstance(1, np.array([0, 0], np.int32), np.zeros(0, np.int32),
                                np.zeros(0, np.int16), np.array([0, 0], np.int32),
                                np.zeros(0, np.int32), np.array([3], np.int32), 1,
                                np.zeros(1, np.int32), np.array([0, 1], np.int32))
    ctx, orc = both(pt, None, None, np.array([0.1, 0.3], np.float32), np.array([0, 1], np.int32),
                    3, 2, [(50, 5)], phys=(one_p, one_o))
    assert_same(pt, ctx, orc)


def test_errors_and_empty_runs(pt, tiny_config):
    cfg = tiny_config
    phys = pt.sparsify(cfg["inst"].Jq, "fixed", 2)
    ctx = pt.PT2D(phys, cfg["beta"], cfg["P"], 2)
    with pytest.raises(pt.Pt2dError):
        ctx.read(pt.STATES)  # before the first run
    ctx.run(0, 5, 1)  # no event: only initialisation
    assert list(ctx.read(pt.COUNTERS)) == [0, 0, 1, 1]
    ctx.run(4, 5, 1)  # fewer sweeps than the interval: nothing happens
    assert list(ctx.read(pt.COUNTERS)) == [0, 0, 1, 1]
    with pytest.raises(pt.Pt2dError):
        ctx.run(10, 5, 2)  # another seed
    with pytest.raises(pt.Pt2dError):
        ctx.run(10, 0, 1)
    with pytest.raises(pt.Pt2dError):
        pt.PT2D(phys, cfg["beta"][::-1].copy(), cfg["P"], 1)  # descending ladder


def test_largest_replica_grid(pt, tiny_config):
    """I x J = 8192 slots (the largest grid a run may have; one more is refused),
    swaps on both axes, bit-exact with the oracle."""
    cfg = tiny_config
    beta = synth.beta_ladder(128, 0.05, 3.0, cfg["inst"].scale)
    P = synth.penalty_ladder(64, 0.1, 4.0, 32767)
    ctx, orc = both(pt, cfg["inst"], ("fixed", 2), beta, P, 1, 5, [(24, 2)], trace=16)
    assert_same(pt, ctx, orc)
    with pytest.raises(pt.Pt2dError):
        pt.PT2D(pt.sparsify(cfg["inst"].Jq, "fixed", 2), beta, np.append(P, P[-1]).astype(np.int32), 1)


def test_checkpoint_moves_between_sweep_kernels(pt):
    """The spin layout in device memory is the same for every sweep kernel: a
    checkpoint taken under one tiling and restored under another continues
    exactly as an uninterrupted run."""
    inst = synth.wishart_planted(30, 0.5, 21)
    beta = synth.beta_ladder(5, 0.2, 3.0, inst.scale)
    P = synth.penalty_ladder(3, 0.5, 4.0, 32767)
    phys = pt.sparsify(inst.Jq, "max_edges", 3)
    ref = pt.PT2D(phys, beta, P, 3, trace_capacity=32, sweep_kernel="global", walkers_per_cta=16)
    ref.run(60, 5, 9)
    order = [("global", 16), ("bits", 8), ("smem", 16), ("bits", 64), ("global", 4), ("smem", 32)]
    prev = None
    for kernel, wpc in order:
        ctx = pt.PT2D(phys, beta, P, 3, trace_capacity=32, sweep_kernel=kernel, walkers_per_cta=wpc)
        if prev is not None:
            for what, _ in ARRAYS + [("COUNTERS", None)]:
                if what in ("F", "G"):
                    continue
                ctx.write(getattr(pt, what), prev.read(getattr(pt, what)))
            prev.close()
        ctx.run(10, 5, 9)  # six contexts x 10 sweeps = the reference's 60
        assert ctx.tiling["kernel"] == kernel
        prev = ctx
    for what, _ in ARRAYS:
        assert np.array_equal(prev.read(getattr(pt, what)), ref.read(getattr(pt, what))), what


def test_checkpoint_restore_matches_uninterrupted(pt, tiny_config):
    inst = synth.wishart_planted(24, 0.75, 8)
    phys = pt.sparsify(inst.Jq, "max_edges", 3)
    beta = synth.beta_ladder(4, 0.2, 2.0, inst.scale)
    P = synth.penalty_ladder(4, 0.5, 4, 32767)
    seed = 2**64 - 3
    ref = pt.PT2D(phys, beta, P, 3, trace_capacity=32)
    ref.write(pt.TARGET, np.full(3, inst.E_planted))
    ref.run(60, 5, seed)
    a = pt.PT2D(phys, beta, P, 3, trace_capacity=32)
    a.write(pt.TARGET, np.full(3, inst.E_planted))
    a.run(25, 5, seed)
    saved = {w: a.read(getattr(pt, w)) for w in ("STATES", "WALKER_AT", "COUNTERS", "BEST_F",
                                                  "BEST_EVENT", "BEST_STATE", "SOLVED_EVENT",
                                                  "ACC_P", "ACC_B", "SUM_F", "SUM_G",
                                                  "N_FEASIBLE", "TRACE_F", "TRACE_G", "TARGET")}
    a.close()
    b = pt.PT2D(phys, beta, P, 3, trace_capacity=32, workspace="torch")
    for w, v in saved.items():
        if w != "COUNTERS":
            b.write(getattr(pt, w), v)
    b.write(pt.COUNTERS, saved["COUNTERS"])
    b.run(35, 5, seed)
    for w in saved:
        assert np.array_equal(b.read(getattr(pt, w)), ref.read(getattr(pt, w))), w
    assert np.array_equal(b.read(pt.F), ref.read(pt.F))


def test_torch_stream_and_workspace(pt, tiny_config):
    import torch

    cfg = tiny_config
    phys = pt.sparsify(cfg["inst"].Jq, "fixed", 2)
    s = torch.cuda.Stream()
    a = pt.PT2D(phys, cfg["beta"], cfg["P"], 5, stream=s, workspace="torch")
    a.run(300, 3, 77)
    b = pt.PT2D(phys, cfg["beta"], cfg["P"], 5)
    b.run(300, 3, 77)
    for what, _ in ARRAYS:
        assert np.array_equal(a.read(getattr(pt, what)), b.read(getattr(pt, what))), what


# ---- general constraint functions (penalty terms) -------------------------------------
def _penalty_pair(pt, n, groups, seed, chains=()):
    """The same instance for both sides: random couplings and fields, one-hot
    groups expanded by each side's own routine, optional copy links (K = 1)."""
    from oracle.penalties import onehot

    rng = np.random.default_rng(seed)
    A = np.zeros((n, n), np.int16)
    for a in range(n):
        for b in range(a + 1, n):
            if rng.random() < 0.2:
                A[a, b] = A[b, a] = rng.integers(-400, 401)
    cp_ptr = np.concatenate([[0], np.cumsum((A != 0).sum(1))]).astype(np.int32)
    cp_col = np.concatenate([np.nonzero(A[a])[0] for a in range(n)]).astype(np.int32)
    cp_J = np.concatenate([A[a][A[a] != 0] for a in range(n)]).astype(np.int16)
    h = rng.integers(-100, 101, n).astype(np.int32)
    sides = []
    for expand in (pt.onehot_penalty, onehot):
        lk_ptr, lk_col, lk_w, hk, g0 = expand(n, groups)
        # copy links between chained spins add weight-1 entries
        rows = [dict(zip(lk_col[lk_ptr[a]:lk_ptr[a + 1]].tolist(), lk_w[lk_ptr[a]:lk_ptr[a + 1]].tolist()))
                for a in range(n)]
        for a, b in chains:
            rows[a][b] = rows[a].get(b, 0) + 1
            rows[b][a] = rows[b].get(a, 0) + 1
        ptr = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32)
        col = np.array([b for r in rows for b in sorted(r)], np.int32)
        w = np.array([r[b] for r in rows for b in sorted(r)], np.int16)
        sides.append((ptr, col, w, hk, g0))
    (p1, c1, w1, k1, g1), (p2, c2, w2, k2, g2) = sides
    phys_p = pt.PhysicalInstance(n, cp_ptr, cp_col, cp_J, p1, c1, h=h, lk_w=w1, hk=k1, g0=g1)
    phys_o = oracle.PhysInstance(n, cp_ptr, cp_col, cp_J, p2, c2, h, n, np.arange(n, dtype=np.int32),
                                 np.arange(n + 1, dtype=np.int32), lk_w=w2, hk=k2, g0=g2)
    return phys_p, phys_o


@pytest.mark.parametrize("swap_mode,kernel", [("2d", "auto"), ("jcolumn", "auto"), ("2d", "global")])
def test_general_penalty_terms_bit_exact(pt, swap_mode, kernel):
    """One-hot groups (negative link weights, penalty fields, g0) plus copy links
    run on the generic kernels (slab in shared or global memory), bit-exact with
    the oracle."""
    groups = [list(range(k, k + 4)) for k in range(0, 40, 4)] + [[1, 5, 9], [38, 2, 17, 23, 30]]
    phys = _penalty_pair(pt, 44, groups, 7, chains=[(40, 41), (41, 42), (42, 43)])
    beta = np.array([2e-4, 5e-4, 1.2e-3, 3e-3], np.float32)
    P = np.array([50, 200, 600], np.int32)
    ctx, orc = both(pt, None, None, beta, P, 5, 31337, [(30, 3), (12, 3)], phys=phys, trace=32,
                    target=-2000, swap_mode=swap_mode, kernel=kernel)
    assert ctx.tiling["kernel"] == ("generic_smem" if kernel == "auto" else "generic")
    assert_same(pt, ctx, orc)
    assert np.all(ctx.read(pt.G) >= 0)


def test_batches_reject_general_penalty_terms(pt):
    phys, _ = _penalty_pair(pt, 12, [[0, 1, 2], [3, 4, 5, 6]], 2)
    batch = pt.Batch(1 << 24, 3, 4, trace_capacity=4)
    with pytest.raises(pt.Pt2dError):
        batch.add(phys, np.array([1e-3], np.float32), np.array([10], np.int32), 1, 1, 0)
    batch.close()


def _colouring_pair(pt, V, k, seed, capacity=None):
    """A k-colouring of a random cubic graph with one-hot groups, optionally
    with "at most `capacity` vertices per colour" inequalities through slack
    spins; each side expands the constraints with its own routine."""
    from oracle.penalties import equality

    prob = synth.colouring(V, k, seed, w_max=3)
    n = prob.n
    cons = [(g, [1] * len(g), 1) for g in prob.groups]
    if capacity is not None:
        sl = synth.slack_coefficients(capacity)
        for c in range(k):
            slack = list(range(n, n + len(sl)))
            n += len(sl)
            cons.append(([v * k + c for v in range(V)] + slack, [1] * V + sl, capacity))
    pad = n - prob.n  # slack spins carry no cost
    cp_ptr = np.concatenate([prob.cp_ptr, np.full(pad, prob.cp_ptr[-1], np.int32)])
    h = np.concatenate([prob.h, np.zeros(pad, np.int32)])
    sides = []
    for expand in (pt.equality_penalty, equality):
        sides.append(expand(n, cons))
    (p1, c1, w1, k1, g1), (p2, c2, w2, k2, g2) = sides
    phys_p = pt.PhysicalInstance(n, cp_ptr, prob.cp_col, prob.cp_J, p1, c1, h=h, lk_w=w1, hk=k1, g0=g1)
    phys_o = oracle.PhysInstance(n, cp_ptr, prob.cp_col, prob.cp_J, p2, c2, h, n, np.arange(n, dtype=np.int32),
                                 np.arange(n + 1, dtype=np.int32), lk_w=w2, hk=k2, g0=g2)
    return prob, (phys_p, phys_o)


@pytest.mark.parametrize("capacity,kernel", [(None, "auto"), (None, "global"), (9, "auto"), (9, "global")])
def test_colouring_with_equality_constraints_bit_exact(pt, capacity, kernel):
    """Graph colouring with one-hot constraints, and with per-colour capacity
    inequalities through slack spins (dense constraint rows, weights up to
    -capacity^2 / 4 between slacks), bit-exact with the oracle on the generic
    kernels."""
    prob, phys = _colouring_pair(pt, 24, 3, 5, capacity)
    beta = np.array([0.02, 0.08, 0.3, 1.0], np.float32)
    P = np.array([1, 3, 8], np.int32)
    ctx, orc = both(pt, None, None, beta, P, 5, 2468, [(60, 6), (24, 6)], phys=phys, trace=32,
                    target=prob.f_proper, kernel=kernel)
    expect = "generic" if kernel == "global" else ("penalty_smem" if capacity is None else "generic_smem")
    assert ctx.tiling["kernel"] == expect
    assert_same(pt, ctx, orc)
    assert np.all(ctx.read(pt.G) >= 0)


def _graph_colouring_pair(pt, V, k, max_deg, seed):
    """One-hot k-colouring of a random graph with degrees <= max_deg and edge
    weights 1..3; each side expands the one-hot groups with its own routine."""
    from oracle.penalties import onehot

    rng = np.random.default_rng(seed)
    deg = np.zeros(V, np.int64)
    edges = set()
    for _ in range(V * max_deg * 4):
        u, v = (int(x) for x in rng.integers(V, size=2))
        e = (min(u, v), max(u, v))
        if u == v or deg[u] >= max_deg or deg[v] >= max_deg or e in edges:
            continue
        edges.add(e)
        deg[u] += 1
        deg[v] += 1
    n = V * k
    rows = [dict() for _ in range(n)]
    h = np.zeros(n, np.int32)
    for u, v in sorted(edges):
        w = int(rng.integers(1, 4))
        for c in range(k):
            a, b = u * k + c, v * k + c
            rows[a][b] = rows[b][a] = -w
            h[a] -= w
            h[b] -= w
    cp_ptr = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32)
    cp_col = np.array([b for r in rows for b in sorted(r)], np.int32)
    cp_J = np.array([r[b] for r in rows for b in sorted(r)], np.int16)
    groups = [list(range(v * k, v * k + k)) for v in range(V)]
    p1, c1, w1, k1, g1 = pt.onehot_penalty(n, groups)
    p2, c2, w2, k2, g2 = onehot(n, groups)
    phys_p = pt.PhysicalInstance(n, cp_ptr, cp_col, cp_J, p1, c1, h=h, lk_w=w1, hk=k1, g0=g1)
    phys_o = oracle.PhysInstance(n, cp_ptr, cp_col, cp_J, p2, c2, h, n, np.arange(n, dtype=np.int32),
                                 np.arange(n + 1, dtype=np.int32), lk_w=w2, hk=k2, g0=g2)
    return phys_p, phys_o, int(deg.max())


@pytest.mark.parametrize("k,max_deg,wpc,kernel,wpt", [
    (3, 3, 0, "auto", 0), (4, 3, 16, "auto", 0), (3, 4, 0, "auto", 0), (4, 4, 32, "auto", 0),
    (3, 6, 0, "auto", 0), (4, 5, 64, "auto", 0), (3, 3, 8, "bits", 0), (4, 3, 16, "bits", 0),
    (3, 4, 64, "bits", 0), (4, 5, 128, "bits", 0), (3, 3, 8, "bits", 4), (4, 5, 32, "bits", 4)])
def test_penalty_specialised_kernel_bit_exact(pt, k, max_deg, wpc, kernel, wpt):
    """Instances with penalty terms and coupling degree <= 6, link degree <= 3
    run on the degree-specialised kernels (records padded to coupling width 3,
    4 or 6 and link width 2 or 3), with the slab as int8 or bit-packed in
    shared memory, bit-exact with the oracle, over several slab widths and a
    ragged last tile."""
    phys_p, phys_o, dmax = _graph_colouring_pair(pt, 40, k, max_deg, 100 + 10 * k + max_deg)
    assert dmax == max_deg
    beta = np.array([0.03, 0.1, 0.4, 1.2, 3.0], np.float32)
    P = np.array([1, 2, 4, 9], np.int32)
    ctx, orc = both(pt, None, None, beta, P, 7, 97531, [(48, 4), (20, 4)], phys=(phys_p, phys_o), trace=24,
                    target=-10 ** 6, wpc=wpc, kernel=kernel, wpt=wpt)
    assert ctx.tiling["kernel"] == ("penalty_bits" if kernel == "bits" else "penalty_smem")
    if kernel == "bits":
        assert ctx.tiling["walkers_per_thread"] == (wpt or 8)
    assert_same(pt, ctx, orc)
    assert np.all(ctx.read(pt.G) >= 0)


def test_three_copies_per_node_generic_smem(pt):
    """The paper's sparsification for its ground-state runs (three copies per
    node, ~N/3 couplings per copy) runs on the generic shared-memory kernel."""
    inst = synth.wishart_planted(40, 0.75, 12)
    beta = synth.beta_ladder(8, 0.1, 5.0, inst.scale)
    P = synth.penalty_ladder(4, 0.5, 64.0, 32767)
    ctx, orc = both(pt, inst, ("fixed", 3), beta, P, 6, 4040, [(40, 5), (10, 5)],
                    target=inst.E_planted, trace=16)
    assert ctx.tiling["kernel"] == "generic_smem"
    assert_same(pt, ctx, orc)


# ---- the J-column PT baseline ----------------------------------------------------------
@pytest.mark.parametrize("kernel,wpc", [("global", 16), ("smem", 16), ("bits", 8), ("auto", 0)])
def test_jcolumn_baseline_bit_exact(pt, kernel, wpc):
    """Beta-swaps only, equal penalties in every column (the paper's comparison:
    J standard PTs at the mean 2D-PT penalty), best last-row record."""
    inst = synth.wishart_planted(30, 0.5, 21)
    beta = synth.beta_ladder(5, 0.2, 3.0, inst.scale)
    P_2d = synth.penalty_ladder(3, 0.5, 4.0, 32767)
    P = np.full(3, int(np.rint(P_2d.mean())), np.int32)
    ctx, orc = both(pt, inst, ("max_edges", 3), beta, P, 7, 0xABCDEF, [(35, 7), (21, 7)],
                    target=inst.E_planted, wpc=wpc, kernel=kernel, swap_mode="jcolumn")
    assert_same(pt, ctx, orc)
    assert ctx.read(pt.ACC_P).sum() == 0 and ctx.read(pt.COUNTERS)[2] == -1


def test_jcolumn_tiny_config_bit_exact(pt, tiny_config):
    cfg = tiny_config
    P = np.full(4, int(np.rint(cfg["P"].mean())), np.int32)
    ctx, orc = both(pt, cfg["inst"], ("fixed", 2), cfg["beta"], P, 2, 7, [(3000, 1)],
                    target=cfg["inst"].E_planted, trace=128, swap_mode="jcolumn")
    assert_same(pt, ctx, orc)


# ---- full-size configurations, checked on samples the oracle computes -----------------
def _bench_workload(key):
    """The benchmark's own workload (instance, ladders, runs, swap interval)."""
    import bench

    return bench.make_workload(key)


def _oracle_runs_in_threads(oinst, beta, P, run_ids, seed, sweeps, interval, **kw):
    """One OracleRun per run id, run in parallel threads (the oracle's C code
    releases the interpreter lock)."""
    import threading

    orcs = [oracle.OracleRun(oinst, beta, P, [r], seed, **kw) for r in run_ids]
    ths = [threading.Thread(target=o.run, args=(sweeps, interval)) for o in orcs]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    return orcs


def test_n200_full_size_sampled_runs(pt):
    """The benchmark's N=200 workload exactly as it is timed: planted Wishart
    N=200, alpha=0.5, <=3 edges per copy (13,400 spins), I=32 x J=8 with the
    benchmark's ladders (beta 0.1..5.0 / s, P 0.5..64 x 32767), 64 runs, swap
    interval 50, in the benchmark's launch configuration (its own stream,
    torch-allocated workspace, kernel timing on); two runs checked in full by
    the oracle after two events (100 sweeps)."""
    import torch

    wl = _bench_workload("n200")
    inst, beta, P, runs, interval = wl["inst"], wl["beta"], wl["P"], wl["runs"], wl["interval"]
    assert (interval, runs, len(beta), len(P)) == (50, 64, 32, 8)
    phys_p = pt.sparsify(inst.Jq, "max_edges", 3)
    assert phys_p.n == 13400 == int(np.ceil(inst.degrees / 3).sum())
    seed = 100
    stream = torch.cuda.Stream()
    ctx = pt.PT2D(phys_p, beta, P, runs, stream=stream, workspace="torch", trace_capacity=8,
                  profile=True)
    assert ctx.tiling["kernel"] == "smem" and ctx.tiling["walkers_per_thread"] == 8
    assert ctx.tiling["walkers_per_cta"] == 16 and ctx.tiling["threads_per_cta"] == 768
    ctx.write(pt.TARGET, np.full(runs, inst.E_planted))
    with torch.cuda.stream(stream):
        ctx.run(2 * interval, interval, seed)
    oinst = oracle.OracleInstance(oracle.sparsify(inst.Jq, "max_edges", 3))
    orcs = _oracle_runs_in_threads(oinst, beta, P, (0, 45), seed, 2 * interval, interval, trace_cap=8,
                                   target=inst.E_planted)
    for run_id, orc in zip((0, 45), orcs):
        assert_same(pt, ctx, orc, runs_sel=[run_id])
    ctx.close()


def test_n800_full_size_sampled_walkers(pt):
    """The benchmark's N=800 workload as it is timed (213,551 spins, I=64 x
    J=16, 16 runs, 3.5 GB of spins, the benchmark's ladders, one event of 50
    sweeps): sampled walkers match the oracle spin for spin, their f and g
    match, and the event's P-swap decisions match the oracle's swap event
    replayed on the GPU's f and g."""
    wl = _bench_workload("n800")
    inst, beta, P, runs, interval = wl["inst"], wl["beta"], wl["P"], wl["runs"], wl["interval"]
    assert (interval, runs, len(beta), len(P)) == (50, 16, 64, 16)
    phys_p = pt.sparsify(inst.Jq, "max_edges", 3)
    # ~3 edges per copy of ~799 neighbours (a few quantised couplings round to 0)
    assert phys_p.n == int(np.ceil(inst.degrees / 3).sum()) and phys_p.n > 213000
    seed = 100
    ctx = pt.PT2D(phys_p, beta, P, runs, trace_capacity=4, profile=True)
    # the automatic tiling holds this instance bit-packed in shared memory, 8 walkers a CTA
    assert ctx.tiling["kernel"] == "bits" and ctx.tiling["walkers_per_cta"] == 8
    ctx.run(interval, interval, seed)
    oinst = oracle.OracleInstance(oracle.sparsify(inst.Jq, "max_edges", 3))
    f_gpu = ctx.read(pt.F)
    g_gpu = ctx.read(pt.G)
    for run_id, w in ((0, 0), (3, 511), (3, 1023), (15, 777), (9, 14)):
        s = oinst.init_walker(seed, run_id, w)
        i, j = divmod(w, 16)  # walker w starts in slot w
        for t in range(interval):
            oinst.sweep_walker(s, seed, run_id, w, t, beta[i], P[j])
        assert np.array_equal(ctx.read_walker(run_id, w), s), (run_id, w)
        assert f_gpu[run_id, w] == oinst.cost_f(s)
        assert g_gpu[run_id, w] == oinst.constraint_g(s)
    at_gpu = ctx.read(pt.WALKER_AT)
    acc_gpu = ctx.read(pt.ACC_P)
    for run_id in (3, 15):
        at, accP, accB = ocore.swap_event(beta, P, f_gpu[run_id], g_gpu[run_id],
                                          np.arange(64 * 16), seed, run_id, 1, 1)
        assert np.array_equal(at_gpu[run_id], at)
        assert np.array_equal(acc_gpu[run_id], accP)
    ctx.close()


def _bench_ladder_pairs():
    """(beta, H) pairs from the benchmark's ladders: betas of a few rows of the
    N=200, N=800 and uneven-batch ladders, each with fields H that put the
    heat-bath probability 1/(1 + exp(-beta H)) at several levels between
    2^-23 and 1 - 2^-23 (where the decision turns on the uniform), within the
    largest field the benchmark's instances produce, |H| <= 2 x 3 x 32767
    (three couplings) + 2 x 64 x 32767 (two links at the largest penalty),
    and that largest field itself."""
    import bench

    betas = []
    for key in ("n200", "n800"):
        wl = bench.make_workload(key)
        b = wl["beta"]
        betas += [b[k * (len(b) - 1) // 5] for k in range(6)]
    inst = synth.wishart_planted(57, 0.25, 1001)
    b = synth.beta_ladder(16, bench.BETA_MIN, bench.BETA_MAX, inst.scale)
    betas += [b[0], b[-1]]
    big = 2 * 3 * 32767 + 2 * 64 * 32767
    pairs = set()
    for k, beta in enumerate(betas):
        beta = np.float32(beta)
        for z in (-15.5, -5.1, -0.7, 2.3, 9.6):
            H = int(np.clip(np.rint((z + 0.01 * k) / float(beta)), -big, big))
            pairs.add((beta, H))
    for beta in (betas[0], betas[4], betas[-2]):
        pairs |= {(np.float32(beta), big), (np.float32(beta), -big)}
    return sorted(pairs)


def test_heatbath_fast_path_band_over_bench_ladders(pt):
    """The hardware-exponential fast path decides only outside its error band
    and defers to the exact single-precision contract inside it; over every
    uniform of the 2^23-point grid, for (beta, H) pairs taken from the
    benchmark's ladders, the decisions equal the oracle's one by one and their
    count equals the oracle's exhaustive count."""
    pairs = _bench_ladder_pairs()
    assert len(pairs) >= 50
    r = (np.arange(2**23, dtype=np.uint64) << np.uint64(9)).astype(np.uint32)
    for beta, H in pairs:
        assert abs(H) < 2**24
        b = np.full(r.size, beta, np.float32)
        h = np.full(r.size, H, np.int32)
        got = pt.diag_heatbath(b, h, r)
        exp = ocore.heatbath_array(b, h, r)
        if not np.array_equal(got, exp):
            bad = np.nonzero(got != exp)[0]
            raise AssertionError(f"beta={beta!r} H={H}: {bad.size} uniforms differ, first {bad[:4]}")
        assert int((got > 0).sum()) == oracle.heatbath_count(float(beta), H), (beta, H)


def test_colouring_full_size_sampled_runs(pt):
    """The constrained workload at full size: 3-colouring of a random cubic
    graph, V=2000 (6000 spins, one-hot groups), I=16 x J=8, 256 runs, on the
    degree-specialised penalty kernel in the automatic launch configuration the
    benchmark uses; three runs checked in full by the oracle after two events."""
    from oracle.penalties import onehot

    prob = synth.colouring(2000, 3, 7)
    p1, c1, w1, k1, g1 = pt.onehot_penalty(prob.n, prob.groups)
    p2, c2, w2, k2, g2 = onehot(prob.n, prob.groups)
    phys_p = pt.PhysicalInstance(prob.n, prob.cp_ptr, prob.cp_col, prob.cp_J, p1, c1, h=prob.h, lk_w=w1,
                                 hk=k1, g0=g1)
    phys_o = oracle.PhysInstance(prob.n, prob.cp_ptr, prob.cp_col, prob.cp_J, p2, c2, prob.h, prob.n,
                                 np.arange(prob.n, dtype=np.int32), np.arange(prob.n + 1, dtype=np.int32),
                                 lk_w=w2, hk=k2, g0=g2)
    beta = np.geomspace(0.05, 2.0, 16).astype(np.float32)
    P = np.array([1, 2, 3, 5, 8, 12, 17, 24], np.int32)
    seed = 2024
    ctx = pt.PT2D(phys_p, beta, P, 256, trace_capacity=8)
    assert ctx.tiling["kernel"] == "penalty_smem" and ctx.tiling["walkers_per_cta"] == 32
    ctx.write(pt.TARGET, np.full(256, prob.f_proper))
    ctx.run(20, 10, seed)
    oinst = oracle.OracleInstance(phys_o)
    for run_id in (0, 137, 255):
        orc = oracle.OracleRun(oinst, beta, P, [run_id], seed, trace_cap=8, target=prob.f_proper)
        orc.run(20, 10)
        assert_same(pt, ctx, orc, runs_sel=[run_id])


@pytest.mark.parametrize("kernel", ["auto", "global"])
def test_wide_records_without_links(pt, kernel):
    """An instance with no copy links at all (a plain Ising model, g = 0) and
    coupling degree up to 9: wide records with link width 0 on the
    runtime-degree kernels, bit-exact with the oracle."""
    rng = np.random.default_rng(31)
    n = 70
    A = np.zeros((n, n), np.int16)
    deg = np.zeros(n, int)
    for _ in range(n * 20):
        a, b = (int(x) for x in rng.integers(n, size=2))
        if a != b and A[a, b] == 0 and deg[a] < 9 and deg[b] < 9:
            A[a, b] = A[b, a] = int(rng.integers(-32767, 32768)) or 1
            deg[a] += 1
            deg[b] += 1
    cp_ptr = np.concatenate([[0], np.cumsum((A != 0).sum(1))]).astype(np.int32)
    cp_col = np.concatenate([np.nonzero(A[a])[0] for a in range(n)]).astype(np.int32)
    cp_J = np.concatenate([A[a][A[a] != 0] for a in range(n)]).astype(np.int16)
    lk_ptr = np.zeros(n + 1, np.int32)
    lk_col = np.zeros(0, np.int32)
    h = rng.integers(-500, 501, n).astype(np.int32)
    phys_p = pt.PhysicalInstance(n, cp_ptr, cp_col, cp_J, lk_ptr, lk_col, h=h)
    phys_o = oracle.PhysInstance(n, cp_ptr, cp_col, cp_J, lk_ptr, lk_col, h, n, np.arange(n, dtype=np.int32),
                                 np.arange(n + 1, dtype=np.int32))
    beta = np.geomspace(1e-5, 3e-4, 6).astype(np.float32)
    P = np.array([1, 5], np.int32)
    ctx, orc = both(pt, None, None, beta, P, 4, 4711, [(30, 5), (15, 5)], phys=(phys_p, phys_o), trace=16,
                    kernel=kernel)
    assert ctx.tiling["kernel"] == ("generic_smem" if kernel == "auto" else "generic")
    assert_same(pt, ctx, orc)
    assert np.all(ctx.read(pt.G) == 0)


def test_contexts_on_concurrent_threads(pt):
    """Contexts of different sizes (so different shared-memory slabs, on the
    int8, bit-packed and runtime-degree kernels) run at the same time from
    several host threads on their own streams; each gives the same result as
    the same context run alone."""
    import concurrent.futures as cf

    import torch

    jobs = []
    for k, (N, rule) in enumerate([(30, ("max_edges", 3)), (60, ("max_edges", 3)), (24, ("fixed", 3)),
                                   (45, ("fixed", 3)), (80, ("max_edges", 3)), (36, ("max_edges", 3))]):
        inst = synth.wishart_planted(N, 0.5, 70 + k)
        kern = "bits" if k == 5 else "auto"
        jobs.append((pt.sparsify(inst.Jq, *rule), synth.beta_ladder(8, 0.2, 3.0, inst.scale),
                     synth.penalty_ladder(4, 0.5, 4.0, 32767), 3 + k, 900 + k, kern))

    def run(job, stream=None):
        phys, beta, P, runs, seed, kern = job
        ctx = pt.PT2D(phys, beta, P, runs, stream=stream, trace_capacity=8, sweep_kernel=kern,
                      walkers_per_cta=8 if kern == "bits" else 0)
        for _ in range(6):
            ctx.run(20, 5, seed)
        out = (ctx.read(pt.STATES), ctx.read(pt.F), ctx.read(pt.WALKER_AT), ctx.tiling["kernel"])
        ctx.close()
        return out

    alone = [run(j) for j in jobs]
    assert {a[3] for a in alone} >= {"smem", "bits", "generic_smem"}
    with cf.ThreadPoolExecutor(len(jobs)) as ex:
        for rep in range(3):
            mixed = list(ex.map(lambda j: run(j, torch.cuda.Stream()), jobs))
            for a, b in zip(alone, mixed):
                for x, y in zip(a[:3], b[:3]):
                    assert np.array_equal(x, y), rep
