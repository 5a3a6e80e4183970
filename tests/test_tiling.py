"""The sweep tiling a context chooses, planned on the host (pt2d_plan_tiling)
with no GPU: the slab kernel, walkers and threads per CTA and walkers per
thread for the benchmark's workloads and the edge cases of the rules (a GPU
run reports the same tilings through pt2d_tiling)."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import synth  # noqa: E402


@pytest.fixture(scope="module")
def pt():
    from paper_2506_14781_gb300 import build as b

    b.build()
    import paper_2506_14781_gb300 as m

    return m


def _bench_instance(pt, key):
    import bench

    w = bench.make_workload(key)
    return pt.sparsify(w["inst"].Jq, "max_edges", 3), w


def test_n200_workload_takes_eight_walkers_per_thread(pt):
    phys, w = _bench_instance(pt, "n200")
    t = pt.plan_tiling(phys, w["I"], w["J"], w["runs"])
    assert t == dict(kernel="smem", walkers_per_cta=16, threads_per_cta=768, walkers_per_thread=8)
    # four walkers a thread when asked for, up to 1024 threads
    t4 = pt.plan_tiling(phys, w["I"], w["J"], w["runs"], walkers_per_thread=4)
    assert t4["walkers_per_thread"] == 4 and t4["threads_per_cta"] == 1024


def test_n800_workload_takes_bit_packed_bytes(pt):
    phys, w = _bench_instance(pt, "n800")
    t = pt.plan_tiling(phys, w["I"], w["J"], w["runs"])
    assert t == dict(kernel="bits", walkers_per_cta=8, threads_per_cta=896, walkers_per_thread=8)
    # more threads than the byte kernel takes: a nibble per thread
    assert pt.plan_tiling(phys, w["I"], w["J"], w["runs"], threads_per_cta=1024)["walkers_per_thread"] == 4
    with pytest.raises(pt.Pt2dError):
        pt.plan_tiling(phys, w["I"], w["J"], w["runs"], threads_per_cta=1024, walkers_per_thread=8)


def test_runtime_degree_kernel_sizes_ctas_to_the_grid(pt):
    """Three copies per node: 256-thread CTAs when the grid has CTAs enough to
    share the SMs, the full width when it has no more CTAs than SMs."""
    inst = synth.wishart_planted(100, 0.75, 3)
    phys = pt.sparsify(inst.Jq, "fixed", 3)
    many = pt.plan_tiling(phys, 20, 20, 64)  # 25,600 walkers in 64-walker slabs: 400 CTAs
    assert many == dict(kernel="generic_smem", walkers_per_cta=64, threads_per_cta=256, walkers_per_thread=4)
    few = pt.plan_tiling(phys, 20, 20, 1)    # 400 walkers: fewer CTAs than SMs
    assert few["kernel"] == "generic_smem" and few["threads_per_cta"] > 256
    mid = pt.plan_tiling(phys, 20, 20, 64, walkers_per_cta=128)  # 200 CTAs: two per SM
    assert mid["threads_per_cta"] == 320


def test_penalty_terms_take_the_penalty_kernels(pt):
    for V, runs, kernel, wpc, threads, wpt in ((2000, 256, "penalty_smem", 32, 1024, 4),
                                               (40000, 64, "penalty_bits", 8, 512, 8)):
        prob = synth.colouring(V, 3, 7)
        lk_ptr, lk_col, lk_w, hk, g0 = pt.onehot_penalty(prob.n, prob.groups)
        phys = pt.PhysicalInstance(prob.n, prob.cp_ptr, prob.cp_col, prob.cp_J, lk_ptr, lk_col, h=prob.h,
                                   lk_w=lk_w, hk=hk, g0=g0)
        t = pt.plan_tiling(phys, 16, 8, runs)
        assert t == dict(kernel=kernel, walkers_per_cta=wpc, threads_per_cta=threads, walkers_per_thread=wpt)


def test_global_kernel_and_invalid_requests(pt):
    inst = synth.wishart_planted(30, 0.5, 21)
    phys = pt.sparsify(inst.Jq, "max_edges", 3)
    g = pt.plan_tiling(phys, 5, 3, 7, sweep_kernel="global")
    assert g["kernel"] == "global" and g["threads_per_cta"] == 256
    for bad in (dict(walkers_per_cta=12), dict(threads_per_cta=48), dict(walkers_per_thread=2),
                dict(sweep_kernel="smem", walkers_per_cta=4)):
        with pytest.raises(pt.Pt2dError):
            pt.plan_tiling(phys, 5, 3, 7, **bad)
