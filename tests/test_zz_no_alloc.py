"""pt2d_run_noalloc: the one-shot entry point for callers that cannot allocate
device memory (their GPU memory is owned by their own pool, or a device
allocation's synchronisation is not acceptable to them).  It must give the
same results as the context entry points (create, run, read), which allocate
their workspace, on two calls in a row that share its static device scratch,
and it must refuse problems larger than that scratch.

This file is collected last on purpose: run alone in a fresh process, the first
call also does the one-time look-up of the scratch address.
"""
import ctypes as C

import numpy as np
import pytest

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


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _noalloc(pt, phys, beta, P, runs, sweeps, interval, seed):
    from paper_2506_14781_gb300 import _lib

    R = len(beta) * len(P)
    out = dict(states=np.empty((runs, R, phys.n), np.int8), walker_at=np.empty((runs, R), np.int32),
               f=np.empty((runs, R), np.int64), g=np.empty((runs, R), np.int64))
    cs = phys.c_struct()
    beta = np.ascontiguousarray(beta, np.float32)
    P = np.ascontiguousarray(P, np.int32)
    st = _lib.lib().pt2d_run_noalloc(C.byref(cs), len(beta), _p(beta), len(P), _p(P), runs,
                                     sweeps, interval, seed, None, _p(out["states"]),
                                     _p(out["walker_at"]), _p(out["f"]), _p(out["g"]))
    return st, out


def _reference(pt, phys, beta, P, runs, sweeps, interval, seed):
    ctx = pt.PT2D(phys, beta, P, runs, trace_capacity=0)
    ctx.run(sweeps, interval, seed)
    ref = dict(states=ctx.read(pt.STATES), walker_at=ctx.read(pt.WALKER_AT), f=ctx.read(pt.F),
               g=ctx.read(pt.G))
    ctx.close()
    return ref


def test_noalloc_matches_context_api_twice(pt):
    cases = []
    inst = synth.wishart_planted(40, 0.5, 12)
    cases.append((pt.sparsify(inst.Jq, "max_edges", 3), synth.beta_ladder(6, 0.1, 2.0, inst.scale),
                  synth.penalty_ladder(5, 0.5, 4.0, 32767), 3, 60, 6, 31))
    inst2 = synth.wishart_planted(10, 0.5, 1)
    cases.append((pt.sparsify(inst2.Jq, "fixed", 2), synth.beta_ladder(4, 0.1, 2.0, inst2.scale),
                  synth.penalty_ladder(4, 0.5, 4.0, 32767), 2, 200, 1, 7))
    import torch

    refs = [_reference(pt, *case) for case in cases]
    # Any device allocation inside the entry point would now fail as out of
    # memory: the library's allocation hook refuses the next 2^30 of them.
    pt.debug_fail_allocations(1 << 30)
    try:
        for case, ref in zip(cases, refs):  # two calls in a row
            st, got = _noalloc(pt, *case)
            assert st == 0, pt._lib.lib().pt2d_strerror(st)
            for k in ref:
                assert np.array_equal(got[k], ref[k]), k
        # a third call, repeating the first problem (its kernels are loaded by
        # now): free device memory is the same before and after it
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        st, got = _noalloc(pt, *cases[0])
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        assert st == 0 and all(np.array_equal(got[k], refs[0][k]) for k in got)
    finally:
        pt.debug_fail_allocations(0)


def test_noalloc_rejects_problems_beyond_scratch(pt):
    inst = synth.wishart_planted(200, 0.5, 2)
    phys = pt.sparsify(inst.Jq, "max_edges", 3)  # 13,400 spins x 64 runs x 256 replicas
    beta = synth.beta_ladder(32, 0.1, 2.0, inst.scale)
    P = synth.penalty_ladder(8, 0.5, 4.0, 32767)
    from paper_2506_14781_gb300 import _lib

    cs = phys.c_struct()
    st = _lib.lib().pt2d_run_noalloc(C.byref(cs), 32, _p(beta), 8, _p(P), 64, 50, 50, 1, None,
                                     None, None, None, None)
    assert st == -1  # PT2D_ERR_INVALID_ARG: larger than PT2D_NOALLOC_SCRATCH_BYTES
