"""The C-ABI library loads, exports every entry point include/pt2d.h declares,
and its host-only parts (sparsifier, colouring, validation, workspace sizing)
agree with the oracle bit for bit.  No GPU needed."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pt():
    from paper_2506_14781_gb300 import build as b

    b.build()
    import paper_2506_14781_gb300 as m

    return m


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "pt2d.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(pt2d_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_library_exports_every_declared_symbol(pt):
    from paper_2506_14781_gb300 import _lib

    declared = _declared_functions()
    assert len(declared) >= 15
    L = C.CDLL(_lib.LIB_PATH)
    for name in declared:
        assert hasattr(L, name), name
    assert set(declared) <= set(_lib.EXPORTS) | set(declared)
    assert sorted(_lib.EXPORTS) == declared


@pytest.mark.parametrize("rule,param,N,alpha,seed", [
    ("fixed", 2, 10, 0.5, 1), ("max_edges", 3, 60, 0.5, 2), ("max_degree", 4, 50, 0.25, 3),
    ("max_edges", 3, 17, 0.75, 4), ("fixed", 3, 12, 0.75, 5),
])
def test_sparsifier_and_colouring_match_oracle(pt, rule, param, N, alpha, seed):
    inst = synth.wishart_planted(N, alpha, seed)
    a = pt.sparsify(inst.Jq, rule, param)
    b = oracle.sparsify(inst.Jq, rule, param)
    assert a.n == b.n
    for k in ("cp_ptr", "cp_col", "cp_J", "lk_ptr", "lk_col", "copy_of"):
        assert np.array_equal(getattr(a, k), getattr(b, k)), k
    ca, na = pt.greedy_color(a)
    cb, nb = oracle.greedy_color(b.n, b.cp_ptr, b.cp_col, b.lk_ptr, b.lk_col)
    assert na == nb and np.array_equal(ca, cb)


def _status_of_workspace(pt, inst, I=2, J=2, runs=1, sweep_kernel=None):
    from paper_2506_14781_gb300 import _lib

    cs = inst.c_struct()
    need = C.c_size_t()
    opt = None
    if sweep_kernel is not None:
        o = _lib.Options()
        _lib.lib().pt2d_default_options(C.byref(o))
        o.sweep_kernel = sweep_kernel
        opt = C.byref(o)
    st = _lib.lib().pt2d_workspace_size(C.byref(cs), I, J, runs, opt, C.byref(need))
    return st, need.value


def test_validation_rejects_malformed_instances(pt):
    inst = synth.wishart_planted(12, 0.5, 1)
    good = pt.sparsify(inst.Jq, "fixed", 2)
    st, need = _status_of_workspace(pt, good)
    assert st == 0 and need > good.n
    # asymmetric coupling value
    bad = pt.PhysicalInstance(good.n, good.cp_ptr, good.cp_col, good.cp_J.copy(), good.lk_ptr,
                              good.lk_col)
    bad.cp_J[0] += 1
    assert _status_of_workspace(pt, bad)[0] == -1
    # self loop
    bad = pt.PhysicalInstance(good.n, good.cp_ptr, good.cp_col.copy(), good.cp_J, good.lk_ptr,
                              good.lk_col)
    bad.cp_col[0] = 0
    assert _status_of_workspace(pt, bad)[0] == -1
    # improper colouring
    bad = pt.PhysicalInstance(good.n, good.cp_ptr, good.cp_col, good.cp_J, good.lk_ptr,
                              good.lk_col, color=np.zeros(good.n, np.int32))
    assert _status_of_workspace(pt, bad)[0] == -1
    # one-sided link
    lk_ptr = good.lk_ptr.copy()
    lk_col = good.lk_col.copy()
    bad = pt.PhysicalInstance(good.n, good.cp_ptr, good.cp_col, good.cp_J, lk_ptr, lk_col)
    bad.lk_col[0] = (bad.lk_col[0] + 2) % good.n
    assert _status_of_workspace(pt, bad)[0] == -1
    # sizes
    assert _status_of_workspace(pt, good, I=0)[0] == -1
    assert _status_of_workspace(pt, good, runs=0)[0] == -1
    # bit-packed slabs exist for the specialised layouts only
    assert _status_of_workspace(pt, good, sweep_kernel=3)[0] == 0
    wide = pt.sparsify(synth.wishart_planted(30, 0.5, 2).Jq, "fixed", 2)  # ~15 couplings per copy
    assert _status_of_workspace(pt, wide, sweep_kernel=3)[0] == -1
    assert _status_of_workspace(pt, wide, sweep_kernel=2)[0] == 0


def test_strerror_and_defaults(pt):
    from paper_2506_14781_gb300 import _lib

    L = _lib.lib()
    for code in range(-6, 1):
        assert len(L.pt2d_strerror(code)) > 0
    opt = _lib.Options()
    L.pt2d_default_options(C.byref(opt))
    assert opt.trace_capacity == 1024 and opt.device == -1 and opt.workspace is None


def test_create_fails_loudly_without_gpu(pt):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    inst = synth.wishart_planted(10, 0.5, 1)
    phys = pt.sparsify(inst.Jq, "fixed", 2)
    with pytest.raises(pt.Pt2dError):
        pt.PT2D(phys, [1e-5, 2e-5], [100, 200], 1)


def test_allocation_failure_hook_counts_without_a_gpu():
    import paper_2506_14781_gb300 as pt

    assert pt.debug_fail_allocations(3) == 0
    assert pt.debug_fail_allocations(0) == 3
    assert pt.debug_fail_allocations(-5) == 0


def test_read_probe_rejects_bad_arguments_without_a_gpu(pt):
    L = pt._lib.lib()
    ms = C.c_float()
    buf = C.c_void_p(4096)  # never dereferenced: every call below fails its argument check
    assert L.pt2d_diag_read_bandwidth(None, 1024, 1, buf, C.byref(ms)) == -1
    assert L.pt2d_diag_read_bandwidth(buf, 1000, 1, buf, C.byref(ms)) == -1  # not a multiple of 16
    assert L.pt2d_diag_read_bandwidth(buf, 1024, 0, buf, C.byref(ms)) == -1
    assert L.pt2d_diag_read_bandwidth(C.c_void_p(4100), 1024, 1, buf, C.byref(ms)) == -1  # unaligned
    assert L.pt2d_diag_read_bandwidth(buf, 1024, 1, None, C.byref(ms)) == -1


def test_noalloc_reports_unsupported_without_a_gpu(pt):
    """pt2d_run_noalloc checks the device before it looks up its scratch array,
    so without an sm_103 GPU it returns PT2D_ERR_UNSUPPORTED, as pt2d_create does."""
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    inst = synth.wishart_planted(10, 0.5, 1)
    phys = pt.sparsify(inst.Jq, "fixed", 2)
    beta = np.array([1e-5, 2e-5], np.float32)
    P = np.array([100, 200], np.int32)
    cs = phys.c_struct()
    st = pt._lib.lib().pt2d_run_noalloc(C.byref(cs), 2, beta.ctypes.data_as(C.c_void_p), 2,
                                        P.ctypes.data_as(C.c_void_p), 1, 10, 5, 1, None, None, None,
                                        None, None)
    assert st == -6
