"""Failure handling on the GPU without a GPU fault: injected allocation
failures (a host-side hook) and refused inputs leave the library usable."""
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


def _problem(pt):
    inst = synth.wishart_planted(12, 0.5, 3)
    return (pt.sparsify(inst.Jq, "fixed", 2), synth.beta_ladder(4, 0.1, 2.0, inst.scale),
            synth.penalty_ladder(4, 0.5, 4.0, 32767))


def test_injected_allocation_failures(pt):
    phys, beta, P = _problem(pt)
    assert pt.debug_fail_allocations(2) == 0
    with pytest.raises(pt.Pt2dError) as e:
        pt.PT2D(phys, beta, P, 2)
    assert "OOM" in str(e.value)
    with pytest.raises(pt.Pt2dError) as e:
        pt.Batch(1 << 24, 3, 4)
    assert "OOM" in str(e.value)
    assert pt.debug_fail_allocations(0) == 0
    ctx = pt.PT2D(phys, beta, P, 2)  # the next allocation works again
    ctx.run(20, 5, 1)
    assert ctx.read(pt.COUNTERS)[1] == 4
    ctx.close()
    b = pt.Batch(1 << 24, 64, 4)  # two copies of 12 nodes: ~6 couplings per copy
    b.add(phys, beta, P, 1, 1, 0)
    b.run(2, 5)
    b.close()


def test_refused_inputs_leave_the_context_usable(pt):
    phys, beta, P = _problem(pt)
    ctx = pt.PT2D(phys, beta, P, 2)
    ctx.run(10, 5, 7)
    for bad in (lambda: ctx.run(10, 5, 8),              # another seed
                lambda: ctx.run(-1, 5, 7),              # negative sweeps
                lambda: ctx.write(pt.F, ctx.read(pt.F)),  # f is not writable
                lambda: ctx.read(99)):                  # unknown array
        with pytest.raises((pt.Pt2dError, KeyError)):
            bad()
    ctx.run(10, 5, 7)
    assert ctx.read(pt.COUNTERS)[1] == 4
    ctx.close()


@pytest.mark.gpu
def test_read_probe_times_l2_and_rejects_bad_calls():
    """The read-bandwidth probe returns a positive time for an L2-sized buffer
    and a larger one for more passes; misaligned or unsized calls are refused."""
    import torch

    import paper_2506_14781_gb300 as pt

    buf = torch.ones(8 << 20, dtype=torch.uint8, device="cuda")
    out = torch.zeros(4, dtype=torch.int32, device="cuda")
    pt.diag_read_bandwidth(buf, 2, out)
    t1 = pt.diag_read_bandwidth(buf, 10, out)
    t2 = pt.diag_read_bandwidth(buf, 200, out)
    assert 0 < t1 < t2
    with pytest.raises(pt.Pt2dError):
        pt.diag_read_bandwidth(buf[1:17], 1, out)  # not 16-byte aligned
