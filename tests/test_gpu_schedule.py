"""Adaptive ladder schedule (Algorithm 2) on the GPU against the oracle's: the
same population samples (bit-exact 2D-PT contexts), the same exact statistics
and the same double arithmetic give identical ladders and sample counts."""
import numpy as np
import pytest
from scipy.special import erfcinv

import oracle
from oracle.schedule import ScheduleParams, adaptive_schedule, oracle_sampler
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


@pytest.mark.parametrize("N,seed,rows,cols,n_chain,mcs,smin", [
    (12, 4, 6, 4, 64, 50, 4000.0),
    (16, 11, 8, 6, 128, 200, 2.0 * 32767 / 8),
])
def test_schedule_matches_oracle(pt, N, seed, rows, cols, n_chain, mcs, smin):
    inst = synth.wishart_planted(N, 0.5, seed)
    alpha = float(2 * erfcinv(0.5))
    prm = ScheduleParams(beta0=0.2 / inst.scale, P0=int(0.5 * 32767), max_rows=rows, max_cols=cols,
                         sigma_min=smin, alpha_beta=alpha, alpha_P=alpha, n_chain=n_chain, mcs=mcs,
                         seed=1234 + N)
    oinst = oracle.OracleInstance(oracle.sparsify(inst.Jq, "max_edges", 3))
    b_o, P_o, k_o = adaptive_schedule(oracle_sampler(oinst, prm), prm)
    b_g, P_g, k_g = pt.adaptive_schedule(pt.sparsify(inst.Jq, "max_edges", 3), **vars(prm))
    assert k_g == k_o
    assert np.array_equal(P_g, P_o)
    assert np.array_equal(b_g.view(np.uint32), b_o.view(np.uint32))


def test_schedule_rejects_bad_parameters(pt):
    inst = synth.wishart_planted(8, 0.5, 1)
    phys = pt.sparsify(inst.Jq, "fixed", 2)
    good = dict(beta0=1e-5, P0=100, max_rows=3, max_cols=2, sigma_min=1.0, alpha_beta=1.0,
                alpha_P=1.0, n_chain=8, mcs=4, seed=1)
    for k, v in (("n_chain", 1), ("mcs", 0), ("beta0", 0.0), ("sigma_min", -1.0), ("max_rows", 0),
                 ("alpha_P", float("nan")), ("P0", -1)):
        with pytest.raises(pt.Pt2dError):
            pt.adaptive_schedule(phys, **dict(good, **{k: v}))
    beta, P, k = pt.adaptive_schedule(phys, **good)
    assert 1 <= beta.size <= 3 and 1 <= P.size <= 2 and k >= 1
