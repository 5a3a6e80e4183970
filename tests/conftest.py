import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: takes more than ~20 s on the CPU")


@pytest.fixture(scope="session")
def tiny_config():
    """The tiny bit-exact / KL configuration: Wishart-planted N=10, alpha=0.5,
    2 copies per node (20 physical spins, 10 links), I=4 beta (geometric
    0.1..2.0) x J=4 P (linear 0.5..4.0 x 32767), swaps every sweep."""
    import synth
    import oracle

    inst = synth.wishart_planted(10, 0.5, seed=1)
    phys = oracle.sparsify(inst.Jq, "fixed", 2)
    beta = synth.beta_ladder(4, 0.1, 2.0, inst.scale)
    P = synth.penalty_ladder(4, 0.5, 4.0, 32767)
    return dict(inst=inst, phys=phys, beta=beta, P=P)
