"""CPU oracle for two-dimensional parallel tempering (2D-PT).

TEST INFRASTRUCTURE ONLY.  A plain, slow, obviously correct restatement of the
paper's method (arxiv 2506.14781): copy-chain sparsification, greedy colouring,
heat-bath sweeps, P-swaps (Eq. 2), beta-swaps (Eq. 3) and the 2D-PT loop
(Algorithm 1), plus brute-force Boltzmann distributions for pinning.  Only the
tests, the smoke check and the CPU-baseline leg of the benchmark import it; the
GPU library never does, and the two share no code.

Parity status of each function (what pins it) is listed in the test files
``tests/test_oracle_*.py``.
"""
from .sparsify import PhysInstance, sparsify, lift, project
from .coloring import greedy_color, is_proper
from .core import (OracleInstance, OracleRun, philox4x32_10, pt_exp, heatbath, swap_accept,
                   heatbath_count, swap_count, pt_exp_constants)
from . import boltzmann

__all__ = [
    "PhysInstance",
    "sparsify",
    "lift",
    "project",
    "greedy_color",
    "is_proper",
    "OracleInstance",
    "OracleRun",
    "philox4x32_10",
    "pt_exp",
    "heatbath",
    "swap_accept",
    "heatbath_count",
    "swap_count",
    "pt_exp_constants",
    "boltzmann",
]
