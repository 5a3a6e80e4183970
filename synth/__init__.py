"""Seeded synthetic inputs for two-dimensional parallel tempering (2D-PT).

This package produces the *workloads* only: planted Wishart Ising instances
(the problem class the paper's ground-state experiments use, Section
"Ground-state optimization under constraints", citing Hamze et al. 2020),
one-hot constrained colouring problems, temperature / penalty ladders and
request-arrival streams.  It holds none of
the method's arithmetic (no sparsification, colouring, sweeps or swaps), so
both the CPU oracle and the GPU library can consume the same inputs without
sharing any method code.
"""
from .wishart import WishartInstance, wishart_planted
from .ladders import beta_ladder, penalty_ladder
from .arrivals import batch_specs, poisson_arrivals, request_specs
from .constrained import ColoringProblem, colouring, random_cubic_graph, slack_coefficients

__all__ = [
    "WishartInstance",
    "wishart_planted",
    "beta_ladder",
    "penalty_ladder",
    "poisson_arrivals",
    "request_specs",
    "batch_specs",
    "ColoringProblem",
    "colouring",
    "random_cubic_graph",
    "slack_coefficients",
]
