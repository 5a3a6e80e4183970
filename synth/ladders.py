"""Inverse-temperature and penalty ladders for an I x J replica grid.

Rows carry increasing inverse temperatures beta_i and columns increasing
penalty strengths P_j (the paper's replica array, Fig. 1a).  Both are given in
the integer units of the quantised couplings: a physical beta is divided by the
quantisation scale, and P is an integer multiple-of-coupling value, so that the
penalised energy E_j = f + P_j g (Eq. 1) stays an exact integer.
"""
from __future__ import annotations

import numpy as np


def beta_ladder(I: int, beta_min: float, beta_max: float, scale: float = 1.0) -> np.ndarray:
    """Geometric ladder of I inverse temperatures, as float32 in coupling units."""
    if I < 1:
        raise ValueError("I must be >= 1")
    if I == 1:
        b = np.array([beta_max], dtype=np.float64)
    else:
        b = beta_min * (beta_max / beta_min) ** (np.arange(I) / (I - 1))
    return (b / scale).astype(np.float32)


def penalty_ladder(J: int, c_min: float, c_max: float, unit: int) -> np.ndarray:
    """Linear ladder of J integer penalties: rint(c * unit), c in [c_min, c_max]."""
    if J < 1:
        raise ValueError("J must be >= 1")
    if J == 1:
        c = np.array([c_max], dtype=np.float64)
    else:
        c = np.linspace(c_min, c_max, J)
    return np.rint(c * unit).astype(np.int32)
