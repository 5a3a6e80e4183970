"""Brute-force Boltzmann distributions and KL divergence (test infrastructure).

For tiny instances (n <= ~22 physical spins) every state is enumerated, giving
the exact target of each replica slot (beta_i, P_j):
pi(s) proportional to exp(-beta_i (f(s) + P_j g(s)))      (Eq. 1, App. A)
and the empirical KL divergence D(p_hat || p) with 0 log 0 = 0 (App. B).
State index convention: bit a of the index is 1 iff spin a is +1.
"""
from __future__ import annotations

import numpy as np

from .sparsify import PhysInstance


def all_states(n: int) -> np.ndarray:
    idx = np.arange(1 << n, dtype=np.int64)
    bits = (idx[:, None] >> np.arange(n, dtype=np.int64)[None, :]) & 1
    return (2 * bits - 1).astype(np.int8)


def energies(inst: PhysInstance, S: np.ndarray):
    """Exact f (int64) and g (int64) of every row of S (states x n)."""
    S64 = S.astype(np.int64)
    f = np.zeros(S.shape[0], dtype=np.int64)
    for a in range(inst.n):
        for k in range(inst.cp_ptr[a], inst.cp_ptr[a + 1]):
            b = int(inst.cp_col[k])
            if b > a:
                f -= int(inst.cp_J[k]) * S64[:, a] * S64[:, b]
        if inst.h is not None:
            f -= int(inst.h[a]) * S64[:, a]
    g = np.zeros(S.shape[0], dtype=np.int64)
    for a in range(inst.n):
        for k in range(inst.lk_ptr[a], inst.lk_ptr[a + 1]):
            b = int(inst.lk_col[k])
            if b > a:
                g += (S[:, a] != S[:, b]).astype(np.int64)
    return f, g


def boltzmann(f: np.ndarray, g: np.ndarray, beta: float, P: int) -> np.ndarray:
    E = f.astype(np.float64) + float(P) * g.astype(np.float64)
    x = -float(beta) * (E - E.min())
    w = np.exp(x)
    return w / w.sum()


def kl(p_hat: np.ndarray, p: np.ndarray) -> float:
    """D(p_hat || p) = sum p_hat log(p_hat / p), with 0 log 0 = 0."""
    m = p_hat > 0
    return float(np.sum(p_hat[m] * np.log(p_hat[m] / p[m])))


def logical_energies(Jq: np.ndarray, h: np.ndarray | None = None):
    """Exact cost of every logical state of a dense int16 coupling matrix."""
    N = Jq.shape[0]
    S = all_states(N).astype(np.int64)
    Ji = np.triu(Jq.astype(np.int64), 1)
    f = -np.einsum("si,ij,sj->s", S, Ji, S)
    if h is not None:
        f -= S @ np.asarray(h, dtype=np.int64)
    return f
