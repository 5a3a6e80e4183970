"""Planted Wishart Ising instances with integer (int16) couplings.

Construction (the paper uses planted Wishart instances with density
alpha = M/N, Section "Ground-state optimization under constraints"; the
ensemble is Hamze et al. 2020):

* a planted configuration t in {-1,+1}^N;
* M = round(alpha*N) Gaussian columns z_mu, each projected orthogonal to t:
  w_mu = z_mu - t (t . z_mu) / N, so that W^T t = 0;
* couplings J = -W W^T / N with the diagonal set to zero.

With the Ising cost f(s) = -sum_{i<j} J_ij s_i s_j one has
f(s) = |W^T s|^2 / (2N) - sum_{i,mu} W_{i mu}^2 / (2N) >= f(t), so t is a
ground state of the real-valued instance.  The couplings are then quantised
to int16 at the scale s_q = 32767 / max|J_ij| (round half to even), which
makes every local field and energy an exact integer.  Quantisation may move
the ground state; ``E_planted`` is the exact integer cost of t under the
quantised couplings.
"""
from __future__ import annotations

import dataclasses

import numpy as np

QMAX = 32767


@dataclasses.dataclass(frozen=True)
class WishartInstance:
    N: int
    M: int
    alpha: float
    seed: int
    t: np.ndarray  # int8 [N], planted configuration
    J: np.ndarray  # float64 [N, N], real-valued couplings (zero diagonal)
    Jq: np.ndarray  # int16 [N, N], quantised couplings (zero diagonal)
    scale: float  # Jq ~= J * scale
    E_planted: int  # exact int64 cost of t under Jq
    E_planted_real: float  # cost of t under J (closed form -sum W^2 / 2N)
    W: np.ndarray  # float64 [N, M]

    @property
    def degrees(self) -> np.ndarray:
        return (self.Jq != 0).sum(axis=1)


def _num_patterns(N: int, alpha: float) -> int:
    return max(1, int(np.floor(alpha * N + 0.5)))


def wishart_planted(N: int, alpha: float, seed: int, qmax: int = QMAX) -> WishartInstance:
    """Generate one planted Wishart instance (see module docstring)."""
    if N < 2:
        raise ValueError("N must be >= 2")
    rng = np.random.Generator(np.random.Philox(int(seed)))
    M = _num_patterns(N, alpha)
    t = np.where(rng.random(N) < 0.5, -1, 1).astype(np.int8)
    Z = rng.standard_normal((N, M))
    tf = t.astype(np.float64)
    W = Z - np.outer(tf, tf @ Z) / N
    J = -(W @ W.T) / N
    np.fill_diagonal(J, 0.0)
    jmax = float(np.abs(J).max())
    if jmax == 0.0:
        raise ValueError("degenerate instance (all couplings zero)")
    scale = qmax / jmax
    Jq = np.rint(J * scale).astype(np.int64)
    Jq = np.clip(Jq, -qmax, qmax).astype(np.int16)
    # Integer cost of the planted state: -sum_{i<j} Jq_ij t_i t_j.
    Ji = Jq.astype(np.int64)
    ti = t.astype(np.int64)
    E_planted = -int(ti @ Ji @ ti) // 2
    E_planted_real = -float((W * W).sum()) / (2.0 * N)
    return WishartInstance(
        N=N,
        M=M,
        alpha=float(alpha),
        seed=int(seed),
        t=t,
        J=J,
        Jq=Jq,
        scale=scale,
        E_planted=E_planted,
        E_planted_real=E_planted_real,
        W=W,
    )
