"""Adaptive ladder schedule for 2D-PT (Algorithm 2 of the paper's appendix).

TEST INFRASTRUCTURE ONLY (part of the CPU oracle).  A plain restatement of the
schedule: the first column (penalty P0) grows rows, each new inverse
temperature one learning-rate step alpha_beta / sigma_E above the last, until
the energy standard deviation of a row's population falls to sigma_min or the
row cap is reached; each row also proposes the next column's penalty, one step
alpha_P / (beta sigma_g) above its own, and the next column takes the median
proposal.  Further columns repeat the row walk from beta0 at their penalty and
stop once the coldest row's population is feasible on average (mean g < 1/2)
or the column cap is reached.  The final beta ladder is the median over the
columns of each row's beta.

Readings where the pseudo-code is open (the same on the GPU side):
  * A population sample at (beta, P) is n_chain independent chains: n_chain
    runs of a 1 x 1 grid started from the INIT stream, `mcs` heat-bath sweeps
    each (one event of `mcs` sweeps, so no swap ever happens), with E = f + P g
    and g of each chain's final state.  Sample k (0, 1, 2, ... in the order the
    schedule draws them) uses seed + k and run ids 0 .. n_chain - 1.
  * sigma_E and sigma_g are population standard deviations over the chains
    (divide by n_chain), from exact integer sums: var = (n S2 - S1^2) / n^2 with
    the numerator rounded once to double, then sqrt; mean_g = S1 / n.
  * Every row of column j runs at that column's penalty P(j) (column 1: P0).
  * Penalties are integers: each new column's median is rounded to nearest.
  * The first column keeps rows 1 .. i, where i is the row at which sigma_E
    <= sigma_min stopped the walk, and at most max_rows rows.  Its proposals
    for column 2 come from the rows that stepped (sigma_E > sigma_min).
  * In later columns sigma_E is floored at sigma_min before the beta step (the
    first column's stopping rule already keeps it above that).
  * A row whose population has sigma_g = 0 makes no penalty proposal; when no
    row of a column proposes one, no further column is added.
  * The break test of a later column uses mean_g of its last (coldest) row;
    that column is kept.
  * Medians of an even count average the two middle values ((a + b) / 2).
Arithmetic is IEEE double in the order written here; beta is rounded to
float32 when it is sampled or returned.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class ScheduleParams:
    beta0: float          # first inverse temperature (coupling units)
    P0: int               # penalty of the first column (coupling units)
    max_rows: int         # I cap
    max_cols: int         # J cap
    sigma_min: float      # energy standard deviation at which the row walk stops
    alpha_beta: float     # learning rate of the beta steps
    alpha_P: float        # learning rate of the penalty steps
    n_chain: int          # population size
    mcs: int              # sweeps per population sample
    seed: int             # sample k uses seed + k


def int_to_double(v: int) -> float:
    """Round an exact integer to the nearest double (ties to even)."""
    return float(v)


def population_stats(E, g):
    """(sigma_E, sigma_g, mean_g) of one population, from exact integer sums."""
    E = [int(x) for x in E]
    g = [int(x) for x in g]
    n = len(E)
    s1, s2 = sum(E), sum(x * x for x in E)
    t1, t2 = sum(g), sum(x * x for x in g)
    nn = int_to_double(n * n)
    sig_E = math.sqrt(int_to_double(n * s2 - s1 * s1) / nn)
    sig_g = math.sqrt(int_to_double(n * t2 - t1 * t1) / nn)
    mean_g = int_to_double(t1) / int_to_double(n)
    return sig_E, sig_g, mean_g


def median(values):
    v = sorted(values)
    m = len(v)
    if m % 2:
        return v[m // 2]
    return (v[m // 2 - 1] + v[m // 2]) / 2


def adaptive_schedule(sampler, prm: ScheduleParams):
    """Algorithm 2.  `sampler(beta_f32, P_int, k)` returns the (E, g) arrays of
    population sample k.  Returns (beta float32 [I], P int32 [J], samples)."""
    k = 0

    def sample(beta, P):
        nonlocal k
        E, g = sampler(np.float32(beta), int(P), k)
        k += 1
        return population_stats(E, g)

    # first column, penalty P0: rows until sigma_E <= sigma_min or the cap
    cols_beta = []
    col = [prm.beta0]
    proposals = []
    i = 0
    while i < prm.max_rows:
        b = col[i]
        sig_E, sig_g, _ = sample(b, prm.P0)
        if sig_E > prm.sigma_min:
            if i + 1 < prm.max_rows:
                col.append(b + prm.alpha_beta / sig_E)
            if sig_g > 0:
                proposals.append(prm.P0 + prm.alpha_P / (b * sig_g))
            i += 1
        else:
            i += 1
            break
    I = len(col)
    cols_beta.append(col)
    P = [int(prm.P0)]
    # remaining columns
    while len(P) < prm.max_cols and proposals:
        P.append(int(round(median(proposals))))
        Pj = P[-1]
        col = [prm.beta0]
        proposals = []
        mean_g = 0.0
        for i in range(I):
            b = col[i]
            sig_E, sig_g, mean_g = sample(b, Pj)
            if i + 1 < I:
                col.append(b + prm.alpha_beta / max(sig_E, prm.sigma_min))
            if sig_g > 0:
                proposals.append(Pj + prm.alpha_P / (b * sig_g))
        cols_beta.append(col)
        if mean_g < 0.5:  # the coldest row of this column is feasible on average
            break
    beta = np.array([median([c[i] for c in cols_beta]) for i in range(I)], dtype=np.float32)
    return beta, np.array(P, dtype=np.int32), k


def oracle_sampler(oinst, prm: ScheduleParams):
    """Population samples from the oracle's 2D-PT loop (1 x 1 grid, n_chain runs)."""
    from .core import OracleRun

    def sampler(beta, P, k):
        orc = OracleRun(oinst, [beta], [P], list(range(prm.n_chain)), prm.seed + k)
        orc.run(prm.mcs, prm.mcs)
        f = orc.f[:, 0]
        g = orc.g[:, 0]
        return f + int(P) * g, g

    return sampler
