"""Seeded request streams for the serving workload.

A request is one constrained Ising problem (a planted Wishart instance to be
copy-chain sparsified) with its own replica grid and stopping rule.  Arrival
times follow a Poisson process with a given rate (requests per minute).
"""
from __future__ import annotations

import numpy as np


def poisson_arrivals(rate_per_min: float, duration_s: float, seed: int) -> np.ndarray:
    """Arrival times in seconds of a Poisson process on [0, duration_s)."""
    rng = np.random.Generator(np.random.Philox(int(seed)))
    lam = rate_per_min / 60.0
    times = []
    t = 0.0
    while True:
        t += rng.exponential(1.0 / lam)
        if t >= duration_s:
            break
        times.append(t)
    return np.asarray(times, dtype=np.float64)


def request_specs(count: int, seed: int, n_min: int = 50, n_max: int = 800,
                  alpha_min: float = 0.25, alpha_max: float = 0.75):
    """Per-request (N, alpha, instance seed), drawn uniformly."""
    rng = np.random.Generator(np.random.Philox(int(seed) + 7919))
    Ns = rng.integers(n_min, n_max + 1, size=count)
    alphas = rng.uniform(alpha_min, alpha_max, size=count)
    seeds = rng.integers(1, 2**31 - 1, size=count)
    return [(int(n), float(a), int(s)) for n, a, s in zip(Ns, alphas, seeds)]


def batch_specs(count: int, seed: int, n_min: int = 50, n_max: int = 400,
                alphas=(0.25, 0.5, 0.75)):
    """Per-instance (N, alpha, instance seed) for a batch of uneven instances:
    N uniform on {n_min..n_max}, alpha uniform on the given set."""
    rng = np.random.Generator(np.random.Philox(int(seed) + 104729))
    Ns = rng.integers(n_min, n_max + 1, size=count)
    al = rng.choice(np.asarray(alphas, dtype=np.float64), size=count)
    return [(int(n), float(a), int(seed) + i) for i, (n, a) in enumerate(zip(Ns, al))]
