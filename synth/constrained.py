"""Seeded constrained problems with one-hot groups: graph colouring as an Ising
cost plus a constraint function g >= 0 (Eq. 1 with a general g).

Colouring of a random cubic graph with k colours: spin (v, c) = v * k + c is
+1 when vertex v takes colour c.  The cost counts the weight of edges whose
ends share a colour, F = sum_{(u,v)} w_uv sum_c x_uc x_vc with
x = (1 + s) / 2.  Multiplying by 4 gives integer Ising terms:
    4 F = k W + sum_{(u,v),c} w_uv s_uc s_vc + sum_{u,c} s_uc sum_{v~u} w_uv,
so with couplings J_{uc,vc} = -w_uv and fields h_uc = -sum_{v~u} w_uv the
library's cost f = -sum J s s - sum h s equals 4 F - k W.  A proper colouring
is f = -k W.  The one-hot groups {v*k .. v*k+k-1} say every vertex takes
exactly one colour; the constraint function is their squared residual, which
each side expands with its own routine.

This module only builds inputs (graph, weights, groups); it holds none of
2D-PT's arithmetic.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class ColoringProblem:
    V: int                   # vertices
    k: int                   # colours
    edges: np.ndarray        # int32 [E][2], u < v
    w: np.ndarray            # int32 [E] edge weights
    cp_ptr: np.ndarray       # coupling CSR over n = V k spins
    cp_col: np.ndarray
    cp_J: np.ndarray         # int16
    h: np.ndarray            # int32 [n]
    groups: list             # one-hot groups (spin ids)
    W: int                   # total edge weight
    f_proper: int            # f of any proper colouring (-k W)

    @property
    def n(self) -> int:
        return self.V * self.k

    def same_colour_weight(self, f):
        """F = (f + k W) / 4 for a feasible state's cost f."""
        return (np.asarray(f, np.int64) + self.k * self.W) // 4


def random_cubic_graph(V: int, seed: int) -> np.ndarray:
    """Simple 3-regular graph from the pairing model (stubs paired at random,
    redrawn until there is no loop and no repeated edge).  V even."""
    if V % 2 or V < 4:
        raise ValueError("V must be even and >= 4")
    rng = np.random.default_rng(seed)
    stubs = np.repeat(np.arange(V, dtype=np.int64), 3)
    for _ in range(10000):
        p = rng.permutation(stubs).reshape(-1, 2)
        u, v = np.minimum(p[:, 0], p[:, 1]), np.maximum(p[:, 0], p[:, 1])
        if np.any(u == v):
            continue
        key = u * V + v
        if np.unique(key).size != key.size:
            continue
        order = np.argsort(key)
        return np.stack([u[order], v[order]], 1).astype(np.int32)
    raise RuntimeError("pairing model did not give a simple graph")


def colouring(V: int, k: int, seed: int, w_max: int = 1) -> ColoringProblem:
    """k-colouring of a random cubic graph on V vertices, edge weights uniform
    on 1..w_max (1: plain colouring)."""
    edges = random_cubic_graph(V, seed)
    rng = np.random.default_rng(seed + 1)
    w = rng.integers(1, w_max + 1, edges.shape[0]).astype(np.int32)
    n = V * k
    rows = [[] for _ in range(n)]
    h = np.zeros(n, np.int64)
    for (u, v), we in zip(edges.tolist(), w.tolist()):
        for c in range(k):
            a, b = u * k + c, v * k + c
            rows[a].append((b, -we))
            rows[b].append((a, -we))
            h[a] -= we
            h[b] -= we
    ptr = np.zeros(n + 1, np.int32)
    col, J = [], []
    for a in range(n):
        for b, j in sorted(rows[a]):
            col.append(b)
            J.append(j)
        ptr[a + 1] = len(col)
    W = int(w.sum())
    groups = [list(range(v * k, v * k + k)) for v in range(V)]
    return ColoringProblem(V, k, edges, w, ptr, np.array(col, np.int32), np.array(J, np.int16),
                           h.astype(np.int32), groups, W, -k * W)


def slack_coefficients(b: int):
    """Coefficients 1, 2, ..., 2^(T-1), b + 1 - 2^T (T = floor(log2(b + 1)); a
    zero last term dropped) of slack spins whose subset sums are exactly
    0..b, which turn an inequality sum A x <= b into an equality."""
    b = int(b)
    if b < 0:
        raise ValueError("negative bound")
    T = (b + 1).bit_length() - 1
    c = [1 << t for t in range(T)]
    if b + 1 - (1 << T) > 0:
        c.append(b + 1 - (1 << T))
    return c
