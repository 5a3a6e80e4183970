"""Greedy graph colouring of the physical graph (oracle side; test infrastructure).

The paper does not say how a sweep orders its spin updates.  Reading used:
spins are updated colour class by colour class, where the colouring is the
greedy one over the union of coupling edges and copy links: vertices in
ascending id, each taking the smallest colour not used by an already coloured
neighbour.  Spins of one class share no edge, so they can be updated together
without changing the result.
"""
from __future__ import annotations

import numpy as np


def greedy_color(n: int, cp_ptr, cp_col, lk_ptr, lk_col) -> tuple[np.ndarray, int]:
    color = np.full(n, -1, dtype=np.int32)
    for a in range(n):
        used = set()
        for k in range(cp_ptr[a], cp_ptr[a + 1]):
            b = cp_col[k]
            if b < a:
                used.add(int(color[b]))
        for k in range(lk_ptr[a], lk_ptr[a + 1]):
            b = lk_col[k]
            if b < a:
                used.add(int(color[b]))
        c = 0
        while c in used:
            c += 1
        color[a] = c
    n_colors = int(color.max()) + 1 if n else 0
    return color, n_colors


def is_proper(color, cp_ptr, cp_col, lk_ptr, lk_col) -> bool:
    n = len(color)
    for a in range(n):
        for k in range(cp_ptr[a], cp_ptr[a + 1]):
            if color[cp_col[k]] == color[a]:
                return False
        for k in range(lk_ptr[a], lk_ptr[a + 1]):
            if color[lk_col[k]] == color[a]:
                return False
    return True
