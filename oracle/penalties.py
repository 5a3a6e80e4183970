"""Penalty terms of one-hot and linear equality constraints for the oracle
(test infrastructure).

A constraint function g >= 0 of Eq. 1 in the links form the oracle evaluates:
    g(s) = g0 + sum_{links a<b} K_ab [s_a != s_b] + sum_a k_a [s_a = -1].
For a one-hot group c of m spins (binary x_a = [s_a = +1]), expand
(sum_a x_a - 1)^2 with x_a = 1 - y_a, y_a = [s_a = -1]:
    (m - 1 - sum y)^2 = (m-1)^2 - 2(m-1) sum y + sum y + 2 sum_{a<b} y_a y_b,
and 2 y_a y_b = y_a + y_b - [s_a != s_b], so the pair sum is
(m - 1) sum y - sum_{a<b} [s_a != s_b].  Hence g0 += (m-1)^2, k_a += 2 - m,
K_ab += -1 for every pair of the group.

A linear equality constraint sum_{a in c} A_a x_a = b generalises this: with
S = sum_a A_a the residual is (S - b) - sum_a A_a y_a, and squaring it,
    (S - b)^2 - 2 (S - b) sum_a A_a y_a + sum_a A_a^2 y_a + 2 sum_{a<b} A_a A_b y_a y_b,
where the pair sum is sum_a A_a (S - A_a) y_a - sum_{a<b} A_a A_b [s_a != s_b].
Collecting the y_a terms: g0 += (S - b)^2, k_a += A_a (2b - S),
K_ab += -A_a A_b.  One-hot is A = 1, b = 1.
"""
from __future__ import annotations

import numpy as np


def onehot(n: int, groups):
    """(lk_ptr, lk_col, lk_w, hk, g0) of g = sum_c (sum_{a in c} x_a - 1)^2."""
    K = [dict() for _ in range(n)]
    hk = np.zeros(n, np.int64)
    g0 = 0
    for grp in groups:
        m = len(grp)
        g0 += (m - 1) ** 2
        for a in grp:
            hk[a] += 2 - m
            for b in grp:
                if b != a:
                    K[a][b] = K[a].get(b, 0) - 1
    ptr, col, w = [0], [], []
    for a in range(n):
        for b in sorted(K[a]):
            if K[a][b] != 0:
                col.append(b)
                w.append(K[a][b])
        ptr.append(len(col))
    return (np.array(ptr, np.int32), np.array(col, np.int32), np.array(w, np.int16),
            hk.astype(np.int32), int(g0))


def equality(n: int, constraints):
    """(lk_ptr, lk_col, lk_w, hk, g0) of g = sum_c (sum_{a in c} A_a x_a - b_c)^2
    for constraints given as (spin ids, coefficients A, b)."""
    K = [dict() for _ in range(n)]
    hk = [0] * n
    g0 = 0
    for ids, coef, b in constraints:
        ids = [int(a) for a in ids]
        coef = [int(c) for c in coef]
        b = int(b)
        S = sum(coef)
        g0 += (S - b) ** 2
        for a, A in zip(ids, coef):
            hk[a] += A * (2 * b - S)
            for bb, B in zip(ids, coef):
                if bb != a:
                    K[a][bb] = K[a].get(bb, 0) - A * B
    ptr, col, w = [0], [], []
    for a in range(n):
        for b in sorted(K[a]):
            if K[a][b] != 0:
                if not -32768 <= K[a][b] <= 32767:
                    raise ValueError("link weight outside int16")
                col.append(b)
                w.append(K[a][b])
        ptr.append(len(col))
    if any(not -2 ** 31 <= k < 2 ** 31 for k in hk):
        raise ValueError("penalty field outside int32")
    return (np.array(ptr, np.int32), np.array(col, np.int32), np.array(w, np.int16),
            np.array(hk, np.int32), int(g0))

