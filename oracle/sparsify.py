"""Copy-chain graph sparsification (oracle side; test infrastructure).

Section "Graph sparsification with copy constraints": a compiler maps each
logical node to a chain of physical copies and distributes the node's
neighbours among them; copies are tied by copy constraints
g = sum over chain links (S_a - S_b)^2, equivalent to a ferromagnetic
coupling between consecutive copies.  Fig. 2a uses two copies per node, the
Wishart experiments three copies per node.

Readings used here (the paper gives no assignment rule):
* logical node i with K_i copies owns physical ids offset_i + c, c = 0..K_i-1,
  chained c <-> c+1;
* the neighbours j of i (nonzero couplings) are taken in ascending order and
  dealt round-robin over the copies, skipping a copy whose edge capacity is
  full; logical edge (i, j) becomes one physical coupling between the copy of i
  that received j and the copy of j that received i, with the same J_ij;
* copy counts: ``fixed`` K copies (uncapped); ``max_edges`` m (K = ceil(d/m),
  at most m original edges per copy); ``max_degree`` D (total physical degree
  including chain links <= D: one copy if d <= D, else the smallest K with
  2(D-1) + (K-2)(D-2) >= d, chain ends holding <= D-1 edges and interior
  copies <= D-2).
g counts broken links, g = sum (s_a - s_b)^2 / 4, so g = 0 iff every chain agrees.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class PhysInstance:
    n: int
    cp_ptr: np.ndarray  # int32 [n+1]
    cp_col: np.ndarray  # int32 [nnz]
    cp_J: np.ndarray  # int16 [nnz]
    lk_ptr: np.ndarray  # int32 [n+1]
    lk_col: np.ndarray  # int32 [2*links]
    h: np.ndarray | None  # int32 [n] or None
    N: int  # logical spins
    copy_of: np.ndarray  # int32 [n] logical id of each physical spin
    offset: np.ndarray  # int32 [N+1] first physical id of each chain
    # general penalty terms g = g0 + sum_links K [s_a != s_b] + sum_a k_a [s_a = -1]
    # (None / 0: copy constraints, K = 1, k = 0)
    lk_w: np.ndarray | None = None  # int16 [2*links] weight K of each link entry
    hk: np.ndarray | None = None  # int32 [n] penalty field k
    g0: int = 0

    @property
    def n_links(self) -> int:
        return int(self.lk_col.size // 2)


def _copies(d: int, rule: str, param: int) -> tuple[int, list[int | None]]:
    if rule == "fixed":
        K = int(param)
        return K, [None] * K
    if rule == "max_edges":
        m = int(param)
        K = max(1, math.ceil(d / m))
        return K, [m] * K
    if rule == "max_degree":
        D = int(param)
        if d <= D:
            return 1, [D]
        if D < 3:
            raise ValueError("max_degree rule needs D >= 3 for chains")
        K = 2
        while 2 * (D - 1) + (K - 2) * (D - 2) < d:
            K += 1
        caps = [D - 1] + [D - 2] * (K - 2) + [D - 1]
        return K, caps
    raise ValueError(f"unknown rule {rule!r}")


def sparsify(Jq: np.ndarray, rule: str, param: int) -> PhysInstance:
    """Copy-chain sparsify a dense symmetric int16 logical coupling matrix."""
    Jq = np.asarray(Jq)
    N = Jq.shape[0]
    nbrs = [[j for j in range(N) if j != i and Jq[i, j] != 0] for i in range(N)]
    Ks = []
    caps = []
    for i in range(N):
        K, cap = _copies(len(nbrs[i]), rule, param)
        Ks.append(K)
        caps.append(cap)
    offset = np.zeros(N + 1, dtype=np.int64)
    offset[1:] = np.cumsum(Ks)
    n = int(offset[-1])
    # which copy of i receives neighbour j
    copy_for = [dict() for _ in range(N)]
    for i in range(N):
        K = Ks[i]
        load = [0] * K
        c = 0
        for j in nbrs[i]:
            tries = 0
            while caps[i][c] is not None and load[c] >= caps[i][c]:
                c = (c + 1) % K
                tries += 1
                if tries > K:
                    raise RuntimeError("copy capacities exhausted")
            copy_for[i][j] = c
            load[c] += 1
            c = (c + 1) % K
    adj = [dict() for _ in range(n)]
    for i in range(N):
        for j in nbrs[i]:
            if j <= i:
                continue
            a = int(offset[i] + copy_for[i][j])
            b = int(offset[j] + copy_for[j][i])
            adj[a][b] = int(Jq[i, j])
            adj[b][a] = int(Jq[i, j])
    links = [[] for _ in range(n)]
    for i in range(N):
        for c in range(Ks[i] - 1):
            a = int(offset[i] + c)
            links[a].append(a + 1)
            links[a + 1].append(a)
    cp_ptr = np.zeros(n + 1, dtype=np.int32)
    cols, vals = [], []
    for a in range(n):
        for b in sorted(adj[a]):
            cols.append(b)
            vals.append(adj[a][b])
        cp_ptr[a + 1] = len(cols)
    lk_ptr = np.zeros(n + 1, dtype=np.int32)
    lcols = []
    for a in range(n):
        lcols.extend(sorted(links[a]))
        lk_ptr[a + 1] = len(lcols)
    copy_of = np.repeat(np.arange(N, dtype=np.int32), Ks)
    return PhysInstance(
        n=n,
        cp_ptr=cp_ptr,
        cp_col=np.asarray(cols, dtype=np.int32),
        cp_J=np.asarray(vals, dtype=np.int16),
        lk_ptr=lk_ptr,
        lk_col=np.asarray(lcols, dtype=np.int32),
        h=None,
        N=N,
        copy_of=copy_of,
        offset=offset.astype(np.int32),
    )


def lift(inst: PhysInstance, sigma: np.ndarray) -> np.ndarray:
    """Physical state with every copy of logical i set to sigma_i (g = 0)."""
    return np.asarray(sigma, dtype=np.int8)[inst.copy_of]


def project(inst: PhysInstance, s: np.ndarray) -> np.ndarray:
    """Logical state read from the first copy of each chain."""
    return np.asarray(s, dtype=np.int8)[inst.offset[:-1]]
