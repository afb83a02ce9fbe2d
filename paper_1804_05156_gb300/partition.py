"""Host-side sharding of assembly work over ranks (one GPU per rank, no collective on the data path).

Row ownership, for one mesh: rank r owns a contiguous range of vertex ids [lo, hi) (ranges balanced by
incidence count), takes every element with a vertex in its range (elements on the cut are taken by
every rank they touch) and assembles the sub-mesh those elements span. The sub-mesh keeps the global
order of vertices and elements (local ids ascend with global ids), so each owned row of the local
matrix has the same columns in the same order as the global row, and every entry sums the same
element contributions in the same (ascending element) order: the owned rows are the global rows, bit
for bit, and the ranks never exchange data.

Cost partition, for a batch of independent meshes: longest-processing-time-first on the element counts.
"""
from __future__ import annotations

import numpy as np


def row_ranges(N: int, P: int, elem: np.ndarray | None = None) -> list[tuple[int, int]]:
    """P contiguous vertex ranges covering [0, N). With `elem`, the cuts balance the number of incident
    (element, vertex) pairs per range; otherwise the vertex counts."""
    if P < 1:
        raise ValueError("P must be >= 1")
    if elem is None or N == 0:
        cuts = [round(N * r / P) for r in range(P + 1)]
    else:
        deg = np.bincount(np.asarray(elem, dtype=np.int64).ravel(), minlength=N)
        cum = np.concatenate([[0], np.cumsum(deg)])
        total = cum[-1]
        cuts = [0] + [int(np.searchsorted(cum, total * r / P, side="left")) for r in range(1, P)] + [N]
        cuts = [min(max(c, 0), N) for c in cuts]
        for r in range(1, P + 1):
            cuts[r] = max(cuts[r], cuts[r - 1])
    return [(int(cuts[r]), int(cuts[r + 1])) for r in range(P)]


def shard_mesh(elem: np.ndarray, lo: int, hi: int) -> dict:
    """The sub-mesh of rank owning vertices [lo, hi).

    Returns elem_ids (global ids of the taken elements, ascending), vert_ids (global ids of the
    sub-mesh's vertices, ascending; local id = position), elem_local (the taken elements in local
    vertex ids) and owned_local (local ids of the owned vertices, ascending)."""
    elem = np.asarray(elem)
    take = np.any((elem >= lo) & (elem < hi), axis=1)
    elem_ids = np.nonzero(take)[0]
    sub = elem[elem_ids]
    vert_ids, inv = np.unique(sub.ravel(), return_inverse=True)
    elem_local = inv.reshape(sub.shape).astype(np.int32)
    owned_local = np.nonzero((vert_ids >= lo) & (vert_ids < hi))[0]
    return {"elem_ids": elem_ids, "vert_ids": vert_ids, "elem_local": elem_local, "owned_local": owned_local}


def owned_rows(shard: dict, row_ptr: np.ndarray, col_idx: np.ndarray, val: np.ndarray, b: np.ndarray | None = None):
    """Extract the owned rows of a sub-mesh assembly in global numbering: (rows, row_len, cols, vals, b)."""
    rp = np.asarray(row_ptr, dtype=np.int64)
    own = shard["owned_local"]
    lens = rp[own + 1] - rp[own]
    idx = np.concatenate([np.arange(rp[r], rp[r + 1]) for r in own]) if len(own) else np.zeros(0, np.int64)
    cols = shard["vert_ids"][np.asarray(col_idx)[idx]]
    out_b = None if b is None else np.asarray(b)[own]
    return shard["vert_ids"][own], lens, cols, np.asarray(val)[idx], out_b


def cost_partition(costs, P: int) -> list[list[int]]:
    """Assign items with the given costs to P ranks, largest first onto the least-loaded rank (ties by
    rank id); each rank's list is returned in ascending item order."""
    if P < 1:
        raise ValueError("P must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0] * P
    parts: list[list[int]] = [[] for _ in range(P)]
    for i in order:
        r = min(range(P), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += costs[i]
    return [sorted(p) for p in parts]
