"""Partition of one problem's targets and chart nodes across ranks, one
process per GPU.

Targets are independent of one another, and so are chart nodes: each node's
Newton iteration reads only Phi and grad Phi at its own position, and a node
that has converged simply leaves the active set (Sec. 5).  A problem is
therefore split into contiguous ranges of the points' Morton order, one per
rank, with the mesh (sources, tiles, trees) replicated on every rank.  No rank
needs another rank's results, so evaluation and solve have no exchange step;
`gather` reassembles the shards in the caller's order only when one rank wants
the whole result.  Contiguous Morton ranges keep each rank's points spatially
compact, which keeps its target blocks small and its near/far split as good as
the single-GPU run's.

This module is host logic only (index bookkeeping); every evaluation still
runs in the library's kernels on each rank's GPU.
"""
from __future__ import annotations

import numpy as np


def _spread10(v: np.ndarray) -> np.ndarray:
    """Interleave the low 10 bits of v with two zero bits each."""
    v = v.astype(np.uint64) & np.uint64(0x3FF)
    v = (v | (v << np.uint64(16))) & np.uint64(0x030000FF)
    v = (v | (v << np.uint64(8))) & np.uint64(0x0300F00F)
    v = (v | (v << np.uint64(4))) & np.uint64(0x030C30C3)
    v = (v | (v << np.uint64(2))) & np.uint64(0x09249249)
    return v


def morton_keys(points: np.ndarray) -> np.ndarray:
    """30-bit Morton keys of points [n, 3] on a 1024^3 grid over their bounding box."""
    p = np.asarray(points, dtype=np.float64)
    if p.shape[0] == 0:
        return np.zeros(0, dtype=np.uint64)
    lo, hi = p.min(axis=0), p.max(axis=0)
    span = np.where(hi > lo, hi - lo, 1.0)
    q = np.clip(((p - lo) / span * 1024.0).astype(np.int64), 0, 1023)
    return _spread10(q[:, 0]) | (_spread10(q[:, 1]) << np.uint64(1)) | (_spread10(q[:, 2]) << np.uint64(2))


def morton_ranges(points: np.ndarray, nparts: int, align: int = 256) -> list[np.ndarray]:
    """Indices (into `points`) of nparts contiguous ranges of the Morton order.

    Range sizes are multiples of `align` (a target block of the pair kernels)
    except the last, and differ by at most one block; every point is in
    exactly one range, and each range lists its points in Morton order."""
    if nparts < 1:
        raise ValueError("nparts must be >= 1")
    n = int(np.asarray(points).shape[0])
    order = np.argsort(morton_keys(points), kind="stable")
    blocks = -(-n // align)
    cuts = [min(n, (blocks * k // nparts) * align) for k in range(nparts + 1)]
    cuts[-1] = n
    return [order[cuts[k]:cuts[k + 1]] for k in range(nparts)]


def chart_node_positions(verts: np.ndarray, tris: np.ndarray, tri: np.ndarray, uvw: np.ndarray) -> np.ndarray:
    """Starting points of chart nodes on the skeleton, P1 + u (P2 - P1) + v (P3 - P1),
    used only to order the nodes for partitioning."""
    t = np.asarray(tris)[np.asarray(tri)]
    v = np.asarray(verts)
    p1, p2, p3 = v[t[:, 0]], v[t[:, 1]], v[t[:, 2]]
    u, w = np.asarray(uvw)[:, 0:1], np.asarray(uvw)[:, 1:2]
    return p1 + u * (p2 - p1) + w * (p3 - p1)


def gather(dist, idx: np.ndarray, values: np.ndarray, n_total: int, dst: int = 0):
    """Reassemble per-rank results in the caller's order on rank `dst`.

    idx: this rank's indices into the whole problem; values: its results,
    one row per index.  Returns the full array on `dst` and None elsewhere.
    With dist None (one process) the values are scattered into place."""
    values = np.asarray(values)
    if dist is None:
        out = np.empty((n_total,) + values.shape[1:], dtype=values.dtype)
        out[idx] = values
        return out
    parts = [None] * dist.get_world_size() if dist.get_rank() == dst else None
    dist.gather_object((np.asarray(idx), values), parts, dst=dst)
    if dist.get_rank() != dst:
        return None
    out = np.empty((n_total,) + values.shape[1:], dtype=values.dtype)
    seen = np.zeros(n_total, dtype=bool)
    for i, v in parts:
        if seen[i].any():
            raise ValueError("shards overlap")
        seen[i] = True
        out[i] = v
    if not seen.all():
        raise ValueError("shards do not cover the problem")
    return out
