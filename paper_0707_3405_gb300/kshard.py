"""k-point sharding across processes, one GPU each (Sec. 5.2: the k-points of a
cell are independent, so the outermost level of the paper's three-level
parallelisation needs no communication during the eigensolve).

Every rank builds its own handle over its share of the k-points (the
potential is replicated, the projectors of a k-point exist only on the rank
that owns it), solves them, and the eigenvalues and residual norms are
gathered once at the end.  No collective runs on the data path; the gather
moves nk x M doubles twice.

Host-side helpers only: the partition and the gather (``torch.distributed``,
any backend).
"""
from __future__ import annotations

import numpy as np

__all__ = ["partition", "gather_results"]


def partition(nk: int, world_size: int, cost=None) -> list:
    """Split k-point indices 0..nk-1 over ``world_size`` ranks.

    ``cost`` (optional, length nk) weighs each k-point (e.g. its plane-wave
    count); k-points are dealt largest first to the least loaded rank (ties to
    the lowest rank), so uneven spheres spread evenly.  Each rank's list is
    ascending.  Every k-point goes to exactly one rank; ranks beyond nk get
    none.
    """
    if nk < 0 or world_size < 1:
        raise ValueError("need nk >= 0 and world_size >= 1")
    c = np.ones(nk) if cost is None else np.asarray(cost, dtype=np.float64)
    if c.shape != (nk,):
        raise ValueError("cost must have one entry per k-point")
    order = sorted(range(nk), key=lambda k: (-c[k], k))
    load = np.zeros(world_size)
    out = [[] for _ in range(world_size)]
    for k in order:
        r = int(np.argmin(load))
        out[r].append(k)
        load[r] += c[k]
    return [sorted(x) for x in out]


def gather_results(local: dict, nk: int, world_size: int) -> tuple:
    """Assemble per-k results on every rank.

    ``local`` maps each k-point this rank solved to ``(eig, resid)`` (1-D arrays
    of equal length M).  Returns ``(eig, resid)`` of shape (nk, M), row k from the
    rank that owns k.  Raises if a k-point is missing or owned twice.
    """
    items = {int(k): (np.asarray(e, dtype=np.float64), np.asarray(r, dtype=np.float64))
             for k, (e, r) in local.items()}
    if world_size > 1:
        import torch.distributed as dist
        allp = [None] * world_size
        dist.all_gather_object(allp, items)
    else:
        allp = [items]
    seen = {}
    for part in allp:
        for k, v in part.items():
            if k in seen:
                raise RuntimeError(f"k-point {k} was solved by two ranks")
            seen[k] = v
    if sorted(seen) != list(range(nk)):
        raise RuntimeError(f"k-points missing from the gather: {sorted(set(range(nk)) - set(seen))}")
    M = len(seen[0][0]) if nk else 0
    eig = np.zeros((nk, M))
    res = np.zeros((nk, M))
    for k in range(nk):
        eig[k], res[k] = seen[k]
    return eig, res
