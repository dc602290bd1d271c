"""Splitting one batch of independent LPs over several GPUs (one process per GPU).

LPs share nothing, so a batch shards without any data-path collective: each rank
solves the LPs of its own range and keeps its results.  For LPs of one size an equal
count per rank balances the work; for a mixed-size batch the ranks get contiguous
ranges of the batch sorted by estimated cost, cut where the running cost crosses
r / world of the total, so that every rank carries about the same work.

Cost model of one LP (host-side, from the sizes alone): a dense-tableau pivot
touches (m + 1)(n + 1) entries (Section 3.1, Step 3), and the pivots per LP grow
about linearly with the size (about 13 at m = n = 100 and 33 at m = n = 300 for the
type-1 workloads); the tableau build and the refinement add about as much as ten
pivots.  So cost(m, n) = (m + 1)(n + 1) (10 + 1 + min(m, n) / 8).
"""
from __future__ import annotations

import numpy as np


def lp_cost(m, n) -> np.ndarray:
    """Estimated relative cost of solving LPs of sizes m x n (arrays or scalars)."""
    m = np.asarray(m, dtype=np.float64)
    n = np.asarray(n, dtype=np.float64)
    return (m + 1.0) * (n + 1.0) * (11.0 + np.minimum(m, n) / 8.0)


def balanced_ranges(m, n, world: int):
    """Cost-balanced contiguous ranges of the size-sorted batch.

    Returns ``(order, bounds)``: ``order`` lists the LP indices by decreasing estimated
    cost (ties by index), and rank r solves ``order[bounds[r]:bounds[r + 1]]``.  The
    ranges are disjoint, cover the batch, and each cut sits where the running cost is
    closest to r / world of the total."""
    if world < 1:
        raise ValueError("world must be >= 1")
    cost = lp_cost(m, n)
    count = cost.size
    order = np.lexsort((np.arange(count), -cost))
    run = np.concatenate([[0.0], np.cumsum(cost[order])])
    total = run[-1]
    bounds = [0]
    for r in range(1, world):
        target = total * r / world
        k = int(np.searchsorted(run, target))
        if k > 0 and abs(run[k - 1] - target) <= abs(run[min(k, count)] - target):
            k -= 1
        bounds.append(min(max(k, bounds[-1]), count))
    bounds.append(count)
    return order, np.asarray(bounds, dtype=np.int64)


def rank_lps(m, n, rank: int, world: int) -> np.ndarray:
    """Indices (into the batch) of the LPs rank ``rank`` of ``world`` solves."""
    order, bounds = balanced_ranges(m, n, world)
    return order[bounds[rank]:bounds[rank + 1]]
