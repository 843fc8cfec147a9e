"""Root-range sharding of one count over several GPUs (one process per GPU).

The Discussion proposes distributing the method by sending chunks of BFS
roots to different devices.  By Lemma 1 every connected k-set is counted
from exactly one root (its lowest-rank member), so contiguous rank ranges
that cover [0, n) split the sets into disjoint parts and the per-vertex
counts of the parts add up to the full count.  Each rank counts its range
with ``vdmc_count_roots`` on a replica of the graph, then one uint64
sum-reduce combines the partial counts (sums of uint64 counts are carried as
int64 two's-complement additions, which are the same bits).

The degree order puts the heavy roots first, so the ranges are cut at equal
*estimated work* (``vdmc_root_costs``), not at equal numbers of roots.

The partition and the reduce are host logic: ``partition_costs`` and
``reduce_partial`` need no GPU and are exercised with gloo ranks on CPU.
"""
from __future__ import annotations

import ctypes

import numpy as np

__all__ = ["partition_costs", "root_costs", "partition", "reduce_partial", "count_sharded"]


def partition_costs(costs, parts: int) -> list:
    """Cut ranks 0..n-1 into `parts` contiguous ranges of about equal total cost.

    Returns bounds b[0] = 0 <= b[1] <= ... <= b[parts] = n; range i is
    [b[i], b[i+1]).  Cut i is the first rank at which the inclusive cost sum
    reaches i/parts of the total, so each range holds at most 1/parts of the
    total plus one root.  Deterministic: every rank computes the same bounds.
    """
    if parts < 1:
        raise ValueError("parts must be >= 1")
    c = np.asarray(costs, dtype=np.uint64)
    n = int(c.size)
    cum = np.cumsum(c, dtype=np.uint64)
    total = int(cum[-1]) if n else 0
    bounds = [0]
    for i in range(1, parts):
        target = (total * i + parts - 1) // parts
        b = int(np.searchsorted(cum, np.uint64(target), side="left")) + 1 if total else (n * i) // parts
        bounds.append(min(n, max(bounds[-1], b)))
    bounds.append(n)
    return bounds


def root_costs(g, k: int, stream=None) -> np.ndarray:
    """Per-rank work estimates of graph g (host uint64[n])."""
    import torch
    from . import vdmc
    cost = torch.zeros(max(g.n, 1), dtype=torch.int64, device="cuda")
    st = vdmc._lib().vdmc_root_costs(g.handle, int(k), ctypes.c_void_p(cost.data_ptr()), vdmc._stream_ptr(stream))
    vdmc._check(st, "vdmc_root_costs")
    return cost[:g.n].cpu().numpy().view(np.uint64)


def partition(g, k: int, parts: int) -> list:
    """Rank bounds of `parts` ranges of equal estimated work for graph g."""
    return partition_costs(root_costs(g, k), parts)


def reduce_partial(partial, dist, group=None):
    """Sum the ranks' partial per-vertex counts in place (uint64 viewed as int64)."""
    import torch
    t = partial.view(torch.int64) if partial.dtype == torch.uint64 else partial
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return partial


def count_sharded(g, k: int, out, bounds, rank: int, dist, group=None, stream=None):
    """This rank's share of vdmc_count(g, k): its range's counts, then the sum over ranks.

    On return `out` (uint64[n, C_k]) holds the full count on every rank."""
    from . import vdmc
    vdmc.count_roots(g, k, bounds[rank], bounds[rank + 1], out, stream=stream)
    return reduce_partial(out, dist, group)
