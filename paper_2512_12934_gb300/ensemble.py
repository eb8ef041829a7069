"""Partition of an ensemble of independent LBM instances over ranks.

Instances of an ensemble never exchange data, so running one on several
GPUs needs no collective on the data path: each rank (one process per GPU)
steps its own share as one batch, and only the timing and, where wanted,
the per-instance results are gathered afterwards.  Shares are balanced by
work (fluid nodes, the unit every lattice update costs) with the
longest-processing-time rule: instances in decreasing order of work, each
to the rank with the least work so far (ties to the lower rank, so every
rank computes the same partition without communicating).
"""


def partition(work, world):
    """Instance indices of each of `world` ranks: a list of `world` sorted
    lists that together hold every index of `work` exactly once."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(work)), key=lambda i: (-work[i], i))
    load = [0] * world
    shares = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        shares[r].append(i)
        load[r] += work[i]
    return [sorted(s) for s in shares]


def share_of(work, world, rank):
    """The instance indices rank `rank` steps."""
    return partition(work, world)[rank]
