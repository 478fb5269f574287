"""Splitting one ensemble over several GPUs and combining the shards.

Trajectories are independent (Sec. 1 and 2.2 of the QTM paper: the method is
"scale-free"), and every random draw is keyed by (seed, global trajectory id),
so an ensemble of `ntraj` trajectories can be cut into contiguous id ranges, one
per GPU, run with ``qtm_run_range`` and recombined: the result equals one run
over all ids.  The one exchange step is an integer sum of the shards' exact
moment words (``qtm_moments_device``, then ``qtm_combine_moments``) -- the
paper's master/worker averaging (Sec. 3) restated as a single all-reduce whose
result does not depend on the order in which the collective adds.
"""

from __future__ import annotations


def shard(ntraj: int, world: int, rank: int):
    """Contiguous id range (first, count) of `rank` among `world` shards; the first
    ntraj % world ranks take one extra trajectory."""
    if world < 1 or not 0 <= rank < world or ntraj < 0:
        raise ValueError("need world >= 1, 0 <= rank < world, ntraj >= 0")
    base, extra = divmod(ntraj, world)
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)
