"""Splitting one ensemble over several GPUs and combining the shards.

Trajectories are independent (Sec. 1 and 2.2 of the QTM paper: the method is
"scale-free"), and every random draw is keyed by (seed, global trajectory id),
so an ensemble of `ntraj` trajectories can be cut into contiguous id ranges, one
per GPU, run with ``qtm_run_range`` and recombined: the result equals one run
over all ids.  The one exchange step is the sum of the per-shard FP64 sums --
the paper's master/worker averaging (Sec. 3) restated as a single all-reduce.
"""

from __future__ import annotations

import numpy as np


def shard(ntraj: int, world: int, rank: int):
    """Contiguous id range (first, count) of `rank` among `world` shards; the first
    ntraj % world ranks take one extra trajectory."""
    if world < 1 or not 0 <= rank < world or ntraj < 0:
        raise ValueError("need world >= 1, 0 <= rank < world, ntraj >= 0")
    base, extra = divmod(ntraj, world)
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def combine_sums(total_sum, total_sumsq, count):
    """Mean and standard error (sample variance, n - 1 divisor) from the summed
    per-shard sums of x and x^2 over `count` trajectories."""
    s1 = np.asarray(total_sum, dtype=np.float64)
    s2 = np.asarray(total_sumsq, dtype=np.float64)
    if count <= 0:
        return np.zeros_like(s1), np.zeros_like(s1)
    mean = s1 / count
    if count < 2:
        return mean, np.zeros_like(s1)
    var = np.maximum((s2 - s1 * mean) / (count - 1), 0.0)
    return mean, np.sqrt(var / count)
