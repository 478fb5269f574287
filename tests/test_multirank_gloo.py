"""The multi-GPU host logic on CPU ranks (gloo): each rank runs its contiguous
shard of trajectory ids with the oracle, turns its values into the library's
exact moment words (qtm_moments_of_values, the rule the GPU reduction applies),
the ranks all-reduce the words as int64, and the library's host combination
(qtm_combine_moments) gives the ensemble mean and standard error.  Integer sums
do not depend on the collective's order, so world sizes 1, 2 and 3 give the
same bits, equal to the combination of one run over all ids -- the property the
GPU shards rely on (draws keyed by global trajectory id, Sec. 3's two-level
average restated as one exact all-reduce)."""

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1810_03047_gb300 import shards, systems as S

NTRAJ = 61


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, ntraj, out_path):
    import torch
    import torch.distributed as dist
    from oracle import oracle
    from paper_1810_03047_gb300 import qtm as Q
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    prob = S.jaynes_cummings_driven()
    first, count = shards.shard(ntraj, world, rank)
    res = oracle.mcwf(prob, traj0=first, ntraj=count, nthreads=2)
    E = Q.qtm_scale_exponents(prob)
    words = torch.from_numpy(Q.qtm_moments_of_values(res["obs"], len(prob.A), E))
    n = torch.tensor([count], dtype=torch.int64)
    dist.all_reduce(words)
    dist.all_reduce(n)
    if rank == 0:
        mean, se, s1, s2 = Q.qtm_combine_moments(words.numpy(), [int(n.item())], len(prob.A), E)
        np.save(out_path, np.stack([mean, se, s1, s2]))
    dist.barrier()
    dist.destroy_process_group()


def _run_world(world, tmp_path):
    out = str(tmp_path / f"stats{world}.npy")
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, NTRAJ, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    return np.load(out)


def test_shard_ranges_cover_the_ensemble():
    for ntraj in (0, 1, 7, 20000):
        for world in (1, 2, 3, 8):
            ranges = [shards.shard(ntraj, world, r) for r in range(world)]
            ids = [i for f, c in ranges for i in range(f, f + c)]
            assert ids == list(range(ntraj))


def test_rank_shards_equal_single_run_bitwise(tmp_path):
    from oracle import oracle
    from paper_1810_03047_gb300 import qtm as Q
    got = {w: _run_world(w, tmp_path) for w in (1, 2, 3)}
    for w in (2, 3):
        np.testing.assert_array_equal(got[w], got[1])
    prob = S.jaynes_cummings_driven()
    ref = oracle.mcwf(prob, ntraj=NTRAJ)
    E = Q.qtm_scale_exponents(prob)
    one = Q.qtm_combine_moments(Q.qtm_moments_of_values(ref["obs"], len(prob.A), E), [NTRAJ], len(prob.A), E)
    np.testing.assert_array_equal(got[1], np.stack(one))
    # and the plain FP64 ensemble of the same trajectories to rounding
    ref_mean, ref_se = oracle.ensemble(ref["obs"])
    np.testing.assert_allclose(got[1][0], ref_mean.ravel(), rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(got[1][1], ref_se.ravel(), rtol=1e-11, atol=1e-15)
