"""The multi-GPU host logic on CPU ranks (gloo, world size 2): each rank runs its
contiguous shard of trajectory ids with the oracle, the ranks all-reduce their
FP64 sums, and the combined ensemble equals one run over all ids -- the property
the GPU shards rely on (draws keyed by global trajectory id)."""

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1810_03047_gb300 import shards, systems as S


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, ntraj, out_path):
    import torch
    import torch.distributed as dist
    from oracle import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    prob = S.jaynes_cummings_driven()
    first, count = shards.shard(ntraj, world, rank)
    res = oracle.mcwf(prob, traj0=first, ntraj=count, nthreads=2)
    obs = res["obs"]
    sums = torch.tensor(np.concatenate([obs.sum(axis=0).ravel(), (obs ** 2).sum(axis=0).ravel(), [count]]),
                        dtype=torch.float64)
    dist.all_reduce(sums)
    if rank == 0:
        np.save(out_path, sums.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_shard_ranges_cover_the_ensemble():
    for ntraj in (0, 1, 7, 20000):
        for world in (1, 2, 3, 8):
            ranges = [shards.shard(ntraj, world, r) for r in range(world)]
            ids = [i for f, c in ranges for i in range(f, f + c)]
            assert ids == list(range(ntraj))


def test_two_rank_shards_equal_single_run(tmp_path):
    from oracle import oracle
    ntraj = 61
    out = str(tmp_path / "sums.npy")
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, ntraj, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    sums = np.load(out)
    prob = S.jaynes_cummings_driven()
    P = len(prob.t) * len(prob.A)
    count = int(sums[-1])
    assert count == ntraj
    mean, se = shards.combine_sums(sums[:P], sums[P:2 * P], count)
    ref = oracle.mcwf(prob, ntraj=ntraj)
    ref_mean, ref_se = oracle.ensemble(ref["obs"])
    np.testing.assert_allclose(mean, ref_mean.ravel(), rtol=0, atol=1e-12)
    np.testing.assert_allclose(se, ref_se.ravel(), rtol=0, atol=1e-9)
