"""The N > 1 path of bench.py on CPU with gloo ranks (world size 2): each rank takes its own
block of LPs from one seeded stream (weak scaling, no data-path collective), the blocks are
disjoint and together equal the single-process batch, and the step time reported is the
maximum over ranks."""
import os

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
import synth


def _worker(rank, world, port, count, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lo, hi = bench.rank_range(rank, count)
    sb = synth.type1(hi, 6, 5, seed=bench.SEED, first=lo, stop=hi)
    np.save(os.path.join(out_dir, f"A{rank}.npy"), sb.A)
    t = torch.tensor([float(rank + 1)], dtype=torch.float64)    # this rank's "step time"
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    np.save(os.path.join(out_dir, f"t{rank}.npy"), t.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_the_batch(tmp_path):
    world, count = 2, 300
    port = 29500 + (os.getpid() % 1000)
    mp.start_processes(_worker, args=(world, port, count, str(tmp_path)), nprocs=world, start_method="spawn")
    whole = synth.type1(world * count, 6, 5, seed=bench.SEED)
    parts = [np.load(tmp_path / f"A{r}.npy") for r in range(world)]
    assert all(p.size == count * 30 for p in parts)
    assert np.array_equal(np.concatenate(parts), whole.A)
    for r in range(world):
        assert float(np.load(tmp_path / f"t{r}.npy")[0]) == float(world)


def _shard_worker(rank, world, port, out_dir):
    from paper_1609_08114_gb300 import shard
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sb = synth.mixed_sizes(20000, seed=4, first=0, stop=2000)     # sizes only are needed
    mine = shard.rank_lps(sb.m, sb.n, rank, world)
    cost = float(shard.lp_cost(sb.m[mine], sb.n[mine]).sum())
    got = [None] * world
    dist.all_gather_object(got, (mine.tolist(), cost))
    if rank == 0:
        np.save(os.path.join(out_dir, "parts.npy"), np.array([np.array(g[0]) for g in got], dtype=object),
                allow_pickle=True)
        np.save(os.path.join(out_dir, "costs.npy"), np.array([g[1] for g in got]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_cost_balanced_mixed_batch(tmp_path):
    """A mixed-size batch (m, n ~ U{8..256}) split over two gloo ranks by estimated cost:
    the ranges are disjoint, cover the batch, and carry equal cost within the largest
    single LP's cost."""
    from paper_1609_08114_gb300 import shard
    world = 2
    port = 29500 + (os.getpid() % 1000) + 7
    mp.start_processes(_shard_worker, args=(world, port, str(tmp_path)), nprocs=world, start_method="spawn")
    parts = np.load(tmp_path / "parts.npy", allow_pickle=True)
    costs = np.load(tmp_path / "costs.npy")
    allidx = np.concatenate([np.asarray(p, dtype=np.int64) for p in parts])
    assert np.array_equal(np.sort(allidx), np.arange(2000))
    sb = synth.mixed_sizes(20000, seed=4, first=0, stop=2000)
    biggest = float(shard.lp_cost(sb.m, sb.n).max())
    assert abs(costs[0] - costs[1]) <= biggest
    assert len(parts[0]) < len(parts[1])        # the larger LPs come first: fewer of them on rank 0


def test_balanced_ranges_host_logic():
    from paper_1609_08114_gb300 import shard
    rng = np.random.default_rng(0)
    for world in (1, 2, 3, 4, 8):
        m = rng.integers(1, 300, size=997)
        n = rng.integers(1, 300, size=997)
        order, bounds = shard.balanced_ranges(m, n, world)
        assert bounds[0] == 0 and bounds[-1] == 997 and np.all(np.diff(bounds) >= 0)
        assert np.array_equal(np.sort(order), np.arange(997))
        cost = shard.lp_cost(m, n)
        per = np.array([cost[order[bounds[r]:bounds[r + 1]]].sum() for r in range(world)])
        assert per.max() - per.min() <= 2 * cost.max()
    # one size: equal counts
    order, bounds = shard.balanced_ranges(np.full(1000, 100), np.full(1000, 100), 4)
    assert list(np.diff(bounds)) == [250, 250, 250, 250]
    assert list(order[:5]) == [0, 1, 2, 3, 4]
