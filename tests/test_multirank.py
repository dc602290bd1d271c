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
