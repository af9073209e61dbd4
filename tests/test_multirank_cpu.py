"""Multi-GPU sharding logic on CPU ranks (gloo, world size 2).

The path shards with no data exchange: rank r of N solves p_A rows r, r+N, ...
of a 362N x 362 grid (bench.km_slice).  Two gloo ranks check that their
slices partition the global grid exactly, carry equal system counts and the
same cost mix (p_A distribution), and that the whole-job aggregate of the
timing line (max time over ranks, summed steps) is formed as bench.py does.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    sl = bench.km_slice(world, rank, m=362, n_phases=1)
    pa = torch.from_numpy(sl["phys"]["pA1"])
    f = torch.from_numpy(sl["phys"]["f1"])
    # global indices of this rank's systems in the 362N x 362 grid
    row = np.rint(sl["phys"]["pA1"][::362] / 2.0e5 * (362 * world - 1)).astype(np.int64)
    gathered = [torch.zeros(362, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(gathered, torch.from_numpy(row.astype(np.int64)))
    # aggregate as bench.py does: max time, summed steps
    tt = torch.tensor([float(rank + 1), float(pa.numel())], dtype=torch.float64)
    mx = tt.clone()
    dist.all_reduce(mx[0:1], op=dist.ReduceOp.MAX)
    dist.all_reduce(tt[1:2], op=dist.ReduceOp.SUM)
    if rank == 0:
        np.save(os.path.join(out_dir, "rows.npy"), torch.stack(gathered).numpy())
        np.save(os.path.join(out_dir, "agg.npy"), np.array([float(mx[0]), float(tt[1])]))
        np.save(os.path.join(out_dir, "pa0.npy"), pa.numpy())
    if rank == 1:
        np.save(os.path.join(out_dir, "pa1.npy"), pa.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharding_partitions_the_grid(tmp_path):
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    rows = np.load(tmp_path / "rows.npy")
    allrows = np.sort(rows.ravel())
    assert np.array_equal(allrows, np.arange(362 * world))      # exact partition, no overlap
    assert rows.shape == (world, 362)
    pa0, pa1 = np.load(tmp_path / "pa0.npy"), np.load(tmp_path / "pa1.npy")
    assert pa0.size == pa1.size == 362 * 362
    # interleaved rows: the two shards see the same driving distribution
    assert abs(pa0.mean() - pa1.mean()) / pa0.mean() < 0.01
    agg = np.load(tmp_path / "agg.npy")
    assert agg[0] == 2.0 and agg[1] == 2 * 362 * 362
