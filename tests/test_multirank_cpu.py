"""Multi-GPU sharding logic on CPU ranks (gloo, world size 2).

The path shards with no data exchange: rank r of N solves p_A rows r, r+N, ...
of a 362N x 362 grid (workloads.shard_rows, used by bench.km_slice).  Two gloo
ranks check that

  * their slices partition the global grid exactly, carry equal system counts
    and the same cost mix (p_A distribution), and that the whole-job aggregate
    of the timing line (max time over ranks, summed steps) is formed as
    bench.py does;
  * solving each shard separately and concatenating the results gives the
    unsharded solve bit for bit: every rank runs the oracle on its shard of a
    small Keller-Miksis grid, rank 0 gathers the accessories, final states and
    step counts and places them by global index.
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


# small grid of the sharded solve: M_PA x M_F systems, a few phases
M_PA, M_F, PHASES = 10, 12, 3


def _oracle_solve(w):
    import oracle
    ph = w["phys"]
    C = oracle.km_coefficients(ph["pA1"], ph["f1"], ph["pA2"], ph["f2"], ph["theta"], ph["RE"],
                               oracle.liquid(**w["liquid"]))
    t = w["tol"]
    tol = oracle.make_tol(rtol=t.rtol, atol=t.atol, dt0=t.dt0, dt_min=t.dt_min, dt_max=t.dt_max,
                          n_phases=t.n_phases, phase_len=t.phase_len, t0=t.t0)
    return oracle.cashkarp_solve(oracle.KM, C, w["y0"], tol, nthreads=1)


def _solve_worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2011_01740_gb300 import workloads as W
    full = W.km(M_PA, M_F, n_phases=PHASES)
    idx = W.shard_rows(M_PA, M_F, world, rank)
    r = _oracle_solve(W.take(full, idx))
    # one float64 row per system: global index, accessories, state, step counts
    local = np.concatenate([idx[None, :].astype(np.float64), r["acc"], r["y"],
                            r["nacc"][None, :].astype(np.float64), r["nrej"][None, :].astype(np.float64)])
    # shards differ in size when world does not divide M_PA: pad to the largest
    size = torch.tensor([local.shape[1]], dtype=torch.int64)
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(sizes, size)
    width = int(max(s.item() for s in sizes))
    buf = torch.full((local.shape[0], width), float("nan"), dtype=torch.float64)
    buf[:, :local.shape[1]] = torch.from_numpy(local)
    parts = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf)
    if rank == 0:
        cat = np.concatenate([p.numpy()[:, :int(s.item())] for p, s in zip(parts, sizes)], axis=1)
        np.save(os.path.join(out_dir, f"sharded_{world}.npy"), cat)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_solves_concatenate_to_the_unsharded_solve(tmp_path, world):
    """Each rank solves only its rows; placed by global index, the gathered
    accessories, final states and step counts equal the one-process solve of
    the whole grid bitwise (the systems share nothing, so no result may depend
    on which rank or which other systems ran it).  World 3 leaves the ranks
    with unequal row counts (10 rows)."""
    mp.start_processes(_solve_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    from paper_2011_01740_gb300 import workloads as W
    cat = np.load(tmp_path / f"sharded_{world}.npy")
    gidx = cat[0].astype(np.int64)
    assert np.array_equal(np.sort(gidx), np.arange(M_PA * M_F))
    order = np.argsort(gidx)
    ref = _oracle_solve(W.km(M_PA, M_F, n_phases=PHASES))
    rows = 2 * PHASES
    got_acc = cat[1:1 + rows][:, order]
    got_y = cat[1 + rows:3 + rows][:, order]
    got_nacc, got_nrej = cat[3 + rows][order], cat[4 + rows][order]
    assert np.array_equal(got_acc, ref["acc"])
    assert np.array_equal(got_y, ref["y"])
    assert np.array_equal(got_nacc, ref["nacc"].astype(np.float64))
    assert np.array_equal(got_nrej, ref["nrej"].astype(np.float64))
    assert np.all(ref["status"] == 0)
