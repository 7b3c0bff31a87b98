"""The several-GPU path's host logic on CPU ranks (gloo, world size 2 and 3).

The problems of a run are independent cells; each rank solves its share with
no data-path exchange. What the ranks do share is tested here without a GPU:
the shares, the barrier and maximum of the per-rank times, and gathering the
per-cell results onto rank 0 in cell order.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as tmp

from paper_2312_15554_gb300 import shard as SH


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, n_units, out_dir):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dev = torch.device("cpu")
    mine = SH.shard(n_units, rank, world)
    # stand-in per-cell results: a 3x3 "K" that encodes the cell index
    rows = np.stack([np.full((3, 3), float(c)) + np.eye(3) for c in mine]) if len(mine) else np.zeros((0, 3, 3))
    SH.barrier(dist)
    t = SH.max_over_ranks(10.0 * (rank + 1), dist, dev)
    total = SH.sum_over_ranks(len(mine), dist, dev)
    full = SH.gather_rows(rows, n_units, dist, dev, world)
    if rank == 0:
        np.savez(os.path.join(out_dir, "r0.npz"), t=t, total=total, full=full)
    dist.destroy_process_group()


@pytest.mark.parametrize("world,n_units", [(2, 7), (3, 3), (3, 2)])
def test_ranks_share_cells_time_by_the_slowest_and_gather_in_order(tmp_path, world, n_units):
    port = _free_port()
    tmp.spawn(_worker, args=(world, port, n_units, str(tmp_path)), nprocs=world, join=True)
    r = np.load(tmp_path / "r0.npz")
    assert float(r["t"]) == 10.0 * world
    assert float(r["total"]) == n_units
    full = r["full"]
    assert full.shape == (n_units, 3, 3)
    for c in range(n_units):
        np.testing.assert_array_equal(full[c], np.full((3, 3), float(c)) + np.eye(3))


def test_shards_are_disjoint_balanced_and_complete():
    for world in (1, 2, 3, 4, 8):
        for n in (0, 1, 5, 8, 384, 385):
            parts = [SH.shard(n, r, world) for r in range(world)]
            flat = [u for p in parts for u in p]
            assert flat == list(range(n))
            sizes = [len(p) for p in parts]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        SH.shard(4, 2, 2)


def test_single_process_is_the_identity():
    rows = np.arange(12.0).reshape(4, 3)
    assert SH.max_over_ranks(3.5, None, None) == 3.5
    np.testing.assert_array_equal(SH.gather_rows(rows, 4, None, None, 1), rows)
