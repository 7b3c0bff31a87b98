"""Host-side logic of running many independent unit-cell problems on several GPUs.

The unit-cell problems (cells x load directions, Section 2) are independent:
one process per GPU takes a contiguous share of the cells and solves them with
no exchange on the data path. The only collectives are on the host side of a
run: the barrier and the maximum of the per-rank times that bracket a timed
region, and gathering the per-cell results (K, iteration counts) onto rank 0.

Every function takes the process group module (`torch.distributed`) or None
for a single process, and the device the reduction tensors live on (a CUDA
device under NCCL, the CPU under gloo).
"""
from __future__ import annotations

import numpy as np


def shard(n_units: int, rank: int, world: int) -> range:
    """Contiguous share of units [0, n_units) of one rank; shares differ in size
    by at most one and cover every unit once."""
    if world < 1 or not 0 <= rank < world or n_units < 0:
        raise ValueError("bad shard arguments")
    q, r = divmod(n_units, world)
    start = rank * q + min(rank, r)
    return range(start, start + q + (1 if rank < r else 0))


def barrier(dist) -> None:
    if dist is not None:
        dist.barrier()


def max_over_ranks(x: float, dist, device) -> float:
    """The largest of one float per rank (the time of a bracketed region)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, dist, device) -> float:
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def gather_rows(rows: np.ndarray, n_units: int, dist, device, world: int):
    """Per-unit results of every rank (rows [len(shard)][...] in shard order) in
    unit order on rank 0; None on the other ranks."""
    rows = np.asarray(rows, dtype=np.float64)
    if dist is None:
        return rows
    import torch
    rank = dist.get_rank()
    width = int(np.prod(rows.shape[1:])) if rows.ndim > 1 else 1
    most = max(len(shard(n_units, r, world)) for r in range(world))
    buf = torch.zeros((most, width), dtype=torch.float64, device=device)
    mine = torch.as_tensor(rows.reshape(len(rows), width), device=device)
    buf[:len(rows)] = mine
    parts = [torch.zeros_like(buf) for _ in range(world)] if rank == 0 else None
    if rank == 0:
        dist.gather(buf, gather_list=parts, dst=0)
    else:
        dist.gather(buf, dst=0)
    if rank != 0:
        return None
    out = np.concatenate([parts[r][:len(shard(n_units, r, world))].cpu().numpy() for r in range(world)])
    return out.reshape((n_units,) + rows.shape[1:])
