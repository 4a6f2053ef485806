"""Multi-rank plumbing (one process per GPU).

A single matrix's sweep does not shard without a per-pivot broadcast of the
pivot row (the paper's Fig. 6 design for MPI), so single-matrix runs are
replicas. A batch of independent matrices shards with no data-path collective:
each rank takes a share of the matrices chosen by longest-processing-time order
on the n^3 cost and sweeps it with its own launch; only timings (and, if wanted,
the per-matrix results) are combined.
"""
from __future__ import annotations

import heapq

import torch
import torch.distributed as dist


def lpt_partition(sizes, world: int):
    """Indices of a batch split over `world` ranks, balancing sum(n^3):
    largest first, each to the currently lightest rank. Deterministic."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]) ** 3, i))
    heap = [(0, r) for r in range(world)]
    parts = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + int(sizes[i]) ** 3, r))
    return [sorted(p) for p in parts]


def world_info():
    if dist.is_available() and dist.is_initialized():
        return dist.get_rank(), dist.get_world_size()
    return 0, 1


def max_over_ranks(x: float, device=None) -> float:
    """Largest value of x over all ranks (the job's time is its slowest rank's)."""
    _, world = world_info()
    if world == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t[0])


def sum_over_ranks(x: float, device=None) -> float:
    _, world = world_info()
    if world == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t[0])


def gather_results(indices, values, count: int, device=None):
    """Scatter each rank's (indices, values) into one length-`count` FP64 tensor
    on every rank (the only exchange, after the timed work)."""
    out = torch.zeros(count, dtype=torch.float64, device=device)
    if len(indices):
        out[torch.as_tensor(indices, dtype=torch.long, device=device)] = torch.as_tensor(
            values, dtype=torch.float64, device=device)
    _, world = world_info()
    if world > 1:
        dist.all_reduce(out, op=dist.ReduceOp.SUM)
    return out


def logdet_batched_distributed(sizes, get_matrix, mode="f32_plain", compute=None, device=None):
    """sign and log|det| of a batch of independent matrices sharded over the ranks.

    Every rank passes the whole batch's `sizes`; `get_matrix(i)` returns matrix i
    on this rank's device and is called only for this rank's share (longest
    processing time first on the n^3 cost, `lpt_partition`). Each rank sweeps its
    share in one ld_logdet_batched call (`compute(mats, mode)` replaces that call,
    e.g. in host-only tests); the (sign, log|det|) pairs are then combined once,
    so every rank returns both full FP64 vectors (length len(sizes)) in batch
    order. No collective runs inside the sweep.
    """
    rank, world = world_info()
    mine = lpt_partition(sizes, world)[rank]
    if compute is None:
        from . import api

        def compute(mats, mode):
            s, l = api.logdet_batched(api.BatchedInputs(mats), mode)
            return s, l
    if mine:
        signs, logabs = compute([get_matrix(i) for i in mine], mode)
        signs = torch.as_tensor(signs, dtype=torch.float64).to(device).tolist()
        logabs = torch.as_tensor(logabs, dtype=torch.float64).to(device).tolist()
    else:
        signs, logabs = [], []
    return (gather_results(mine, signs, len(sizes), device=device),
            gather_results(mine, logabs, len(sizes), device=device))
