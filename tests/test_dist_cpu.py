"""Multi-rank host logic on CPU with world size 2 (gloo): batch sharding covers
every matrix once and balances cost; timings reduce to the slowest rank; the
gathered results equal a single-rank computation."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import workloads
from paper_1811_08057_gb300 import dist as ld_dist


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_lpt_partition_properties():
    sizes = workloads.batched_sizes(4096, seed=3)
    for world in [1, 2, 3, 8]:
        parts = ld_dist.lpt_partition(sizes, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(sizes)))
        loads = [sum(int(sizes[i]) ** 3 for i in p) for p in parts]
        assert max(loads) - min(loads) <= 512 ** 3  # within one largest matrix
    assert ld_dist.lpt_partition([5, 5], 1) == [[0, 1]]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sizes = [int(x) for x in workloads.batched_sizes(64, seed=5)]
        parts = ld_dist.lpt_partition(sizes, world)
        mine = parts[rank]
        # stand-in for the per-matrix results: a value only the owner computes
        vals = [float(np.log(sizes[i])) + i for i in mine]
        allv = ld_dist.gather_results(mine, vals, len(sizes))
        t = ld_dist.max_over_ranks(1.0 + rank)
        s = ld_dist.sum_over_ranks(float(len(mine)))
        q.put((rank, allv.numpy().tolist(), t, s))
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_sharding():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sizes = [int(x) for x in workloads.batched_sizes(64, seed=5)]
    want = [float(np.log(n)) + i for i, n in enumerate(sizes)]
    for rank, allv, t, s in out:
        assert np.allclose(allv, want)
        assert t == 2.0
        assert s == 64.0
