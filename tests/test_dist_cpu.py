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


def _slogdet_standin(mats, mode):
    """Host stand-in for the per-rank batched call (LAPACK slogdet)."""
    out = [np.linalg.slogdet(np.asarray(A)) for A in mats]
    return [float(o[0]) for o in out], [float(o[1]) for o in out]


def _sharded_worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sizes = [int(x) for x in workloads.batched_sizes(48, seed=6)]
        mats = workloads.batched_covariances(sizes, seed=6)
        mats[5] = -mats[5]  # some negative determinants (odd sizes flip the sign)
        mats[7][:, 3] = 0.0  # one singular matrix
        touched = []

        def get(i):
            touched.append(i)
            return mats[i]
        s, l = ld_dist.logdet_batched_distributed(sizes, get, compute=_slogdet_standin)
        q.put((rank, sorted(touched), s.numpy().tolist(), l.numpy().tolist()))
    finally:
        dist.destroy_process_group()


def test_two_rank_sharded_batch_matches_one_rank():
    """Each rank sweeps only its LPT share; the gathered (sign, log|det|) vectors
    equal the one-rank result element by element, singular matrix included."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_sharded_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sizes = [int(x) for x in workloads.batched_sizes(48, seed=6)]
    mats = workloads.batched_covariances(sizes, seed=6)
    mats[5] = -mats[5]
    mats[7][:, 3] = 0.0
    want_s, want_l = _slogdet_standin(mats, "f32_plain")
    parts = ld_dist.lpt_partition(sizes, 2)
    for rank, touched, s, l in out:
        assert touched == parts[rank]  # a rank builds only its own share
        assert s == want_s
        assert all((a == b) or (np.isinf(a) and np.isinf(b) and a == b) for a, b in zip(l, want_l))
