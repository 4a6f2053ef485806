"""Row-block condensation host logic (Sec. 2.1, Fig. 6) on CPU: the block sizes
and the schedule, the per-step sign of an arbitrary pivot row, the oracle-driven
schedule against the oracle sweep, and the driver with a host stand-in for the
device steps, in one process (all ranks emulated) and over gloo with 2 and 3
ranks."""
import itertools
import math
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import workloads
from oracle import core as oracle
from paper_1811_08057_gb300 import dist as ld_dist
from rowblock_reference import HostSteps, oracle_rowblock, paper_schedule


def test_counts_and_schedule():
    assert ld_dist.rowblock_counts(16, 4) == [4, 4, 4, 4]
    assert ld_dist.rowblock_counts(10, 4) == [3, 3, 2, 2]
    with pytest.raises(ValueError):
        ld_dist.rowblock_counts(3, 4)
    # Fig. 2: four ranks of four rows; each round every rank pivots once
    assert ld_dist.rowblock_schedule([4, 4, 4, 4])[:5] == [(0, 0), (1, 0), (2, 0), (3, 0), (0, 1)]
    assert ld_dist.rowblock_schedule([3, 2]) == [(0, 0), (1, 0), (0, 1)]
    assert ld_dist.rowblock_schedule([1, 1, 1]) == []
    for counts in ([5, 5, 4], [2], [7, 1, 3]):
        sch = ld_dist.rowblock_schedule(counts)
        assert sch == paper_schedule(counts)
        assert len(sch) == sum(counts) - len(counts)
        for p, c in enumerate(counts):  # every row but the last, in local order
            assert [i for q, i in sch if q == p] == list(range(c - 1))


def _swap_condense(A, k, l):
    """One step in the swap-to-boundary layout: position l refilled from m-1."""
    m = A.shape[0]
    r = A[k] / A[k, l]
    B = A - np.outer(A[:, l], r)
    B[:, l] = B[:, m - 1]
    return np.delete(B, k, axis=0)[:, :m - 1]


def test_step_sign_brute_force():
    rng = np.random.default_rng(4)
    for m in (2, 3, 4, 5, 6):
        A = rng.standard_normal((m, m))
        d = np.linalg.det(A)
        for k, l in itertools.product(range(m), range(m)):
            B = _swap_condense(A.copy(), k, l)
            p = A[k, l]
            got = abs(p) * ld_dist.step_sign(p, k, l, m) * np.linalg.det(B)
            assert got == pytest.approx(d, rel=1e-10), (m, k, l)


@pytest.mark.parametrize("counts", [[4, 4, 4, 4], [3, 2], [6, 5, 5], [1, 1], [9]])
def test_oracle_schedule_equals_oracle_sweep(counts):
    n = sum(counts)
    A = workloads.dense_gaussian(n, seed=30 + n) if n > 1 else np.array([[2.5]])
    s, l, _, _ = oracle_rowblock(A, counts)
    want = oracle.logdet(A)
    assert s == want.sign
    assert l == pytest.approx(want.logabs, rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("n,world", [(37, 4), (40, 1), (33, 3), (5, 5)])
def test_emulated_driver_matches_oracle_schedule(n, world):
    A = workloads.dense_gaussian(n, seed=n)
    At = torch.from_numpy(np.array(A))
    s, l, lab, piv = ld_dist.logdet_rowblock_emulated(At, world, steps=HostSteps())
    rs, rl, rlab, rpiv = oracle_rowblock(A, ld_dist.rowblock_counts(n, world))
    assert lab == rlab
    np.testing.assert_allclose(piv, rpiv, rtol=1e-11)
    assert s == rs
    assert l == pytest.approx(rl, rel=1e-12)
    assert torch.equal(At, torch.from_numpy(np.array(A)))  # input not modified


def test_emulated_driver_singular_and_sign():
    A = workloads.dense_gaussian(12, seed=2)
    A[:, 5] = A[:, 3]  # two equal columns: det = 0 up to rounding
    s, l, _, _ = ld_dist.logdet_rowblock_emulated(torch.from_numpy(A), 3, steps=HostSteps())
    assert s == 0.0 or l < -20
    Z = np.zeros((6, 6))
    Z[np.arange(6), np.arange(6)[::-1]] = 1.0  # anti-diagonal: det = -1
    s, l, _, _ = ld_dist.logdet_rowblock_emulated(torch.from_numpy(Z), 2, steps=HostSteps())
    assert s == -1.0 and abs(l) < 1e-15
    Zr = np.zeros((6, 6))
    Zr[1:, :] = np.eye(6)[1:]
    s, l, _, _ = ld_dist.logdet_rowblock_emulated(torch.from_numpy(Zr), 2, steps=HostSteps())
    assert s == 0.0 and l == -math.inf


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, n, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        A = torch.from_numpy(np.array(workloads.dense_gaussian(n, seed=77)))
        counts = ld_dist.rowblock_counts(n, world)
        r0 = sum(counts[:rank])
        mine = A[r0:r0 + counts[rank]].clone()
        q.put((rank,) + tuple(ld_dist.logdet_rowblock(mine, n, steps=HostSteps())))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,n", [(2, 31), (3, 40)])
def test_gloo_ranks_match_oracle_schedule(world, n):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=180) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    A = workloads.dense_gaussian(n, seed=77)
    rs, rl, rlab, rpiv = oracle_rowblock(A, ld_dist.rowblock_counts(n, world))
    for rank, s, l, lab, piv in out:
        assert lab == rlab
        np.testing.assert_allclose(piv, rpiv, rtol=1e-11)
        assert s == rs
        assert l == pytest.approx(rl, rel=1e-12)
