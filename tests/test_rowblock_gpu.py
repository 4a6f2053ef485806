"""Row-block condensation (Sec. 2.1, Fig. 6) through ld_rowblock_factor /
ld_rowblock_update on one GPU: with one rank it is the plain sweep (pivot on
the first active row), pivots and labels bit for bit the oracle's; with several
ranks emulated in one process (arbitrary pivot rows, ragged blocks) the pivots
and labels equal the oracle-driven schedule bit for bit in FP64; FP32 within
the plain sweep's tolerance."""
import math

import numpy as np
import pytest
import torch

import workloads
from oracle import core as oracle
from paper_1811_08057_gb300 import _lib
from paper_1811_08057_gb300 import dist as ld_dist
from rowblock_reference import oracle_rowblock

pytestmark = pytest.mark.gpu


def test_one_rank_is_the_plain_sweep():
    n = 700
    A = workloads.dense_gaussian(n, seed=91)
    s, l, lab, piv = ld_dist.logdet_rowblock(torch.from_numpy(A).cuda(), n)
    ref = oracle.logdet(A)
    assert lab == [int(x) for x in ref.piv_label[:n - 1]]
    assert piv == [float(x) for x in ref.piv_value[:n - 1]]
    assert s == ref.sign
    assert l == pytest.approx(ref.logabs, rel=1e-13)


@pytest.mark.parametrize("n,world", [(999, 4), (512, 8), (130, 3)])
def test_emulated_ranks_fp64_bitwise(n, world):
    A = workloads.dense_gaussian(n, seed=n + world)
    s, l, lab, piv = ld_dist.logdet_rowblock_emulated(torch.from_numpy(A).cuda(), world)
    rs, rl, rlab, rpiv = oracle_rowblock(A, ld_dist.rowblock_counts(n, world))
    assert lab == rlab
    assert piv == rpiv
    assert s == rs
    assert l == pytest.approx(rl, rel=1e-13)


def test_emulated_ranks_fp32():
    n, world = 600, 3
    A = workloads.dense_gaussian(n, seed=5)
    s, l, _, _ = ld_dist.logdet_rowblock_emulated(
        torch.from_numpy(A).to(torch.float32).cuda(), world)
    ref = oracle.logdet(A.astype(np.float32).astype(np.float64))
    assert s == ref.sign
    assert l == pytest.approx(ref.logabs, rel=2e-5)


def test_equal_to_boundary_and_singular():
    Z = np.zeros((8, 8))
    Z[np.arange(8), np.arange(8)[::-1]] = 2.0  # det = 2^8 (sign +: 4 swaps)
    s, l, _, _ = ld_dist.logdet_rowblock_emulated(torch.from_numpy(Z).cuda(), 4)
    assert s == 1.0 and l == pytest.approx(8 * math.log(2.0), rel=1e-15)
    Z[2, :] = 0.0  # a zero pivot row: singular
    s, l, _, _ = ld_dist.logdet_rowblock_emulated(torch.from_numpy(Z).cuda(), 4)
    assert s == 0.0 and l == -math.inf


def test_entry_points_reject_bad_arguments():
    row = torch.zeros(4, dtype=torch.float64, device="cuda")
    lab = torch.arange(4, dtype=torch.int32, device="cuda")
    step = torch.zeros(4, dtype=torch.float64, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    assert _lib.ld_rowblock_factor(0, _lib.LD_DTYPE_F64, lab.data_ptr(), 4, step.data_ptr(), s) \
        == _lib.LD_ERR_INVALID_ARG
    assert _lib.ld_rowblock_factor(row.data_ptr(), _lib.LD_DTYPE_F64, lab.data_ptr(), 0,
                                   step.data_ptr(), s) == _lib.LD_ERR_INVALID_ARG
    F = torch.zeros((2, 4), dtype=torch.float64, device="cuda")
    assert _lib.ld_rowblock_update(F.data_ptr(), _lib.LD_DTYPE_F64, 2, 3, 4, row.data_ptr(),
                                   lab.data_ptr(), step.data_ptr(), s) == _lib.LD_ERR_INVALID_ARG
    assert _lib.ld_rowblock_update(F.data_ptr(), 7, 2, 4, 4, row.data_ptr(),
                                   lab.data_ptr(), step.data_ptr(), s) == _lib.LD_ERR_INVALID_ARG
