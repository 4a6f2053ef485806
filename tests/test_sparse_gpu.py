"""Sparse matrices on the GPU (ld_logdet_sparse) against the FP64 oracle.

The matrices are block upper triangular up to random row and column
permutations, with irreducible diagonal blocks of mixed sizes: blocks of up to
512 and of 513..1024 go through the two persistent batched launches, larger
ones through the single-matrix sweep in the caller's mode. The reference is the
oracle's condensation of the whole dense matrix (FP64 modes within 1e-12
relative, FP32 modes within 1e-5 on the same FP32 values), or the exact
Leibniz determinant for small integer matrices.
"""
import math
from fractions import Fraction

import numpy as np
import pytest
import torch

import oracle
import workloads
from oracle import exact
from paper_1811_08057_gb300 import api

pytestmark = pytest.mark.gpu

SIZES = [1, 1, 3, 7, 40, 1, 200, 600, 5, 1100, 2, 90]
TOL = {"f64_plain": 1e-12, "f64_blocked": 1e-12, "f64_ozaki": 1e-12, "f32_plain": 1e-5,
       "f32_3xtf32": 1e-5}


def rel(a, b):
    return abs(a - b) / max(abs(b), 1.0)


def run(rp, ci, v, mode, device="cuda"):
    s, l = api.logdet_sparse(torch.from_numpy(rp).to(device), torch.from_numpy(ci).to(device),
                             torch.from_numpy(v).to(device), mode)
    return float(s), float(l)


@pytest.fixture(scope="module")
def mixed():
    rp, ci, v, D = workloads.sparse_block_triangular(SIZES, seed=21)
    ref = oracle.logdet(D, nthreads=8)
    v32 = v.astype(np.float32)
    D32 = np.zeros_like(D)
    R = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    D32[R, ci] = v32.astype(np.float64)
    ref32 = oracle.logdet(D32, nthreads=8)
    return rp, ci, v, v32, ref, ref32


@pytest.mark.parametrize("mode", sorted(TOL))
def test_mixed_block_sizes_against_dense_oracle(mixed, mode):
    rp, ci, v, v32, ref, ref32 = mixed
    if mode.startswith("f64"):
        s, l = run(rp, ci, v, mode)
        want = ref
    else:
        s, l = run(rp, ci, v32, mode)
        want = ref32
    print(f"sparse n={len(rp) - 1} {mode}: rel err {rel(l, want.logabs):.2e}")
    assert s == want.sign
    assert rel(l, want.logabs) <= TOL[mode], (mode, l, want.logabs)


def test_stored_diagonal_structure():
    """Rows and columns permuted alike keep the diagonal stored: the identity
    transversal, the same blocks, the same determinant as the dense oracle."""
    rp, ci, v, D = workloads.sparse_block_triangular([3, 50, 1, 700, 20], seed=41,
                                                     symmetric=True)
    cor, blk, nb = api.sparse_blocks(torch.from_numpy(rp), torch.from_numpy(ci))
    assert np.array_equal(cor.numpy(), np.arange(len(rp) - 1)) and nb == 5
    ref = oracle.logdet(D, nthreads=8)
    for mode in ("f64_plain", "f64_ozaki"):
        s, l = run(rp, ci, v, mode)
        assert s == ref.sign and rel(l, ref.logabs) <= 1e-12


def test_host_and_device_arrays_agree(mixed):
    rp, ci, v, v32, ref, ref32 = mixed
    on_gpu = run(rp, ci, v, "f64_plain", "cuda")
    s, l = api.logdet_sparse(torch.from_numpy(rp), torch.from_numpy(ci), torch.from_numpy(v),
                             "f64_plain")
    assert (float(s), float(l)) == on_gpu


@pytest.mark.parametrize("seed", range(8))
def test_small_integer_matrices_exact(seed):
    """Small integer matrices: the sign exactly and log|det| within 1e-12 of the
    exact (Leibniz) determinant; a zero determinant gives sign 0, or a residue
    below 1e-12 where FP64 divisions rounded."""
    rng = np.random.default_rng(seed)
    sizes = [int(x) for x in rng.integers(1, 4, size=2)]  # n <= 6 (Leibniz)
    rp, ci, v, D = workloads.sparse_block_triangular(sizes, seed=200 + seed, off_density=0.1,
                                                     integer=True)
    det = exact.leibniz_det([[Fraction(int(x)) for x in row] for row in D])
    s, l = run(rp, ci, v, "f64_plain")
    if det == 0:
        # an exact zero, or the FP64 rounding residue of one
        assert s == 0.0 or l < math.log(1e-12)
        return
    assert s == (1.0 if det > 0 else -1.0)
    assert abs(l - math.log(abs(det))) <= 1e-12 * max(1.0, abs(math.log(abs(det))))


def test_singular_cases():
    # no stored entry at all (empty column and value arrays)
    z = np.zeros(0, dtype=np.int64)
    assert run(np.zeros(4, dtype=np.int64), z, np.zeros(0), "f64_plain") == (0.0, -math.inf)
    # no complete transversal: det A = 0 for every value of the entries
    D = np.array([[1.0, 0, 0], [2.0, 0, 0], [1.0, 1.0, 1.0]])
    R, C = np.nonzero(D)
    rp = np.concatenate([[0], np.cumsum(np.bincount(R, minlength=3))]).astype(np.int64)
    assert run(rp, C.astype(np.int64), D[R, C], "f64_plain") == (0.0, -math.inf)
    # a complete transversal but a numerically singular diagonal block
    D = np.array([[1.0, 2.0, 0], [2.0, 4.0, 0], [0, 5.0, 3.0]])
    R, C = np.nonzero(D)
    rp = np.concatenate([[0], np.cumsum(np.bincount(R, minlength=3))]).astype(np.int64)
    assert run(rp, C.astype(np.int64), D[R, C], "f64_plain") == (0.0, -math.inf)


def test_empty_and_diagonal():
    z = np.zeros(0, dtype=np.int64)
    assert run(np.zeros(1, dtype=np.int64), z, np.zeros(0), "f64_plain") == (1.0, 0.0)
    d = np.array([2.0, -0.5, 3.0, -1.0, 7.0])
    rp = np.arange(6, dtype=np.int64)
    ci = np.arange(5, dtype=np.int64)
    s, l = run(rp, ci, d, "f64_plain")
    assert s == float(np.sign(np.prod(d)))
    assert abs(l - float(np.sum(np.log(np.abs(d))))) <= 1e-14


def test_nan_inside_and_outside_the_blocks():
    rp, ci, v, D = workloads.sparse_block_triangular([4, 5, 6], seed=31, off_density=0.2)
    cor, blk, nb = api.sparse_blocks(torch.from_numpy(rp), torch.from_numpy(ci))
    cor, blk = cor.numpy(), blk.numpy()
    row_of_col = np.empty_like(cor)
    row_of_col[cor] = np.arange(len(cor))
    R = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    inside = blk[row_of_col[ci]] == blk[R]
    assert (~inside).any()
    # a NaN in an off-diagonal block does not enter det A
    w = v.copy()
    w[np.nonzero(~inside)[0][0]] = np.nan
    s, l = run(rp, ci, w, "f64_plain")
    ref = oracle.logdet(D)
    assert s == ref.sign and rel(l, ref.logabs) <= 1e-12
    # a NaN in a diagonal block gives NaN
    w = v.copy()
    w[np.nonzero(inside)[0][0]] = np.nan
    s, l = run(rp, ci, w, "f64_plain")
    assert math.isnan(s) and math.isnan(l)
