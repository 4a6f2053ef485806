"""Sparse matrices: the structure analysis of ld_logdet_sparse on the host.

ld_sparse_blocks returns a complete transversal sigma and the strongly
connected components of the graph of A P_sigma. These tests check the result
against what the definitions fix: sigma is a permutation onto stored entries,
every stored entry goes from a higher or equal component number to a lower or
equal one (block triangular order), the partition equals networkx's strongly
connected components of the same graph, and the determinant identity
det A = sgn(sigma) * prod det(diagonal block) holds with the FP64 oracle on
both sides. Structurally singular and malformed inputs are reported. No GPU.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import workloads
from paper_1811_08057_gb300 import _lib, api


def csr_of(D):
    R, C = np.nonzero(D)
    row_ptr = np.zeros(D.shape[0] + 1, dtype=np.int64)
    np.add.at(row_ptr, R + 1, 1)
    return np.cumsum(row_ptr).astype(np.int64), C.astype(np.int64), D[R, C]


def analyse(row_ptr, col_idx):
    cor, blk, nb = api.sparse_blocks(torch.from_numpy(row_ptr), torch.from_numpy(col_idx))
    return cor.numpy(), blk.numpy(), nb


def check_structure(row_ptr, col_idx, cor, blk, nb):
    n = len(row_ptr) - 1
    assert sorted(cor.tolist()) == list(range(n))  # a permutation
    row_of_col = np.empty(n, dtype=np.int64)
    row_of_col[cor] = np.arange(n)
    for i in range(n):
        cols = col_idx[row_ptr[i]:row_ptr[i + 1]]
        assert cor[i] in cols  # a stored entry on every diagonal position of A P_sigma
        for c in cols:  # block triangular order
            assert blk[row_of_col[c]] <= blk[i]
    assert set(blk.tolist()) == set(range(nb))
    return row_of_col


@pytest.mark.parametrize("sizes,seed", [([1, 1, 1, 1], 1), ([5], 2), ([3, 7, 1, 12, 4], 3),
                                        ([40, 1, 2, 25, 9, 1, 60], 4), ([1] * 30, 5)])
def test_structure_is_block_triangular(sizes, seed):
    rp, ci, v, D = workloads.sparse_block_triangular(sizes, seed=seed)
    cor, blk, nb = analyse(rp, ci)
    check_structure(rp, ci, cor, blk, nb)
    # the generator's diagonal blocks are irreducible: the finest block
    # triangular form has exactly those blocks (it is unique up to order)
    assert nb == len(sizes)
    assert sorted(np.bincount(blk).tolist()) == sorted(sizes)


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("diagonal", [False, True])
def test_components_match_networkx(seed, diagonal):
    """Random structures with a complete transversal: a scrambled one (found by
    matching) or a stored diagonal (the identity)."""
    nx = pytest.importorskip("networkx")
    rng = np.random.default_rng(100 + seed)
    n = 60
    D = (rng.random((n, n)) < 0.04) * rng.standard_normal((n, n))
    D[np.arange(n), np.arange(n) if diagonal else rng.permutation(n)] = 1.0
    rp, ci, v = csr_of(D)
    cor, blk, nb = analyse(rp, ci)
    if diagonal:
        assert np.array_equal(cor, np.arange(n))
    row_of_col = check_structure(rp, ci, cor, blk, nb)
    G = nx.DiGraph()
    G.add_nodes_from(range(n))
    for i in range(n):
        for c in ci[rp[i]:rp[i + 1]]:
            G.add_edge(i, int(row_of_col[c]))
    want = sorted(sorted(c) for c in nx.strongly_connected_components(G))
    got = sorted(sorted(np.nonzero(blk == b)[0].tolist()) for b in range(nb))
    assert got == want


@pytest.mark.parametrize("sizes,seed", [([3, 7, 1, 12, 4], 11), ([20, 20, 1, 5], 12)])
def test_determinant_factors_over_the_blocks(sizes, seed):
    """det A = sgn(sigma) * prod_k det B[S_k, S_k], B = A P_sigma, every
    determinant from the FP64 oracle: pins the reduction the GPU path relies on."""
    rp, ci, v, D = workloads.sparse_block_triangular(sizes, seed=seed)
    cor, blk, nb = analyse(rp, ci)
    whole = oracle.logdet(D)
    sign, logabs = 1.0, 0.0
    # sgn(sigma)
    seen = np.zeros(len(cor), dtype=bool)
    for i in range(len(cor)):
        j, length = i, 0
        while not seen[j]:
            seen[j] = True
            j = cor[j]
            length += 1
        if length and length % 2 == 0:
            sign = -sign
    B = D[:, cor]
    for b in range(nb):
        S = np.nonzero(blk == b)[0]
        r = oracle.logdet(B[np.ix_(S, S)])
        sign *= r.sign
        logabs += r.logabs
    assert sign == whole.sign
    assert abs(logabs - whole.logabs) <= 1e-12 * max(1.0, abs(whole.logabs))


def test_structurally_singular():
    # two rows whose only entries share one column: no complete transversal
    D = np.array([[1.0, 0, 0], [2.0, 0, 0], [1.0, 1.0, 1.0]])
    rp, ci, v = csr_of(D)
    assert analyse(rp, ci)[2] == -1
    # an empty row
    D = np.eye(4)
    D[2, 2] = 0.0
    rp, ci, v = csr_of(D)
    assert analyse(rp, ci)[2] == -1


def test_empty_and_malformed():
    assert analyse(np.zeros(1, dtype=np.int64), np.zeros(0, dtype=np.int64))[2] == 0
    bad = [
        (np.array([1, 1], dtype=np.int64), np.array([0], dtype=np.int64)),        # row_ptr[0] != 0
        (np.array([0, 2, 1], dtype=np.int64), np.array([0, 1], dtype=np.int64)),  # decreasing
        (np.array([0, 1, 2], dtype=np.int64), np.array([0, 2], dtype=np.int64)),  # column out of range
        (np.array([0, 2, 3], dtype=np.int64), np.array([1, 1, 0], dtype=np.int64)),  # repeated column
    ]
    for rp, ci in bad:
        with pytest.raises(_lib.LogdetError) as e:
            analyse(rp, ci)
        assert e.value.code == _lib.LD_ERR_INVALID_ARG


def test_sign_of_a_permutation_matrix():
    """A permutation matrix: one block per row, det = sgn(perm) (the oracle's
    value), and the transversal is the permutation itself."""
    rng = np.random.default_rng(7)
    n = 9
    perm = rng.permutation(n)
    D = np.zeros((n, n))
    D[np.arange(n), perm] = 1.0
    rp, ci, v = csr_of(D)
    cor, blk, nb = analyse(rp, ci)
    assert np.array_equal(cor, perm) and nb == n
    assert oracle.logdet(D).sign in (1.0, -1.0) and math.isfinite(oracle.logdet(D).logabs)


def test_small_edge_structures():
    # 1 x 1: one block; with no entry: structurally singular
    assert analyse(np.array([0, 1], dtype=np.int64), np.array([0], dtype=np.int64))[2] == 1
    assert analyse(np.array([0, 0], dtype=np.int64), np.zeros(0, dtype=np.int64))[2] == -1
    # a dense matrix is one irreducible block
    D = np.ones((6, 6))
    rp, ci, v = csr_of(D)
    cor, blk, nb = analyse(rp, ci)
    assert nb == 1 and np.array_equal(cor, np.arange(6))
    # upper triangular with a full diagonal: n blocks of one, in an order in
    # which every stored entry goes to a lower or equal block number
    U = np.triu(np.ones((7, 7)))
    rp, ci, v = csr_of(U)
    cor, blk, nb = analyse(rp, ci)
    assert nb == 7
    check_structure(rp, ci, cor, blk, nb)
