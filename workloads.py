"""Seeded synthetic inputs for the condensation log-determinant.

This module holds generators only: it contains none of the method's arithmetic,
and both the oracle side and the CUDA side draw their inputs from it. All CPU
generators use ``numpy.random.default_rng(seed)`` in FP64.

Workloads (the paper times FP64 dense matrices of size 1000..8000, Sec. 3, with no
stated distribution; these recipes stand in for its matrices):

  dense_gaussian(N, seed, var)   iid N(0, var) entries
  spd_covariance(N, seed, ...)   X^T X / m + ridge * I with X an m x N iid N(0,1) matrix
  spd_spectrum(N, seed, lo, hi)  Q diag(lambda) Q^T, Q Haar orthogonal (QR of a
                                 Gaussian with the sign of diag(R) folded in),
                                 lambda log-uniform in [lo, hi]; returns the exact
                                 sum of log(lambda) alongside
  spd_haar_torch(N, seed, ...)   the same recipe on the GPU for N = 16384 / 32768
  batched_sizes(count, seed)     sizes uniform on {32, 48, ..., 512}
  dyadic_lu(n, seed)             integer/dyadic matrices whose whole condensation
                                 sweep is exact in FP32, with the pivot labels and
                                 determinant known by construction
  sparse_block_triangular(sizes, seed, ...)
                                 a CSR matrix whose rows and columns are randomly
                                 permuted from a block upper triangular matrix
                                 with irreducible diagonal blocks of the given
                                 sizes (stands in for the sparse matrices the
                                 paper leaves to future work)
"""
from __future__ import annotations

import math

import numpy as np

# Named workloads (sizes and seeds of the benchmark and parity suites).
CONFIG_1000 = dict(N=1000, seed=0, var=1.0)           # dense iid N(0,1), FP64
CONFIG_8000 = dict(N=8000, seed=1, var=1.0 / 8000.0)  # dense iid N(0,1/N)
CONFIG_SPD_16384 = dict(N=16384, seed=2, lo=1e-4, hi=1.0)
CONFIG_SPD_32768 = dict(N=32768, seed=2, lo=1e-4, hi=1.0)
CONFIG_BATCH = dict(count=4096, seed=3, ridge=1e-2)
CONFIG_GRAD = dict(batch=256, N=1024, seed=4, lo=1e-2, hi=1.0)


def dense_gaussian(N: int, seed: int, var: float = 1.0, rng=None) -> np.ndarray:
    rng = np.random.default_rng(seed) if rng is None else rng
    return rng.standard_normal((N, N)) * math.sqrt(var)


def spd_covariance(N: int, seed: int = 0, m: int | None = None, ridge: float = 1e-3,
                   rng=None) -> np.ndarray:
    """X^T X / m + ridge * I, X an m x N iid N(0,1) matrix (m = 2N by default)."""
    rng = np.random.default_rng(seed) if rng is None else rng
    m = 2 * N if m is None else m
    X = rng.standard_normal((m, N))
    A = (X.T @ X) / m
    A[np.diag_indices(N)] += ridge
    return A


def dense_and_spd_pair(N: int, seed: int):
    """The two N x N matrices of one seed: iid N(0, 1/N), then from the same
    generator X (2N x N) for X^T X / (2N) + 1e-3 I."""
    rng = np.random.default_rng(seed)
    A = dense_gaussian(N, seed, 1.0 / N, rng=rng)
    S = spd_covariance(N, m=2 * N, ridge=1e-3, rng=rng)
    return A, S


def haar_orthogonal(N: int, rng) -> np.ndarray:
    G = rng.standard_normal((N, N))
    Q, R = np.linalg.qr(G)
    return Q * np.sign(np.diag(R))[None, :]


def spd_spectrum(N: int, seed: int, lo: float = 1e-4, hi: float = 1.0):
    """(A, lam, exact_sum_log) with A = Q diag(lam) Q^T, lam = 10^U(log10 lo, log10 hi)."""
    rng = np.random.default_rng(seed)
    lam = 10.0 ** rng.uniform(math.log10(lo), math.log10(hi), size=N)
    Q = haar_orthogonal(N, rng)
    A = (Q * lam[None, :]) @ Q.T
    A = 0.5 * (A + A.T)
    return A, lam, math.fsum(math.log(x) for x in lam)


def spd_spectrum_torch(N: int, seed: int, lo: float, hi: float, device, dtype=None):
    """GPU generator of the same recipe for sizes where a CPU QR is too slow.

    Draws with a seeded ``torch.Generator`` on ``device``; returns
    (A [FP64 on device], exact_sum_log). Only torch library calls (randn, QR,
    matmul) are used: plumbing, not the method.
    """
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(seed)
    u = torch.rand(N, generator=g, device=device, dtype=torch.float64)
    lam = 10.0 ** (math.log10(lo) + (math.log10(hi) - math.log10(lo)) * u)
    G = torch.randn(N, N, generator=g, device=device, dtype=torch.float64)
    Q, R = torch.linalg.qr(G)
    Q = Q * torch.sign(torch.diagonal(R))[None, :]
    A = (Q * lam[None, :]) @ Q.T
    A = 0.5 * (A + A.T)
    sum_log = math.fsum(float(x) for x in torch.log(lam).cpu().tolist())
    if dtype is not None:
        A = A.to(dtype)
    return A, sum_log


def dense_and_spd_pair_torch(N: int, seed: int, device):
    """GPU generator of the iid N(0,1/N) matrix and X^T X/(2N) + 1e-3 I (FP64)."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(seed)
    A = torch.randn(N, N, generator=g, device=device, dtype=torch.float64) / math.sqrt(N)
    X = torch.randn(2 * N, N, generator=g, device=device, dtype=torch.float64)
    S = (X.T @ X) / (2 * N)
    S.diagonal().add_(1e-3)
    return A, S


def batched_sizes(count: int = 4096, seed: int = 3) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.integers(0, 31, size=count) * 16 + 32


def batched_covariances(sizes, seed: int = 3, ridge: float = 1e-2):
    """One X^T X / (2n) + ridge * I matrix per size (X is 2n x n), one generator."""
    rng = np.random.default_rng(seed + 1000)
    return [spd_covariance(int(n), m=2 * int(n), ridge=ridge, rng=rng) for n in sizes]


def dyadic_lu(n: int, seed: int, density: float = 0.3):
    """A = (L U) P^T with exact pivots: returns (A, det, labels).

    L is unit lower triangular with entries in {-1, 0, 1}; U is upper triangular
    with diagonal +-8 and off-diagonal entries in {-1, 0, 1}; P permutes columns.
    After t condensation steps with the first row as pivot row, the remaining
    matrix is L[t:, t:] U[t:, t:] (permuted), whose first row is U's row t, so the
    largest |entry| of every pivot row is the diagonal entry +-8, unique. The
    pivot of step t is therefore U[t, t] in original column perm[t], and every
    intermediate value is a small dyadic rational (exact in FP32 and in TF32 /
    BF16 splits). det A = prod(diag U) * sgn(P).
    """
    rng = np.random.default_rng(seed)
    L = np.eye(n)
    mask = rng.random((n, n)) < density
    vals = rng.choice([-1.0, 1.0], size=(n, n))
    L += np.tril(mask * vals, -1)
    U = np.triu(rng.choice([-1.0, 0.0, 1.0], size=(n, n)), 1)
    d = rng.choice([-8.0, 8.0], size=n)
    U[np.diag_indices(n)] = d
    perm = rng.permutation(n)
    M = L @ U
    A = np.empty_like(M)
    A[:, perm] = M  # column t of L U lands in original column perm[t]
    inv = 0
    for i in range(n):
        for j in range(i + 1, n):
            inv += perm[i] > perm[j]
    det_sign = (-1.0 if inv % 2 else 1.0) * float(np.prod(np.sign(d)))
    logabs = n * math.log(8.0)
    return A, det_sign, logabs, perm.astype(np.int64)


def batched_covariances_torch(sizes, seed: int = 3, ridge: float = 1e-2, device="cuda",
                              dtype=None):
    """GPU generator of one X^T X / (2n) + ridge * I matrix per size (X is 2n x n),
    drawn per size class with a seeded torch.Generator; FP32 by default. Returns
    the matrices in the order of ``sizes``."""
    import torch

    dtype = dtype or torch.float32
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    sizes = [int(x) for x in sizes]
    out = [None] * len(sizes)
    for n in sorted(set(sizes)):
        idx = [i for i, x in enumerate(sizes) if x == n]
        X = torch.randn(len(idx), 2 * n, n, generator=g, device=device, dtype=torch.float64)
        S = torch.bmm(X.transpose(1, 2), X) / (2 * n)
        S.diagonal(dim1=1, dim2=2).add_(ridge)
        S = S.to(dtype)
        for k, i in enumerate(idx):
            out[i] = S[k].contiguous()
    return out


def _cache_dir():
    import os
    return os.environ.get("LD_INPUT_CACHE", os.path.join("/tmp", "ld_inputs"))


def spd_haar_torch(N: int, seed: int, lo: float = 1e-4, hi: float = 1.0, device="cuda",
                   dtype=None, cache: bool = True):
    """Q diag(lambda) Q^T with Q Haar, lambda log-uniform in [lo, hi], on the GPU.

    Q: QR of an N x N Gaussian (FP32 QR, the sign of diag(R) folded in), then
    every column scaled to unit norm in FP64, so that Q^T Q = I + E with a zero
    diagonal: log det A = sum log(lambda) + log det(Q^T Q), and the second term
    is about -||E||_F^2 / 2 (||E||_F = 4e-4 at N = 16384, i.e. below 1e-7 in
    log det A). A = (Q lambda) Q^T is formed in FP64 (an FP32 product moves
    log det by ~1e-4 relative at N = 16384) and symmetrised. Returns
    (A in ``dtype`` (FP64 by default) on ``device``, exact sum of log(lambda)).

    The result is cached as a file under $LD_INPUT_CACHE (default
    /tmp/ld_inputs) so that later processes skip the minute of FP64 work at
    N = 32768; writing the cache is best effort. Only torch library calls are
    used: plumbing, not the method.
    """
    import json
    import os

    import torch

    dtype = dtype or torch.float64
    tag = f"haar_N{N}_seed{seed}_lo{lo:g}_hi{hi:g}_{str(dtype).split('.')[-1]}"
    path = os.path.join(_cache_dir(), tag)
    if cache and os.path.exists(path + ".json") and os.path.exists(path + ".bin"):
        try:
            with open(path + ".json") as f:
                meta = json.load(f)
            host = torch.from_file(path + ".bin", shared=False, size=N * N, dtype=dtype)
            return host.view(N, N).to(device), meta["sum_log"]
        except Exception:
            pass
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    u = torch.rand(N, generator=g, device=device, dtype=torch.float64)
    lam = 10.0 ** (math.log10(lo) + (math.log10(hi) - math.log10(lo)) * u)
    G = torch.randn(N, N, generator=g, device=device, dtype=torch.float32)
    Q32, R = torch.linalg.qr(G)
    sgn = torch.sign(torch.diagonal(R))
    del G, R
    Q = Q32.double() * sgn.double()[None, :]
    del Q32
    Q /= torch.linalg.vector_norm(Q, dim=0)[None, :]
    A = (Q * lam[None, :]) @ Q.T
    del Q
    A = 0.5 * (A + A.T)
    sum_log = math.fsum(float(x) for x in torch.log(lam).cpu().tolist())
    A = A.to(dtype)
    if cache:
        try:
            os.makedirs(_cache_dir(), exist_ok=True)
            tmp = path + f".tmp{os.getpid()}"
            A.cpu().contiguous().numpy().tofile(tmp + ".bin")
            with open(tmp + ".json", "w") as f:
                json.dump({"sum_log": sum_log, "N": N, "seed": seed, "lo": lo, "hi": hi}, f)
            os.replace(tmp + ".bin", path + ".bin")
            os.replace(tmp + ".json", path + ".json")
        except Exception:
            pass
    return A, sum_log


def spd_reflectors_torch(N: int, seed: int, lo: float, hi: float, device, k: int = 8,
                         dtype=None):
    """Q diag(lambda) Q^T with Q a product of k random Householder reflectors
    (exactly orthogonal, dense), lambda log-uniform in [lo, hi]; FP64 on the GPU in
    O(k N^2). Stands in for the Haar recipe at sizes where an FP64 QR is too slow
    on the device. Returns (A, exact_sum_log)."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(seed)
    u = torch.rand(N, generator=g, device=device, dtype=torch.float64)
    lam = 10.0 ** (math.log10(lo) + (math.log10(hi) - math.log10(lo)) * u)
    A = torch.diag(lam)
    for _ in range(k):
        v = torch.randn(N, generator=g, device=device, dtype=torch.float64)
        v = v / torch.linalg.vector_norm(v)
        # A <- H A H with H = I - 2 v v^T
        w = A @ v
        A = A - 2.0 * torch.outer(v, w) - 2.0 * torch.outer(w, v) + 4.0 * (v @ w) * torch.outer(v, v)
    A = 0.5 * (A + A.T)
    sum_log = math.fsum(float(x) for x in torch.log(lam).cpu().tolist())
    if dtype is not None:
        A = A.to(dtype)
    return A, sum_log


def sparse_block_triangular(sizes, seed: int, off_density: float = 0.002, diag_shift: float = 2.0,
                            integer: bool = False, dense: bool = True, symmetric: bool = False):
    """CSR arrays (row_ptr, col_idx, vals) and the dense matrix of a sparse n x n
    matrix, n = sum(sizes): block upper triangular with diagonal blocks of the
    given sizes, rows and columns then permuted at random.

    Diagonal block of size s: its diagonal, a cyclic superdiagonal (entry (i,
    i+1 mod s)), which makes the block irreducible, and iid entries at density
    min(1, 8/s) with values N(0, 1/s); the diagonal adds diag_shift. Entries above
    the diagonal blocks at density off_density. integer=True draws small integers
    instead (diagonal +-2, others in {-1, 1}). Column indices are sorted within a
    row; the stored values are FP64. dense=False returns None for the dense
    matrix (large n). symmetric=True permutes rows and columns alike, so the
    diagonal stays stored."""
    rng = np.random.default_rng(seed)
    sizes = [int(x) for x in sizes]
    n = int(sum(sizes))
    starts = np.cumsum([0] + sizes[:-1])
    rows, cols, vals = [], [], []

    def draw(k):
        if integer:
            return rng.choice([-1.0, 1.0], size=k)
        return rng.standard_normal(k)

    for b, s0 in zip(sizes, starts):
        idx = np.arange(b)
        # diagonal, cyclic superdiagonal, random interior
        r = [idx, idx] if b > 1 else [idx]
        c = [idx, (idx + 1) % b] if b > 1 else [idx]
        dens = min(1.0, 8.0 / b)
        mask = rng.random((b, b)) < dens
        ri, ci = np.nonzero(mask)
        keep = (ri != ci) & (ci != (ri + 1) % b)
        r.append(ri[keep])
        c.append(ci[keep])
        rr = np.concatenate(r) + s0
        cc = np.concatenate(c) + s0
        v = draw(len(rr))
        if not integer:
            v = v / math.sqrt(b)
        d = rr == cc
        v[d] = (rng.choice([-1.0, 1.0], size=int(d.sum())) * 2.0 if integer
                else v[d] + diag_shift)
        rows.append(rr)
        cols.append(cc)
        vals.append(v)
    # entries above the diagonal blocks
    blk = np.repeat(np.arange(len(sizes)), sizes)
    m = int(off_density * n * n)
    if m > 0 and len(sizes) > 1:
        ri = rng.integers(0, n, size=m)
        ci = rng.integers(0, n, size=m)
        keep = blk[ri] < blk[ci]
        rows.append(ri[keep])
        cols.append(ci[keep])
        vals.append(draw(int(keep.sum())))
    R = np.concatenate(rows)
    C = np.concatenate(cols)
    V = np.concatenate(vals)
    # one entry per position (the first drawn wins)
    key = R * n + C
    _, first = np.unique(key, return_index=True)
    R, C, V = R[first], C[first], V[first]
    # random row and column permutations
    pr = rng.permutation(n)
    pc = pr if symmetric else rng.permutation(n)
    R = pr[R]
    C = pc[C]
    order = np.lexsort((C, R))
    R, C, V = R[order], C[order], V[order]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, R + 1, 1)
    row_ptr = np.cumsum(row_ptr).astype(np.int64)
    full = None
    if dense:
        full = np.zeros((n, n))
        full[R, C] = V
    return row_ptr, C.astype(np.int64), V.astype(np.float64), full

