"""Parity of the blocked sweep (panels + rank-b update) with the CPU oracle.

Exactly representable inputs (workloads.dyadic_lu): every mode takes the oracle's
pivot sequence exactly and returns the exact sign and log|det|. Gaussian inputs:
sign exact; log|det| within the stated relative tolerance (FP64 blocked and the
FP64-accurate sliced tensor-core update 1e-12, 3xTF32 1e-5, BF16x3 1e-4); plain
TF32 is reported against a loose bound only.
"""
import json
import math
import os

import numpy as np
import pytest
import torch

import oracle
import workloads
from paper_1811_08057_gb300 import api

pytestmark = pytest.mark.gpu

TOL = {"f64_blocked": 1e-12, "f64_ozaki": 1e-12, "f32_3xtf32": 1e-5, "f32_bf16x3": 1e-4,
       "f32_tf32": 2e-2}
# BF16x3 carries each FP32 operand as two BF16 pieces (16 significant bits), so
# every product of the trailing update is off by up to 2^-16 relative; the FP32
# accumulation is not the limit (test_rankb_gpu.test_bf16x3_error_is_the_split).
# On the ill-conditioned N = 8000 iid Gaussian matrix the log|det| error this
# leaves is 1.2e-4, above the 1e-4 bound: that case is a known failure (xfail),
# the bound is not widened.
BF16X3_N8000 = ("three BF16 products of a two-piece split carry 16 bits per operand; "
                "measured 1.2e-4 on this matrix, above the 1e-4 bound")
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rel_err(got, want):
    return abs(got - want) / max(abs(want), 1.0)


@pytest.mark.parametrize("mode", sorted(TOL))
@pytest.mark.parametrize("n", [5, 128, 129, 300, 700])
def test_blocked_dyadic_exact(mode, n):
    A, sgn, logabs, perm = workloads.dyadic_lu(n, seed=n + 3)
    f = api.logdet_factor(torch.from_numpy(A).cuda(), mode)
    torch.cuda.synchronize()
    assert np.array_equal(f.pivot_labels().cpu().numpy(), perm)
    assert float(f.sign) == sgn
    assert rel_err(float(f.logabs), logabs) < 1e-14


@pytest.mark.parametrize("mode", sorted(TOL))
@pytest.mark.parametrize("n", [64, 200, 385, 1000])
def test_blocked_gaussian_tolerance(mode, n):
    """Well-conditioned Gaussian matrices (iid N(0,1/n) + 2 I): a wrong update or
    a lost exchange shows up as an error far above the precision bound."""
    A = workloads.dense_gaussian(n, seed=300 + n, var=1.0 / n) + 2.0 * np.eye(n)
    ref = oracle.logdet(A)
    s, l = api.logdet(torch.from_numpy(A).cuda(), mode)
    err = rel_err(float(l), ref.logabs)
    print(f"n={n} {mode}: rel err {err:.3e}")
    if mode == "f32_tf32":  # reported only
        assert math.isfinite(float(l))
        return
    assert float(s) == ref.sign
    assert err <= TOL[mode], (mode, n, float(l), ref.logabs)


@pytest.mark.parametrize("mode", sorted(TOL))
def test_blocked_factors_reconstruct(mode):
    n = 300
    A = workloads.dense_gaussian(n, seed=17, var=1.0 / n)
    f = api.logdet_factor(torch.from_numpy(A).cuda(), mode)
    F = f.F[:, :n].double().cpu().numpy()
    FJ = F[:, ::-1]
    L = np.tril(FJ)
    U = np.triu(FJ, 1) + np.eye(n)
    cp = f.colperm.cpu().numpy()
    AQJ = A[:, cp][:, ::-1]
    tol = 1e-10 if mode in ("f64_blocked", "f64_ozaki") else (1e-2 if mode == "f32_tf32" else 1e-4)
    assert np.abs(L @ U - AQJ).max() <= tol


@pytest.mark.parametrize("mode", ["f64_blocked", "f64_ozaki"])
def test_blocked_f64_matches_plain_pivots(mode):
    """FP64 blocked reorders roundings only, and the sliced tensor-core update
    differs from FP64 FMAs by about 2^-47 of a row's largest entry: on a Gaussian
    matrix both take the plain sweep's pivot labels (no near-ties at this size)."""
    n = 500
    A = workloads.dense_gaussian(n, seed=21)
    fp = api.logdet_factor(torch.from_numpy(A).cuda(), "f64_plain")
    fb = api.logdet_factor(torch.from_numpy(A).cuda(), mode)
    assert torch.equal(fp.pivot_labels(), fb.pivot_labels())
    assert float(fb.sign) == float(fp.sign)
    assert rel_err(float(fb.logabs), float(fp.logabs)) < 1e-12


@pytest.mark.parametrize("mode", [
    pytest.param(m, marks=pytest.mark.xfail(reason=BF16X3_N8000, strict=False))
    if m == "f32_bf16x3" else m for m in sorted(TOL)])
def test_blocked_config_8000(mode):
    """N = 8000 dense iid N(0, 1/N), seed 1, against the stored FP64 oracle result."""
    with open(os.path.join(GOLDEN, "oracle_dense_n8000_seed1.json")) as fh:
        g = json.load(fh)
    A = workloads.dense_gaussian(8000, seed=1, var=1.0 / 8000)
    s, l = api.logdet(torch.from_numpy(A).cuda(), mode)
    err = rel_err(float(l), g["logabs"])
    print(f"N=8000 {mode}: sign {float(s):+.0f} (oracle {g['sign']:+.0f}), rel err {err:.3e}")
    if mode == "f32_tf32":  # reported only: plain TF32 may even flip a late pivot's sign
        assert math.isfinite(float(l))
        return
    assert float(s) == g["sign"]
    assert err <= TOL[mode], (mode, float(l), g["logabs"])


@pytest.mark.parametrize("mode", ["f32_plain", "f32_3xtf32", "f32_bf16x3"])
def test_ill_conditioned_gaussian_reported(mode):
    """iid Gaussian n = 1000 (a small last pivot): FP32-storage errors depend on the
    rounding order; reported, and held only to a condition-scaled bound."""
    n = 1000
    A = workloads.dense_gaussian(n, seed=1300, var=1.0 / n)
    ref = oracle.logdet(A)
    kappa = np.linalg.cond(A)
    s, l = api.logdet(torch.from_numpy(A).cuda(), mode)
    err = abs(float(l) - ref.logabs)
    print(f"n=1000 iid {mode}: |err| {err:.3e} (cond {kappa:.2e})")
    assert float(s) == ref.sign
    # first-order bound |d logdet| <= n ||A^-1|| ||dA|| with ||dA|| ~ n u ||A||
    u = 2.0 ** -24 if mode != "f32_bf16x3" else 2.0 ** -17
    assert err <= n * n * u * kappa


@pytest.mark.parametrize("mode", ["f32_3xtf32", "f32_bf16x3"])
def test_blocked_conventions(mode):
    A = workloads.dense_gaussian(200, seed=8)
    Z = A.copy()
    Z[150] = 0.0  # a zero row in a trailing block
    s, l = api.logdet(torch.from_numpy(Z).cuda(), mode)
    assert float(s) == 0.0 and float(l) == -math.inf
    N = A.copy()
    N[170, 3] = np.nan
    s, l = api.logdet(torch.from_numpy(N).cuda(), mode)
    assert math.isnan(float(s)) and math.isnan(float(l))


@pytest.mark.parametrize("mode", ["f64_blocked", "f32_3xtf32"])
def test_panel_kernel_matches_per_pivot_launches(mode, monkeypatch):
    """The persistent panel kernel performs exactly the per-pivot kernels'
    operations on the panel rows: identical pivots and bits."""
    n = 700
    A = torch.from_numpy(workloads.dense_gaussian(n, seed=44, var=1.0 / n)).cuda()
    fa = api.logdet_factor(A, mode)
    monkeypatch.setenv("LD_PANEL_PER_PIVOT", "1")
    fb = api.logdet_factor(A, mode)
    monkeypatch.setenv("LD_PANEL_PER_PIVOT", "0")
    assert torch.equal(fa.pivot_labels(), fb.pivot_labels())
    assert torch.equal(fa.pivval, fb.pivval)
    assert float(fa.logabs) == float(fb.logabs) and float(fa.sign) == float(fb.sign)
    assert torch.equal(fa.F[:, :n], fb.F[:, :n])  # columns past n are padding


@pytest.mark.parametrize("mode,n", [("f32_3xtf32", 300), ("f32_3xtf32", 700),
                                    ("f32_3xtf32", 2100), ("f64_blocked", 300),
                                    ("f64_blocked", 2100), ("f64_ozaki", 700),
                                    ("f64_ozaki", 9000)])
def test_cluster_panel_matches_grid_panel(mode, n, monkeypatch):
    """The cluster panel (inner blocks of 16 in distributed shared memory, deferred
    in-order updates) and the grid-wide panel kernel perform the same operations:
    identical pivots, factors and log|det| bits, in FP32 storage and in FP64 (at
    n = 9000 the FP64 panel holds 4, 2 and 1 positions per thread as the active
    width shrinks)."""
    A = torch.from_numpy(workloads.dense_gaussian(n, seed=n, var=1.0 / n)).cuda()
    fa = api.logdet_factor(A, mode)
    monkeypatch.setenv("LD_PANEL", "grid")
    fb = api.logdet_factor(A, mode)
    monkeypatch.setenv("LD_PANEL", "")
    assert torch.equal(fa.pivot_labels(), fb.pivot_labels())
    assert torch.equal(fa.pivval, fb.pivval)
    assert float(fa.logabs) == float(fb.logabs)
    assert torch.equal(fa.F[:, :n], fb.F[:, :n])
    # the non-factor path (trailing rows get the composed moves in the multiplier
    # kernel) gives the same result
    s, l = api.logdet(A, mode)
    assert float(l) == float(fa.logabs) and float(s) == float(fa.sign)
