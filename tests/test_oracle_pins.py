"""Pins of the CPU oracle against facts other than itself (no GPU).

Each test ties the oracle to something the paper or the mathematics fixes:
closed forms, brute-force expansion, invariants, special cases and the paper's
worked example (Fig. 3).
"""
import json
import math
import os

import numpy as np
import pytest

import workloads
from oracle import exact

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _rel(a, b):
    return abs(a - b) / max(abs(b), 1.0)


# ---------------------------------------------------------------- closed forms

def test_2x2_closed_form(oracle_mod):
    rng = np.random.default_rng(11)
    for _ in range(200):
        A = rng.standard_normal((2, 2))
        res = oracle_mod.logdet(A)
        det = A[0, 0] * A[1, 1] - A[0, 1] * A[1, 0]
        assert res.sign == math.copysign(1.0, det)
        assert _rel(res.logabs, math.log(abs(det))) < 1e-13
        # Sec. 2.2: the pivot of the first step is the larger |entry| of row 0
        want = 0 if abs(A[0, 0]) >= abs(A[0, 1]) else 1
        assert res.piv_label[0] == want
        assert res.piv_value[0] == A[0, want]


def test_3x3_sarrus(oracle_mod):
    rng = np.random.default_rng(12)
    for _ in range(200):
        A = rng.standard_normal((3, 3))
        a, b, c = A[0]
        d, e, f = A[1]
        g, h, i = A[2]
        det = a * e * i + b * f * g + c * d * h - c * e * g - b * d * i - a * f * h
        res = oracle_mod.logdet(A)
        assert res.sign == math.copysign(1.0, det)
        assert _rel(res.logabs, math.log(abs(det))) < 1e-12


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 8])
def test_leibniz_exact_integers(oracle_mod, n):
    rng = np.random.default_rng(100 + n)
    for trial in range(12 if n <= 6 else 4):
        A = rng.integers(-6, 7, size=(n, n))
        det = exact.leibniz_det(A.tolist())
        res = oracle_mod.logdet(A.astype(np.float64))
        if det == 0:
            # exact zero determinant: the FP64 sweep may leave a tiny residue,
            # so only require a tiny |det| relative to the Hadamard bound
            bound = float(np.prod(np.linalg.norm(A, axis=1) + 1e-300))
            assert res.sign == 0 or res.logabs < math.log(bound) - 25
            continue
        assert res.sign == (1.0 if det > 0 else -1.0), (A, det)
        assert abs(res.logabs - math.log(abs(det))) < 1e-12 * max(1.0, abs(math.log(abs(det))))


def test_exact_rational_sweep_matches_leibniz():
    """The exact-rational sweep (same steps, no rounding) reproduces Leibniz."""
    rng = np.random.default_rng(7)
    for n in range(1, 8):
        for _ in range(5):
            A = rng.integers(-5, 6, size=(n, n)).tolist()
            assert exact.condense_exact(A)["det"] == exact.leibniz_det(A)


# ---------------------------------------------------------------- special cases

@pytest.mark.parametrize("n", [1, 2, 5, 12, 40])
def test_upper_triangular_dominant(oracle_mod, n):
    """Row-dominant upper triangular: every pivot is the diagonal, in order, and
    every update leaves the remaining block unchanged in value."""
    rng = np.random.default_rng(n)
    U = np.triu(rng.uniform(-1, 1, (n, n)), 1)
    d = rng.choice([-1, 1], n) * rng.uniform(2, 3, n)
    U[np.diag_indices(n)] = d
    res = oracle_mod.logdet(U)
    assert list(res.piv_label) == list(range(n))
    assert np.array_equal(res.piv_value, d)
    assert res.sign == float(np.prod(np.sign(d)))
    assert _rel(res.logabs, math.fsum(np.log(np.abs(d)))) < 1e-14


@pytest.mark.parametrize("n", [1, 3, 17])
def test_lower_triangular(oracle_mod, n):
    """Lower triangular: row 0 has one nonzero, so each pivot is the diagonal and
    the condensed block is the trailing lower-triangular block, bit for bit."""
    rng = np.random.default_rng(50 + n)
    L = np.tril(rng.standard_normal((n, n)))
    L[np.diag_indices(n)] += np.sign(L[np.diag_indices(n)]) * 0.5
    res = oracle_mod.logdet(L)
    assert list(res.piv_label) == list(range(n))
    assert np.array_equal(res.piv_value, np.diag(L))


@pytest.mark.parametrize("n", [1, 2, 3, 6, 12, 31])
def test_permutation_matrices(oracle_mod, n):
    rng = np.random.default_rng(200 + n)
    for _ in range(5):
        perm = rng.permutation(n)
        P = np.zeros((n, n))
        P[np.arange(n), perm] = 1.0
        res = oracle_mod.logdet(P)
        assert res.sign == exact.permutation_sign(perm)
        assert res.logabs == 0.0
        assert list(res.piv_label) == list(perm)


def test_fig3_large_pivot(oracle_mod):
    """Fig. 3 (Sec. 2.2): a huge pivot leaves B* equal to A minus its pivot row and column."""
    g = _golden("fig3_large_pivot.json")
    A = np.array(g["A"])
    B, factor = oracle_mod.condense_once(A, g["k"], g["l"])
    assert np.array_equal(B, np.array(g["B_expected"]))
    assert factor == g["factor_expected"]
    # the same matrix through the sweep: put the pivot row first; max-abs picks e
    A2 = A[[1, 0, 2]]
    res = oracle_mod.logdet(A2)
    assert res.piv_label[0] == 1 and res.piv_value[0] == 1e300
    det_b = 1.5 * 2.5 - 3.0 * (-1.25)
    # det A = e * (-1)^(2+2) * det B* (pivot at row 2, column 2 of Fig. 3), and
    # moving the pivot row to the top is one row exchange: det A2 = -det A
    assert res.sign == -math.copysign(1.0, det_b)
    assert _rel(res.logabs, math.log(1e300) + math.log(abs(det_b))) < 1e-15


@pytest.mark.parametrize("name", ["tie_break_3x3.json", "tie_break_negative_first.json"])
def test_tie_break_golden(oracle_mod, name):
    g = _golden(name)
    res = oracle_mod.logdet(np.array(g["A"]))
    assert list(res.piv_label) == g["piv_label"]
    assert list(res.piv_value) == g["piv_value"]
    assert res.sign == g["sign"]
    assert _rel(res.logabs, math.log(abs(g["det"]))) < 1e-15


def test_conventions(oracle_mod):
    res = oracle_mod.logdet(np.zeros((0, 0)))
    assert (res.sign, res.logabs) == (1.0, 0.0)
    res = oracle_mod.logdet(np.array([[-0.5]]))
    assert res.sign == -1.0 and res.logabs == math.log(0.5)
    A = np.random.default_rng(3).standard_normal((6, 6))
    Z = A.copy()
    Z[3] = 0.0  # a zero row stays zero under the updates
    res = oracle_mod.logdet(Z)
    assert res.sign == 0.0 and res.logabs == -math.inf
    Z = A.copy()
    Z[:, 2] = 0.0  # a zero column is never chosen and survives to the last 1x1
    res = oracle_mod.logdet(Z)
    assert res.sign == 0.0 and res.logabs == -math.inf
    N = A.copy()
    N[4, 1] = np.nan
    res = oracle_mod.logdet(N)
    assert math.isnan(res.sign) and math.isnan(res.logabs)


def test_dyadic_family_is_exact(oracle_mod):
    """workloads.dyadic_lu: the FP64 sweep reproduces the construction exactly."""
    for n in [1, 2, 7, 16, 33, 64]:
        A, sgn, logabs, perm = workloads.dyadic_lu(n, seed=n)
        res = oracle_mod.logdet(A)
        assert list(res.piv_label) == list(perm)
        assert np.all(np.abs(res.piv_value) == 8.0)
        assert res.sign == sgn
        assert _rel(res.logabs, logabs) < 1e-14
        if n <= 16:
            ex = exact.condense_exact(A.astype(int).tolist())
            assert ex["labels"] == list(perm)
            # every intermediate value is exact in FP32 (24-bit significand)
            assert all(exact.representable(v, 24) for v in ex["values"])


# ---------------------------------------------------------------- invariants

def test_product_rule(oracle_mod):
    rng = np.random.default_rng(21)
    for n in [4, 30, 90]:
        A = rng.standard_normal((n, n))
        B = rng.standard_normal((n, n))
        ra, rb, rab = oracle_mod.logdet(A), oracle_mod.logdet(B), oracle_mod.logdet(A @ B)
        assert rab.sign == ra.sign * rb.sign
        assert abs(rab.logabs - (ra.logabs + rb.logabs)) < 1e-9 * n


def test_scaling_rule_power_of_two_is_exact(oracle_mod):
    rng = np.random.default_rng(22)
    n = 57
    A = rng.standard_normal((n, n))
    c = -2.0
    ra, rc = oracle_mod.logdet(A), oracle_mod.logdet(c * A)
    # scaling by a power of two commutes with every rounding: same labels,
    # pivots scaled exactly
    assert list(ra.piv_label) == list(rc.piv_label)
    assert np.array_equal(rc.piv_value, c * ra.piv_value)
    assert rc.sign == ra.sign * (-1.0) ** n
    assert abs(rc.logabs - (ra.logabs + n * math.log(2.0))) < 1e-12


def test_scaling_rule_general(oracle_mod):
    rng = np.random.default_rng(23)
    n = 64
    A = rng.standard_normal((n, n))
    c = 3.7
    ra, rc = oracle_mod.logdet(A), oracle_mod.logdet(c * A)
    assert rc.sign == ra.sign
    assert abs(rc.logabs - (ra.logabs + n * math.log(c))) < 1e-11


def test_row_swap_flips_sign(oracle_mod):
    rng = np.random.default_rng(24)
    n = 40
    A = rng.standard_normal((n, n))
    B = A.copy()
    B[[3, 17]] = B[[17, 3]]
    ra, rb = oracle_mod.logdet(A), oracle_mod.logdet(B)
    assert rb.sign == -ra.sign
    assert abs(rb.logabs - ra.logabs) < 1e-12 * abs(ra.logabs) + 1e-12


def test_column_swap_is_exact_relabelling(oracle_mod):
    """Sec. 2.4: exchanging columns changes only the sign. With distinct |values|
    the sweep takes the same pivots in the same order (relabelled), so log|det|
    is bit-identical and the sign flips."""
    rng = np.random.default_rng(25)
    n = 45
    A = rng.standard_normal((n, n))
    i, j = 5, 30
    B = A.copy()
    B[:, [i, j]] = B[:, [j, i]]
    ra, rb = oracle_mod.logdet(A), oracle_mod.logdet(B)
    relabel = {i: j, j: i}
    assert [relabel.get(x, x) for x in ra.piv_label] == list(rb.piv_label)
    assert np.array_equal(ra.piv_value, rb.piv_value)
    assert rb.sign == -ra.sign
    assert rb.logabs == ra.logabs


def test_transpose_invariance(oracle_mod):
    """Sec. 2.3: factoring by row or by column gives the same determinant; the
    row-factored sweep on A^T is the column-factored sweep on A."""
    rng = np.random.default_rng(26)
    A = rng.standard_normal((70, 70))
    ra, rt = oracle_mod.logdet(A), oracle_mod.logdet(A.T)
    assert ra.sign == rt.sign
    assert abs(ra.logabs - rt.logabs) < 1e-11


def test_arbitrary_pivot_identity(oracle_mod):
    """Eq. (1)-(3) with the (-1)^(k+l) sign, any (k, l) (Sec. 2.1): det A = factor * det B."""
    rng = np.random.default_rng(27)
    n = 6
    A = rng.standard_normal((n, n))
    s0, l0 = np.linalg.slogdet(A)
    for k in range(n):
        for l in range(n):
            B, factor = oracle_mod.condense_once(A, k, l)
            s1, l1 = np.linalg.slogdet(B)
            assert math.copysign(1.0, factor) * s1 == s0
            assert abs(math.log(abs(factor)) + l1 - l0) < 1e-12


def test_spd_known_spectrum(oracle_mod):
    A, lam, sum_log = workloads.spd_spectrum(200, seed=5, lo=1e-4, hi=1.0)
    res = oracle_mod.logdet(A)
    assert res.sign == 1.0
    assert abs(res.logabs - sum_log) < 1e-8


@pytest.mark.parametrize("n", [1, 2, 5, 17, 64, 200])
def test_against_lapack_slogdet(oracle_mod, n):
    """Cross-check with LAPACK getrf (a library routine, different pivoting)."""
    A = workloads.dense_gaussian(n, seed=n)
    res = oracle_mod.logdet(A)
    s, l = np.linalg.slogdet(A)
    assert res.sign == s
    assert _rel(res.logabs, l) < 1e-12


def test_threads_do_not_change_bits(oracle_mod):
    A = workloads.dense_gaussian(150, seed=9)
    r1 = oracle_mod.logdet(A, nthreads=1)
    r4 = oracle_mod.logdet(A, nthreads=4)
    assert r1.sign == r4.sign and r1.logabs == r4.logabs
    assert np.array_equal(r1.piv_value, r4.piv_value)
    assert np.array_equal(r1.piv_label, r4.piv_label)


def test_bounded_sample(oracle_mod):
    A = workloads.dense_gaussian(50, seed=10)
    full = oracle_mod.logdet(A)
    part = oracle_mod.logdet(A, max_steps=20)
    assert part.steps == 20
    assert np.array_equal(part.piv_value[:20], full.piv_value[:20])


def test_gradient_definition(oracle_mod):
    """d log|det A| / dA = A^{-T}: central differences of the oracle itself."""
    rng = np.random.default_rng(31)
    n = 12
    A = rng.standard_normal((n, n)) + 4 * np.eye(n)
    G = oracle_mod.grad_logabs(A, 1.0)
    h = 1e-6
    for (i, j) in [(0, 0), (3, 7), (11, 2), (5, 5)]:
        E = np.zeros((n, n))
        E[i, j] = h
        fd = (oracle_mod.logdet(A + E).logabs - oracle_mod.logdet(A - E).logabs) / (2 * h)
        assert abs(fd - G[i, j]) < 1e-7
    # diagonal closed form
    d = rng.uniform(0.5, 2.0, n)
    assert np.allclose(oracle_mod.grad_logabs(np.diag(d), 2.0), np.diag(2.0 / d), rtol=1e-15)
