"""Pins of the oracle's other pivot-column rules and column factoring (CPU only).

Sec. 1 names two rules of earlier work besides the paper's max |a_kj|: the
smallest column index of a nonzero entry, and the nonzero entry closest to 1;
Sec. 1 and Sec. 2.3 note that the pivot may be factored out of column l instead
of row k. Sec. 2.2 argues with an example (a pivot row of entries 1e-10 and
2.01) that closest-to-1 can overflow where max |a_kj| does not. Pins:
  - every rule and factoring side gives det A: 2x2 / 3x3 closed forms, exact
    Leibniz determinants of integer matrices, permutation matrices;
  - each rule picks the column it names on hand-built rows (ties included);
  - an upper-triangular matrix under the first-nonzero rule takes its diagonal
    in order, bit for bit;
  - the Sec. 2.2 example: closest-to-1 and first-nonzero overflow, max |a_kj|
    stays finite and matches the exact determinant.
Mutations planted in copies of the source (tie to the last column, the
multiplier not divided by the pivot) must fail one of these pins.
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import exact

RULES = ["max_abs", "closest_to_one", "first_nonzero"]
SIDES = ["row", "column"]


def _pins(lib=None):
    failed = []

    def lg(A, rule, factor):
        return oracle.logdet(A, rule=rule, factor=factor, _library=lib)

    rng = np.random.default_rng(17)
    for rule, factor in itertools.product(RULES, SIDES):
        for n in (2, 3):
            for _ in range(10):
                A = rng.standard_normal((n, n))
                det = np.linalg.det(A)
                r = lg(A, rule, factor)
                if r.sign != math.copysign(1.0, det) or abs(r.logabs - math.log(abs(det))) > 1e-10:
                    failed.append(f"closed_form_{rule}_{factor}")
                    break
        for n in (4, 6):
            A = rng.integers(-5, 6, size=(n, n))
            det = exact.leibniz_det(A.tolist())
            if det == 0:
                continue
            r = lg(A.astype(float), rule, factor)
            if r.sign != (1.0 if det > 0 else -1.0) or abs(r.logabs - math.log(abs(det))) > 1e-10:
                failed.append(f"leibniz_{rule}_{factor}")
        perm = rng.permutation(7)
        P = np.zeros((7, 7))
        P[np.arange(7), perm] = 1.0
        r = lg(P, rule, factor)
        if r.sign != exact.permutation_sign(perm) or list(r.piv_label) != list(perm):
            failed.append(f"permutation_{rule}_{factor}")
    # the columns each rule names on hand-built first rows
    cases = {
        "max_abs": ([0.2, -1.3, 0.9, 0.0, -5.0], 4),
        # |-1.05| is closest to 1 (a signed distance would pick 0.9)
        "closest_to_one": ([0.2, -1.05, 0.9, 0.0, 5.0], 1),
        "first_nonzero": ([0.0, 0.0, -0.7, 3.0, 1.0], 2),
    }
    for rule, (row, want) in cases.items():
        A = np.eye(5) * 7.0
        A[0] = row
        A[want, want] = 0.0 if want else A[want, want]  # keep A nonsingular below
        A[want, 0] = 1.0
        r = lg(A, rule, "row")
        if r.piv_label[0] != want or r.piv_value[0] != row[want]:
            failed.append(f"choice_{rule}")
    # ties: |1.5| and |0.5| are both 0.5 from 1 (exact); the first column wins
    A = np.array([[0.5, 1.5, 0.0], [1.0, 2.0, 3.0], [0.0, 1.0, 4.0]])
    A2 = A.copy()
    A2[0] = [1.5, 0.5, 0.0]
    if lg(A, "closest_to_one", "row").piv_label[0] != 0 or \
            lg(A2, "closest_to_one", "row").piv_label[0] != 0:
        failed.append("tie_closest")
    # upper triangular, first nonzero: the diagonal in order, exactly
    U = np.triu(rng.standard_normal((9, 9))) + 3.0 * np.eye(9)
    r = lg(U, "first_nonzero", "row")
    if list(r.piv_label) != list(range(9)) or list(r.piv_value) != list(np.diag(U)):
        failed.append("triangular_first_nonzero")
    return failed


def overflow_example():
    """Sec. 2.2: a pivot row of entries 1e-10 and 2.01 above a row of 1e300's."""
    return np.array([[1e-10, 2.01, 2.01],
                     [1e300, 1e300, -1e300],
                     [1.0, 2.0, 3.0]])


def test_rule_pins_pass():
    assert _pins() == []


def test_sec22_overflow_example():
    A = overflow_example()
    det = exact.leibniz_det([[Fraction(x) for x in row] for row in A.tolist()])
    want = math.log(abs(Fraction(det)))
    r = oracle.logdet(A)
    assert math.isfinite(r.logabs) and r.sign == -1.0
    assert abs(r.logabs - want) <= 1e-12 * abs(want)
    for rule in ("closest_to_one", "first_nonzero"):
        bad = oracle.logdet(A, rule=rule)
        assert bad.piv_label[0] == 0  # the 1e-10 entry
        assert not math.isfinite(bad.logabs), (rule, bad.logabs)


def test_column_factoring_same_pivots_on_exact_inputs():
    """Row and column factoring differ only in rounding: on integer matrices with
    exact Schur complements (unit-diagonal triangular factors) the pivots match
    bit for bit."""
    rng = np.random.default_rng(8)
    n = 12
    L = np.tril(rng.integers(-1, 2, size=(n, n)), -1) + np.eye(n)
    U = np.triu(rng.integers(-1, 2, size=(n, n)), 1) + np.diag(rng.choice([-4.0, 4.0], size=n))
    A = L @ U
    a = oracle.logdet(A, factor="row")
    b = oracle.logdet(A, factor="column")
    assert list(a.piv_label) == list(b.piv_label)
    assert list(a.piv_value) == list(b.piv_value)
    assert a.sign == b.sign and a.logabs == b.logabs


MUTANTS = {
    "closest_tie_to_last": ("if (l < 0 || d < best) {", "if (l < 0 || d <= best) {"),
    "closest_signed_distance": ("const double d = fabs(fabs(W[j]) - 1.0);",
                                "const double d = fabs(W[j] - 1.0);"),
    "first_nonzero_skips_first": ("if (rule == 2) return j;", "if (rule == 2 && j > 0) return j;"),
    "colf_not_divided": ("const double c_i = wi[l] / p;", "const double c_i = wi[l];"),
    "colf_wrong_row": ("out[jj++] = fma(-c_i, W[j], wi[j]);", "out[jj++] = fma(-c_i, wi[j], W[j]);"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_rule_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    with open(oracle.core.source_path()) as f:
        src = f.read()
    assert src.count(old) == 1, f"mutation anchor not unique: {old!r}"
    c_path = tmp_path / "mutant.c"
    c_path.write_text(src.replace(old, new, 1))
    lib = oracle.core.compile_c(str(c_path), str(tmp_path / "libmutant.so"))
    assert _pins(lib), f"mutant {name} passed every pin"
