"""The pins catch plausible mistakes in the oracle (CPU only).

Each case plants one mistake in a temporary copy of the oracle's C source
(a dropped sign term, a wrong operand, a flipped comparison, a missing step),
compiles it, and checks that at least one pin fails on the mutant while all
pins pass on the real oracle.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import workloads
from oracle import exact

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

MUTANTS = {
    "drop_laplace_sign": ("if (l & 1) sgn = -sgn;", ""),
    "drop_pivot_sign": ("if (p < 0.0) sgn = -sgn;", ""),
    "wrong_update_sign": ("out[jj++] = fma(-a_il, r[j], wi[j]);", "out[jj++] = fma(a_il, r[j], wi[j]);"),
    "tie_to_last": ("if (fabs(W[j]) > best) {", "if (fabs(W[j]) >= best) {"),
    "min_abs_pivot": ("if (fabs(W[j]) > best) {", "if (fabs(W[j]) < best) {"),
    "multiply_not_divide": ("r[j] = W[j] / p;", "r[j] = W[j] * p;"),
    "transposed_multiplier": ("const double a_il = wi[l];", "const double a_il = W[l * m + i];"),
    "drop_last_pivot": ("if (m == 1) {\n      done = 1;", "if (m == 2) {\n      done = 1;"),
    "labels_not_shifted": ("label[j] = label[j + 1];", "label[j] = label[j];"),
    "pivot_row_not_factored": ("r[j] = W[j] / p;", "r[j] = W[j];"),
}


def _pins(lib):
    """A compact pin suite; returns the names of the pins that fail."""
    failed = []

    def lg(A):
        return oracle.logdet(A, _library=lib)

    rng = np.random.default_rng(5)
    # 2x2 / 3x3 closed forms
    for _ in range(20):
        A = rng.standard_normal((3, 3))
        det = np.linalg.det(A)
        r = lg(A)
        if r.sign != math.copysign(1.0, det) or abs(r.logabs - math.log(abs(det))) > 1e-10:
            failed.append("closed_form")
            break
    # Leibniz on integers
    for n in (4, 5):
        A = rng.integers(-6, 7, size=(n, n))
        det = exact.leibniz_det(A.tolist())
        r = lg(A.astype(float))
        if det == 0:
            continue
        if r.sign != (1.0 if det > 0 else -1.0) or abs(r.logabs - math.log(abs(det))) > 1e-10:
            failed.append("leibniz")
            break
    # permutation matrices
    perm = rng.permutation(9)
    P = np.zeros((9, 9))
    P[np.arange(9), perm] = 1.0
    r = lg(P)
    if r.sign != exact.permutation_sign(perm) or list(r.piv_label) != list(perm):
        failed.append("permutation")
    # tie-break golden example
    with open(os.path.join(GOLDEN, "tie_break_3x3.json")) as f:
        g = json.load(f)
    r = lg(np.array(g["A"]))
    if list(r.piv_label) != g["piv_label"] or list(r.piv_value) != g["piv_value"]:
        failed.append("tie_break")
    # dyadic family: known labels
    A, sgn, logabs, perm = workloads.dyadic_lu(20, seed=3)
    r = lg(A)
    if list(r.piv_label) != list(perm) or r.sign != sgn:
        failed.append("dyadic")
    # SPD with known spectrum
    A, lam, sum_log = workloads.spd_spectrum(30, seed=1, lo=1e-2, hi=1.0)
    r = lg(A)
    if r.sign != 1.0 or abs(r.logabs - sum_log) > 1e-9:
        failed.append("spd")
    return failed


def test_pins_pass_on_the_oracle():
    assert _pins(oracle.build()) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    with open(oracle.core.source_path()) as f:
        src = f.read()
    assert src.count(old) >= 1, f"mutation anchor not found: {old!r}"
    mutated = src.replace(old, new, 1)
    c_path = tmp_path / "mutant.c"
    c_path.write_text(mutated)
    lib = oracle.core.compile_c(str(c_path), str(tmp_path / "libmutant.so"))
    failed = _pins(lib)
    assert failed, f"mutant {name} passed every pin"
