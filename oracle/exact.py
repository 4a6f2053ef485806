"""Exact references for small matrices (test infrastructure only).

``leibniz_det``   det A by the permutation (Leibniz) sum over Python integers or
                  Fractions: brute force, independent of condensation, n <= 8.
``condense_exact`` the condensation sweep (Eqs. (2)-(3), Sec. 2.2, first row as
                  pivot row) in exact rational arithmetic. It returns the exact
                  determinant, the pivot labels and every intermediate value, so a
                  test can tell whether a matrix stays exactly representable in a
                  given floating-point format through the whole sweep.
"""
from __future__ import annotations

import itertools
from fractions import Fraction


def permutation_sign(perm) -> int:
    """Sign of a permutation given as a sequence of 0..n-1 (count of inversions)."""
    perm = list(perm)
    inv = 0
    for i in range(len(perm)):
        for j in range(i + 1, len(perm)):
            if perm[i] > perm[j]:
                inv += 1
    return -1 if inv & 1 else 1


def leibniz_det(A):
    """det A = sum over permutations s of sgn(s) * prod_i a_{i, s(i)}; exact."""
    n = len(A)
    if n == 0:
        return 1
    if n > 8:
        raise ValueError("Leibniz expansion is limited to n <= 8")
    total = 0
    for perm in itertools.permutations(range(n)):
        prod = permutation_sign(perm)
        for i in range(n):
            prod *= A[i][perm[i]]
            if prod == 0:
                break
        total += prod
    return total


def condense_exact(A):
    """Exact-rational condensation sweep with max-abs pivoting in the first row.

    Returns a dict with ``det`` (Fraction), ``labels`` (original column label of
    each pivot), ``pivots`` (Fractions) and ``values`` (the set of every value
    that appears: entries, factored rows and minors).
    """
    W = [[Fraction(x) for x in row] for row in A]
    n = len(W)
    labels = list(range(n))
    det = Fraction(1)
    out_labels, pivots = [], []
    values = set(x for row in W for x in row)
    while W:
        m = len(W)
        row = W[0]
        l = 0
        for j in range(1, m):
            if abs(row[j]) > abs(row[l]):
                l = j
        p = row[l]
        out_labels.append(labels[l])
        pivots.append(p)
        if p == 0:
            return {"det": Fraction(0), "labels": out_labels, "pivots": pivots, "values": values}
        det *= p * (-1 if (l % 2) else 1)
        if m == 1:
            break
        r = [x / p for x in row]
        values.update(r)
        Wn = []
        for i in range(1, m):
            a_il = W[i][l]
            new_row = []
            for j in range(m):
                if j == l:
                    continue
                prod = a_il * r[j]
                values.add(prod)
                new_row.append(W[i][j] - prod)
            values.update(new_row)
            Wn.append(new_row)
        W = Wn
        labels = labels[:l] + labels[l + 1:]
    return {"det": det, "labels": out_labels, "pivots": pivots, "values": values}


def representable(x: Fraction, mantissa_bits: int, max_exp: int = 100) -> bool:
    """True if x is exactly a binary floating-point number with the given
    significand width (including the hidden bit) and |exponent| <= max_exp."""
    if x == 0:
        return True
    num, den = abs(x.numerator), x.denominator
    if den & (den - 1):
        return False  # denominator not a power of two
    while num % 2 == 0:
        num //= 2
    if num.bit_length() > mantissa_bits:
        return False
    e = abs(x).numerator.bit_length() - x.denominator.bit_length()
    return abs(e) <= max_exp
