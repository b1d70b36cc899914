"""ORACLE -- test infrastructure only.  The permanental polynomial
per(xI - A) (Section 4.2, Eq. 11) of a small integer matrix, by brute force
over permutations, and exact interpolation through integer points.

Every permutation sigma contributes prod_i (x [i = sigma(i)] - a_{i sigma(i)}):
a fixed point i gives the factor (x - a_ii), any other index the constant
-a_{i sigma(i)}.  The coefficients are integers, returned lowest degree
first.
"""
from __future__ import annotations

import itertools
from fractions import Fraction

import numpy as np


def _poly_mul(p, q):
    out = [0] * (len(p) + len(q) - 1)
    for i, u in enumerate(p):
        if u:
            for j, v in enumerate(q):
                out[i + j] += u * v
    return out


def permanental_polynomial_bruteforce(a) -> list[int]:
    """Coefficients c_0 .. c_n of per(xI - A), n <= 8."""
    a = [[int(v) for v in row] for row in np.asarray(a)]
    n = len(a)
    if n > 8:
        raise ValueError("brute force is for n <= 8")
    total = [0] * (n + 1)
    for sigma in itertools.permutations(range(n)):
        term = [1]
        for i in range(n):
            j = sigma[i]
            term = _poly_mul(term, [-a[i][j], 1] if i == j else [-a[i][j]])
            if not any(term):
                break
        for k, c in enumerate(term):
            total[k] += c
    return total


def poly_eval(coefs, x) -> int:
    """sum_k coefs[k] x^k (Horner)."""
    v = 0
    for c in reversed(coefs):
        v = v * x + c
    return v


def interpolate(xs, ys) -> list:
    """The polynomial of degree < len(xs) through (x_t, y_t), lowest degree
    first, by Newton's divided differences in exact rationals (Fractions;
    integers when the coefficients are)."""
    xs = [Fraction(int(x)) for x in xs]
    dd = [Fraction(int(y)) for y in ys]
    m = len(xs)
    for lvl in range(1, m):
        for t in range(m - 1, lvl - 1, -1):
            dd[t] = (dd[t] - dd[t - 1]) / (xs[t] - xs[t - lvl])
    # Newton form -> monomial coefficients: p = dd[m-1]; p = p (x - x_t) + dd[t]
    coefs = [dd[m - 1]]
    for t in range(m - 2, -1, -1):
        shifted = [Fraction(0)] + coefs                # x * p
        for k in range(len(coefs)):
            shifted[k] -= xs[t] * coefs[k]            # - x_t * p
        shifted[0] += dd[t]
        coefs = shifted
    return [int(c) if c.denominator == 1 else c for c in coefs]
