"""Pins of the permanental-polynomial oracle (oracle/polynomial.py): closed
forms, agreement with Eq. 1 (brute force) evaluated at integer points, and
exact interpolation of known polynomials."""
import math

import numpy as np
import pytest

import oracle
from oracle import polynomial as P


@pytest.mark.parametrize("n", [1, 3, 5])
def test_closed_forms(n):
    z = np.zeros((n, n), dtype=np.int64)
    assert P.permanental_polynomial_bruteforce(z) == [0] * n + [1]                      # x^n
    want = [math.comb(n, k) * (-1) ** (n - k) for k in range(n + 1)]                    # (x - 1)^n
    assert P.permanental_polynomial_bruteforce(np.eye(n, dtype=np.int64)) == want
    d = np.diag(np.arange(2, 2 + n)).astype(np.int64)                                   # prod (x - d_i)
    want = [1]
    for i in range(n):
        want = P._poly_mul(want, [-(2 + i), 1])
    assert P.permanental_polynomial_bruteforce(d) == want


def test_two_by_two_all_ones():
    # per([[x-1, -1], [-1, x-1]]) = (x-1)^2 + 1
    assert P.permanental_polynomial_bruteforce(np.ones((2, 2), dtype=np.int64)) == [2, -2, 1]


@pytest.mark.parametrize("seed", range(4))
def test_values_match_eq1_at_integer_points(seed):
    rng = np.random.default_rng(seed)
    n = 4 + seed % 3
    a = rng.integers(-2, 3, size=(n, n)).astype(np.int64)
    c = P.permanental_polynomial_bruteforce(a)
    assert c[-1] == 1 and len(c) == n + 1
    for x in (-3, -1, 0, 2, 5):
        assert P.poly_eval(c, x) == oracle.per_bruteforce(x * np.eye(n, dtype=np.int64) - a)


def test_graph_coefficients_from_small_subgraphs():
    """For a simple graph: x^(n-2) -> edges, x^(n-3) -> -2 triangles,
    x^(n-4) -> disjoint edge pairs + 2 four-cycles (the principal 2-, 3-
    and 4-minors of -A)."""
    # the 3-prism: 6 vertices, 9 edges, 2 triangles, 3 four-cycles
    edges = [(0, 1), (1, 2), (2, 0), (3, 4), (4, 5), (5, 3), (0, 3), (1, 4), (2, 5)]
    a = np.zeros((6, 6), dtype=np.int64)
    for u, v in edges:
        a[u, v] = a[v, u] = 1
    c = P.permanental_polynomial_bruteforce(a)
    m = len(edges)
    adjacent_pairs = sum(math.comb(int(d), 2) for d in a.sum(axis=1))
    assert c[6] == 1 and c[5] == 0 and c[4] == m
    assert c[3] == -2 * 2
    assert c[2] == (math.comb(m, 2) - adjacent_pairs) + 2 * 3


def test_interpolate_known_polynomials():
    rng = np.random.default_rng(7)
    for deg in (0, 1, 4, 9):
        coefs = [int(v) for v in rng.integers(-10**6, 10**6, size=deg + 1)]
        xs = list(range(-(deg // 2), deg + 1 - deg // 2))
        ys = [P.poly_eval(coefs, x) for x in xs]
        assert P.interpolate(xs, ys) == coefs
    # points in any order, not consecutive
    coefs = [3, 0, -7, 1]
    xs = [5, -2, 11, 0]
    assert P.interpolate(xs, [P.poly_eval(coefs, x) for x in xs]) == coefs
