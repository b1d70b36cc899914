"""Host logic of the permanental polynomial (paper_1112_6072_gb300/polynomial.py,
no GPU): interpolation modulo p recovers known polynomials' coefficients
modulo p through the points the module uses; the primes, the points and
the coefficient bound."""
import math

import numpy as np
import pytest

from oracle import polynomial as OP
from paper_1112_6072_gb300 import polynomial as PP


def test_interpolate_mod_recovers_known_polynomials():
    rng = np.random.default_rng(3)
    for p in (101, 65537, 2147483647):
        for deg in (0, 1, 2, 7, 30, 60):
            if deg + 1 > p:
                continue
            c = [int(v) for v in rng.integers(-10**9, 10**9, size=deg + 1)]
            xs = PP.points(deg)
            assert PP.interpolate_mod(xs, [OP.poly_eval(c, x) for x in xs], p) == [v % p for v in c]


def test_interpolate_mod_rejects_colliding_points():
    with pytest.raises(ValueError):
        PP.interpolate_mod([0, 7], [1, 2], 7)


def test_points_and_primes():
    assert PP.points(4) == [-2, -1, 0, 1, 2] and PP.points(5) == [-2, -1, 0, 1, 2, 3]
    ps = PP.primes_below(1 << 31, 4)
    assert ps[0] == 2**31 - 1 and len(set(ps)) == 4 and all((1 << 30) < p < (1 << 31) for p in ps)
    for p in ps:
        assert all(p % d for d in range(3, 50000, 2))
    assert math.prod(PP.primes_for(120.0)) > 2 ** 122


def test_coefficient_bound_covers_brute_force():
    """sum_k |c_k| <= prod_i (1 + sum_j |a_ij|) on random small matrices."""
    rng = np.random.default_rng(5)
    for n in (1, 3, 5, 6):
        a = rng.integers(-3, 4, size=(n, n)).astype(np.int64)
        c = OP.permanental_polynomial_bruteforce(a)
        assert sum(abs(v) for v in c) <= 2.0 ** PP.coefficient_log2_bound(a)
        xs = PP.points(n)
        assert all(abs(OP.poly_eval(c, x)) <= 2.0 ** PP.value_log2_bound(a, xs) for x in xs)
