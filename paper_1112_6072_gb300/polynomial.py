"""The permanental polynomial per(xI - A) (Section 4.2, Eq. 11) with exact
integer coefficients, on the residue path.

The paper evaluates per(xI - A) of C60 at complex points (roots of unity)
in floating point.  Here the polynomial is found exactly from integer
points: for each of k primes p, one plan holds the n + 1 matrices
x_t I - A (x_t = t - floor(n / 2), t = 0 .. n) and runs the whole path
(expansion, ordering, evaluation) modulo p (``perm_opts.modulus``); the
n + 1 residues are interpolated modulo p (Newton's divided differences),
which gives every coefficient modulo p; ``perm_crt`` then combines each
coefficient's k residues into the integer itself.

The number of primes follows from a bound on the coefficients: with
per(xI + B) = sum over index sets T of x^|T| per(B restricted to the
complement of T), the coefficients' absolute values sum to at most
per(I + |A|) <= prod_i (1 + sum_j |a_ij|), and k is chosen so that half the
primes' product exceeds that bound.
"""
from __future__ import annotations

import math

import numpy as np

from . import Plan, crt


def primes_below(limit: int, count: int) -> list[int]:
    """The `count` largest odd primes below `limit` (trial division)."""
    out, p = [], limit - 1 if limit % 2 == 0 else limit - 2
    while len(out) < count and p > 2:
        if all(p % d for d in range(3, math.isqrt(p) + 1, 2)):
            out.append(p)
        p -= 2
    return out


def points(n: int) -> list[int]:
    """n + 1 integer points centred on 0."""
    return [t - n // 2 for t in range(n + 1)]


def shifted(a, x: int) -> np.ndarray:
    """x I - A."""
    a = np.asarray(a, dtype=np.int64)
    return x * np.eye(a.shape[0], dtype=np.int64) - a


def coefficient_log2_bound(a) -> float:
    """log2 of prod_i (1 + sum_j |a_ij|), a bound on sum_k |c_k|."""
    a = np.abs(np.asarray(a, dtype=np.float64))
    return float(np.log2(1.0 + a.sum(axis=1)).sum()) if a.size else 0.0


def value_log2_bound(a, xs) -> float:
    """log2 of max over the points of prod_i sum_j |(x I - A)_ij|, a bound
    on |per(x I - A)| at every point."""
    best = 0.0
    for x in xs:
        rs = np.abs(shifted(a, x)).sum(axis=1).astype(np.float64)
        if (rs == 0).any():
            continue
        best = max(best, float(np.log2(rs).sum()))
    return best


def primes_for(bits: float) -> list[int]:
    """Primes above 2^30 whose product exceeds 2^(bits + 2)."""
    return primes_below(1 << 31, max(1, math.ceil((bits + 2) / 30)))


def residues_at(a, xs, p: int, **plan_opts) -> list[int]:
    """per(x I - A) mod p at every point of xs (one plan, one pass of the path)."""
    plan_opts.setdefault("order", "natural")  # every job is evaluated: no order pays for an estimate
    with Plan([shifted(a, x) for x in xs], modulus=p, **plan_opts) as plan:
        plan.expand()
        plan.evaluate()
        return [int(v) for v in plan.results()]


def values(a, xs, primes=None, **plan_opts) -> list[int]:
    """per(x I - A) exactly at every point of xs, from residues and perm_crt."""
    if primes is None:
        primes = primes_for(value_log2_bound(a, xs))
    res = np.zeros((len(xs), len(primes)), dtype=np.uint32)
    for i, p in enumerate(primes):
        res[:, i] = residues_at(a, xs, p, **plan_opts)
    return crt(res, primes)


def interpolate_mod(xs, ys, p: int) -> list[int]:
    """Coefficients (lowest degree first) modulo p of the polynomial of
    degree < len(xs) through (x_t, y_t), by Newton's divided differences
    modulo p (the points must be distinct modulo p)."""
    m = len(xs)
    x = [int(v) % p for v in xs]
    if len(set(x)) != m:
        raise ValueError("interpolation points must be distinct modulo p")
    dd = [int(v) % p for v in ys]
    for lvl in range(1, m):
        for t in range(m - 1, lvl - 1, -1):
            dd[t] = (dd[t] - dd[t - 1]) * pow(x[t] - x[t - lvl], p - 2, p) % p
    # Newton form to monomials: q = dd[m-1];  q = q (X - x_t) + dd[t]
    c = [dd[m - 1]]
    for t in range(m - 2, -1, -1):
        nxt = [0] * (len(c) + 1)
        for k, v in enumerate(c):
            nxt[k + 1] = (nxt[k + 1] + v) % p
            nxt[k] = (nxt[k] - x[t] * v) % p
        nxt[0] = (nxt[0] + dd[t]) % p
        c = nxt
    return c


def permanental_polynomial(a, primes=None, **plan_opts) -> list[int]:
    """Coefficients c_0 .. c_n of per(xI - A), lowest degree first."""
    a = np.asarray(a, dtype=np.int64)
    n = int(a.shape[0])
    xs = points(n)
    if primes is None:
        primes = primes_for(coefficient_log2_bound(a))
    if min(primes) <= n:
        raise ValueError("every prime must exceed the order (distinct points modulo p)")
    res = np.zeros((n + 1, len(primes)), dtype=np.uint32)
    for i, p in enumerate(primes):
        res[:, i] = interpolate_mod(xs, residues_at(a, xs, p, **plan_opts), p)
    return crt(res, primes)
