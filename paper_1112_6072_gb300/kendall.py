"""Kendall rank correlation of job times against permanents, approximate
permanents and model predictions (Section 3.2: Eq. 7-10 and the null
distribution used for the p-values of Tables T2-T4).

tau_b counts concordant minus discordant pairs S and the tied pairs T (in
x) and U (in y), and returns S / sqrt((N0 - T)(N0 - U)), N0 = n(n-1)/2
(Eq. 10); it runs in O(n log n) by counting the inversions of y after a
sort by (x, y) (Knight's method), so it handles 10^5-10^6 jobs.
"""
from __future__ import annotations

import math

import numpy as np


def _tied_pairs(sorted_keys) -> int:
    """Pairs with equal keys in a sorted sequence (sum of t(t-1)/2 over runs)."""
    total, run = 0, 1
    for k in range(1, len(sorted_keys)):
        if sorted_keys[k] == sorted_keys[k - 1]:
            run += 1
        else:
            total += run * (run - 1) // 2
            run = 1
    return total + run * (run - 1) // 2


def _inversions(a: list) -> int:
    """Pairs i < j with a[i] > a[j] (bottom-up merge sort)."""
    n = len(a)
    src, dst = list(a), [None] * n
    inv, width = 0, 1
    while width < n:
        for lo in range(0, n, 2 * width):
            mid, hi = min(lo + width, n), min(lo + 2 * width, n)
            i, j, k = lo, mid, lo
            while i < mid and j < hi:
                if src[j] < src[i]:
                    dst[k] = src[j]
                    inv += mid - i
                    j += 1
                else:
                    dst[k] = src[i]
                    i += 1
                k += 1
            dst[k:hi] = src[i:mid] if i < mid else src[j:hi]
        src, dst = dst, src
        width *= 2
    return inv


def tau_b(x, y) -> float:
    """Kendall's tau with ties (Eq. 10)."""
    x = list(x)
    y = list(y)
    n = len(x)
    if n < 2:
        return 0.0
    order = sorted(range(n), key=lambda i: (x[i], y[i]))
    xs = [x[i] for i in order]
    ys = [y[i] for i in order]
    t = _tied_pairs(xs)                       # tied in x
    v = _tied_pairs(list(zip(xs, ys)))        # tied in both
    u = _tied_pairs(sorted(ys))               # tied in y
    n0 = n * (n - 1) // 2
    disc = _inversions(ys)                    # pairs tied in x are in y order: never counted
    s = n0 - t - u + v - 2 * disc
    den = math.sqrt((n0 - t) * (n0 - u))
    return s / den if den > 0 else 0.0


def p_value(tau: float, n: int) -> float:
    """Two-sided p-value of tau under independence, from the normal limit
    with E(tau) = 0 and var(tau) = 2(2n+5) / (9n(n-1)) (Section 3.2)."""
    if n < 3:
        return 1.0
    z = tau / math.sqrt(2.0 * (2 * n + 5) / (9.0 * n * (n - 1)))
    return math.erfc(abs(z) / math.sqrt(2.0))


def table(times, **rankings) -> dict:
    """T2-T4 style rows: tau and p-value of the times against each ranking."""
    out = {"n": len(times)}
    for name, vals in rankings.items():
        t = tau_b(times, vals)
        out[name] = {"tau": t, "p": p_value(t, len(times))}
    return out


def signed_mod(v: int, bits: int) -> int:
    """The signed integer congruent to v modulo 2^bits (|result| < 2^(bits-1))."""
    v &= (1 << bits) - 1
    return v - (1 << bits) if v >> (bits - 1) else v


def exact_job_permanents(values, coefs, bits: int) -> list:
    """per(job) from the records' coef * per(job) (mod 2^256, exact in the low
    bits) and the coefficients."""
    out = []
    for val, c in zip(values, coefs):
        cv = signed_mod(c, 256)
        pv = signed_mod(val, bits)
        out.append(pv // cv if cv != 0 else 0)
    return out


def words_to_ints(words: np.ndarray) -> list:
    """Rows of four little-endian uint64 words -> Python ints (mod 2^256)."""
    w = np.asarray(words, dtype=np.uint64).reshape(-1, 4)
    return [int(a) | (int(b) << 64) | (int(c) << 128) | (int(d) << 192) for a, b, c, d in w]
