"""Garner's reconstruction as perm_crt's kernel forms it (crt.cu), modelled on
the CPU with 32-bit limbs: mixed-radix digits t = (t - v_j) p_j^-1 mod p_i,
Horner's rule into k + 1 limbs, the balanced value chosen by comparing 2x
(k + 2 limbs) with M, and M - x for the negative side."""
import math
import random

import pytest

from paper_1112_6072_gb300 import polynomial as PP

M32 = (1 << 32) - 1


def crt_model(res, primes):
    k = len(primes)
    inv = {(j, i): pow(primes[j] % primes[i], primes[i] - 2, primes[i]) for i in range(k) for j in range(i)}
    d = []
    for i in range(k):
        t = res[i]
        for j in range(i):
            t = (t + primes[i] - d[j] % primes[i]) % primes[i] * inv[(j, i)] % primes[i]
        d.append(t)
    x = [0] * (k + 1)
    for i in range(k - 1, -1, -1):
        carry = d[i]
        for w in range(k + 1):
            t = x[w] * primes[i] + carry
            x[w] = t & M32
            carry = t >> 32
        assert carry == 0
    M = [0] * (k + 1)
    M[0] = 1
    for p in primes:
        carry = 0
        for w in range(k + 1):
            t = M[w] * p + carry
            M[w] = t & M32
            carry = t >> 32
    cmp = 0
    for w in range(k + 1, -1, -1):
        y = (x[k] >> 31) if w == k + 1 else (((x[w] << 1) & M32) | (x[w - 1] >> 31 if w > 0 else 0))
        mw = M[w] if w <= k else 0
        if y != mw:
            cmp = 1 if y > mw else -1
            break
    mag = sum(v << (32 * w) for w, v in enumerate(x))
    if cmp > 0:
        mag = sum(v << (32 * w) for w, v in enumerate(M)) - mag
    zero = not any(x)
    return 0 if zero else (-mag if cmp > 0 else mag)


@pytest.mark.parametrize("k", [1, 2, 3, 7, 20])
def test_balanced_reconstruction(k):
    primes = PP.primes_below(1 << 31, k)
    half = math.prod(primes) // 2
    rng = random.Random(k)
    vals = [0, 1, -1, half, -half, half - 1, -(half - 1)] + [rng.randrange(-half, half + 1) for _ in range(300)]
    for v in vals:
        assert crt_model([v % p for p in primes], primes) == v
