"""The residue path's modular arithmetic, modelled on the CPU in Python
integers with the kernels' word sizes (modp.cuh, ryser_mod.cuh): Newton's
iteration for -p^-1 mod 2^32 in four steps, Montgomery's product with its
bounds (t + q p < 2^64, the reduced value below 2p), and the leaf formula
per = (-1)^(m-1) Sigma (2^-1)^(m-1) mod p against the oracle."""
import random

import numpy as np
import pytest

from oracle import exact as oracle

M32, M64 = (1 << 32) - 1, (1 << 64) - 1


def modp_make(p):
    x = p  # p * p = 1 mod 8: three correct low bits
    for _ in range(4):
        x = (x * ((2 - p * x) & M32)) & M32
    return (-x) & M32, pow(1 << 32, 2, p)


def mont_mul(a, b, p, pneg):
    t = a * b
    q = ((t & M32) * pneg) & M32
    s = t + q * p
    assert s <= M64 and s & M32 == 0  # exact in 64 bits, divisible by 2^32
    u = s >> 32
    assert u < 2 * p
    return u - p if u >= p else u


PRIMES = [3, 5, 7, 65537, 1000003, 2147483629, 2147483647]


@pytest.mark.parametrize("p", PRIMES)
def test_newton_inverse_and_montgomery_product(p):
    pneg, r2 = modp_make(p)
    assert (p * pneg) & M32 == M32  # p * (-p^-1) = -1 mod 2^32
    rinv = pow(1 << 32, -1, p)
    rng = random.Random(p)
    for _ in range(2000):
        a, b = rng.randrange(p), rng.randrange(p)
        assert mont_mul(a, b, p, pneg) == a * b * rinv % p
    # into and out of Montgomery form
    a = rng.randrange(p)
    am = mont_mul(a, r2, p, pneg)
    assert am == a * (1 << 32) % p and mont_mul(am, 1, p, pneg) == a


def sigma_mod(a, p):
    """The Gray sum of doubled row sums, every value a residue (as the
    modular leaf walk forms it), in plain residues."""
    m = a.shape[0]
    total = 0
    for S in range(1 << (m - 1)):
        prod = 1
        for i in range(m):
            rho = 2 * int(a[i, m - 1]) - int(a[i].sum()) + 2 * sum(int(a[i, j]) for j in range(m - 1) if S >> j & 1)
            prod = prod * (rho % p) % p
        total = (total + (-prod if bin(S).count("1") & 1 else prod)) % p
    return total


@pytest.mark.parametrize("p", [3, 65537, 2147483647])
def test_leaf_formula_modulo_p(p):
    rng = np.random.default_rng(p % 1000)
    for m in range(2, 9):
        a = rng.integers(-5, 6, size=(m, m)).astype(np.int64)
        h = pow((p + 1) // 2, m - 1, p)
        per = sigma_mod(a, p) * h % p
        if (m - 1) & 1:
            per = (-per) % p
        assert per == oracle.permanent(a) % p
