"""The identities the blocked leaf walk rests on, checked on the CPU.

A model of the four-code walk (the leaf kernels' slot layout, Gray column
schedule and block sums, in Python integers) against the oracle's
permanents.  Rows and columns are permuted as in the kernels: Gray
columns 0 and 1 are the column pair touching the fewest rows (column 0 the
one with fewer than the group size of rows), the rows of column 0 take the
first slots, then the other rows of column 1, then the rest; the highest
remaining column carries the Nijenhuis-Wilf offset.  With doubled row sums
rho_i, the Gray sum over all 2^(m-1) codes is (-1)^(m-1) 2^(m-1) per(A).

Within an aligned block of four codes only columns 0 and 1 flip (0 in,
1 in or out, 0 out), so with P the product over the first NN slots and Z
over the rest the block contributes Z (P(0) - P(1) + P(2) - P(3)).  When the
rows of column 0 sit in slots [0, 8) and slots [8, 16) hold none of them,
the product P2 over [8, 16) only changes when column 1 flips, so
P(0) - P(1) + P(2) - P(3) = (P1(0) - P1(1)) P2(0) + (P1(2) - P1(3)) P2(2).
The same split of 8 slots into 4 + 4 applies when column 0 touches at most
4 rows; the leaf kernels then take a pair eligible for it (union within 8
rows, one column within 4) before the fewest-rows pair, column 0 being the
sparser column, and form the quad products in 32 bits (|rho| < 2^7).
"""
import math

import numpy as np
import pytest

from oracle import exact as oracle


def _layout(a, lim0, kernel_rule=False):
    m = a.shape[0]
    nz = a != 0
    cnt = nz.sum(axis=0)
    if kernel_rule:
        # the leaf kernels' rule: a pair for the 4 + 4 split first, then the
        # fewest rows, then the lowest pair; column 0 the sparser column
        def key(x, y):
            u = int((nz[:, x] | nz[:, y]).sum())
            split = u <= 8 and min(cnt[x], cnt[y]) <= 4
            return (0 if split else 1, u, x, y)
        _, u, ca, cb = min(key(x, y) for x in range(m) for y in range(x + 1, m))
        g0, g1 = (ca, cb) if cnt[ca] <= cnt[cb] else (cb, ca)
    else:
        u, ca, cb = min((int((nz[:, x] | nz[:, y]).sum()), x, y) for x in range(m) for y in range(x + 1, m))
        g0, g1 = (ca, cb) if nz[:, ca].sum() <= lim0 else (cb, ca)
    clast = m - 1
    while clast in (ca, cb):
        clast -= 1
    am, tm = nz[:, g0], nz[:, g0] | nz[:, g1]
    order = ([r for r in range(m) if am[r]] + [r for r in range(m) if tm[r] and not am[r]]
             + [r for r in range(m) if not tm[r]])
    slot = {r: i for i, r in enumerate(order)}

    def gray_index(c):
        if c == g0:
            return 0
        if c == g1:
            return 1
        if c == clast:
            return -1
        return 2 + c - (ca < c) - (cb < c) - (clast < c)

    return u, int(am.sum()), slot, gray_index


def _blocked_walk(a, nmax, nn, split, kernel_rule=False):
    m = a.shape[0]
    _, n_col0, slot, gray_index = _layout(a, nn // 2 if split else nn, kernel_rule)
    delta = [[0] * nmax for _ in range(m - 1)]
    rho = [1] * nmax
    for r in range(m):
        rs = last = 0
        for c in range(m):
            v = int(a[r, c])
            if v:
                rs += v
                j = gray_index(c)
                if j >= 0:
                    delta[j][slot[r]] = 2 * v
                else:
                    last = v
        rho[slot[r]] = 2 * last - rs
    half = nn // 2
    if split:
        assert n_col0 <= half and not any(delta[0][half:nn])

    def prod(lo, hi):
        return math.prod(rho[lo:hi])

    def add(col, lo, hi, s=1):
        for i in range(lo, hi):
            rho[i] += s * delta[col][i]

    acc, g, total = 0, 0, 1 << (m - 1)
    while True:
        s1 = -1 if (g >> 2) & 1 else 1
        if split:
            if nn == 8:  # the quads of the 4 + 4 split are formed in 32 bits
                assert all(abs(prod(lo, lo + 4)) < 1 << 28 for lo in (0, 4))
            a0, b0 = prod(0, half), prod(half, nn)
            add(0, 0, half)
            a1 = prod(0, half)
            add(1, 0, nn, s1)
            a2, b2 = prod(0, half), prod(half, nn)
            add(0, 0, half, -1)
            a3 = prod(0, half)
            block = (a0 - a1) * b0 + (a2 - a3) * b2
        else:
            n0 = prod(0, nn)
            add(0, 0, nn)
            n1 = prod(0, nn)
            add(1, 0, nn, s1)
            n2 = prod(0, nn)
            add(0, 0, nn, -1)
            n3 = prod(0, nn)
            block = n0 - n1 + n2 - n3
        acc += block * prod(nn, nmax)
        g += 4
        if g >= total:
            break
        j = (g & -g).bit_length() - 1  # the Gray column that flips at code g (>= 2)
        add(j, 0, nmax, -1 if (g >> (j + 1)) & 1 else 1)
    val = acc if (m - 1) % 2 == 0 else -acc
    assert val % (1 << (m - 1)) == 0
    return val >> (m - 1)


def _sparsest_pair(a):
    nz = a != 0
    m = a.shape[0]
    u, x, y = min((int((nz[:, x] | nz[:, y]).sum()), x, y) for x in range(m) for y in range(x + 1, m))
    return u, min(int(nz[:, x].sum()), int(nz[:, y].sum()))


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_eight_slot_block_identity(seed):
    """Pairs touching at most 8 rows: the unsplit four-code block sum."""
    rng = np.random.default_rng(seed)
    done = 0
    while done < 12:
        n = int(rng.integers(5, 13))
        a = (rng.random((n, n)) < rng.uniform(0.15, 0.4)) * rng.integers(1, 4, size=(n, n))
        if np.abs(a).sum(axis=1).max() >= 128 or _sparsest_pair(a)[0] > 8:
            continue
        assert _blocked_walk(a, 8 if n <= 8 else 16, 8, False) == oracle.permanent(a.astype(np.int64))
        done += 1


@pytest.mark.parametrize("seed", [4, 5, 6])
def test_sixteen_slot_split_identity(seed):
    """Pairs touching 9-16 rows with one column within 8: the two-group sum."""
    rng = np.random.default_rng(seed)
    done = 0
    while done < 8:
        n = int(rng.integers(10, 17))
        a = (rng.random((n, n)) < rng.uniform(0.45, 0.8)) * rng.integers(1, 3, size=(n, n))
        u, kmin = _sparsest_pair(a)
        if np.abs(a).sum(axis=1).max() >= 128 or not (8 < u <= 16 and kmin <= 8):
            continue
        assert _blocked_walk(a, 16, 16, True) == oracle.permanent(a.astype(np.int64))
        done += 1


@pytest.mark.parametrize("seed", [7, 8, 9])
def test_eight_slot_four_plus_four_identity(seed):
    """Pairs eligible for the 4 + 4 split (union within 8 rows, one column
    within 4), chosen and oriented as the leaf kernels do: the split block
    sum with every quad product in 32 bits."""
    rng = np.random.default_rng(seed)
    done = 0
    while done < 12:
        n = int(rng.integers(5, 21))
        a = (rng.random((n, n)) < rng.uniform(0.15, 0.35)) * rng.integers(1, 4, size=(n, n))
        if np.abs(a).sum(axis=1).max() >= 128 or (a != 0).sum(axis=1).min() == 0:
            continue
        nz = a != 0
        cnt = nz.sum(axis=0)
        if not any(int((nz[:, x] | nz[:, y]).sum()) <= 8 and min(cnt[x], cnt[y]) <= 4
                   for x in range(n) for y in range(x + 1, n)):
            continue
        nmax = 8 if n <= 8 else (16 if n <= 16 else 24)
        assert _blocked_walk(a, nmax, 8, True, kernel_rule=True) == oracle.permanent(a.astype(np.int64))
        done += 1
