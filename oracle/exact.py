"""ORACLE -- test infrastructure only.  Exact permanents on the CPU.

``per_bruteforce`` is Eq. 1 of the paper written out; ``per_ryser_py`` is
Ryser's inclusion-exclusion formula (Section 1) over every column subset;
the remaining functions call the C oracle ``hybrid.c`` (Algorithm H_per and
Algorithm PH, Step 2, with exact big integers).
"""
from __future__ import annotations

import ctypes
import itertools
import math
import os

import numpy as np

from . import build as _build

_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        i64p = ctypes.POINTER(ctypes.c_int64)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        i32p = ctypes.POINTER(ctypes.c_int32)
        ip = ctypes.POINTER(ctypes.c_int)
        lib.oracle_ryser.argtypes = [ctypes.c_int, i64p, u32p, ctypes.c_int, ip, ip]
        lib.oracle_permanent.argtypes = [ctypes.c_int, i64p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, u32p, ctypes.c_int, ip, ip]
        lib.oracle_jobs.argtypes = [ctypes.c_int, i64p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    i64p, i64p, i32p, i64p, u32p, ctypes.c_int, i32p]
        lib.oracle_job_permanents.argtypes = [ctypes.c_int64, i32p, i64p, ctypes.c_int, ctypes.c_int,
                                              ctypes.c_int, u32p, ctypes.c_int, i32p, i32p]
        for f in (lib.oracle_ryser, lib.oracle_permanent, lib.oracle_jobs,
                  lib.oracle_job_permanents):
            f.restype = ctypes.c_int
        _LIB = lib
    return _LIB


_ERR = {1: "invalid argument", 2: "int64 overflow or value too large",
        5: "output buffer too short", 6: "out of memory"}


def _check(rc):
    if rc != 0:
        raise RuntimeError("oracle error %d: %s" % (rc, _ERR.get(rc, "?")))


def _ptr(arr, ctype):
    return arr.ctypes.data_as(ctypes.POINTER(ctype))


def _limbs_to_int(limbs, nlimbs, sign):
    v = 0
    for k in range(int(nlimbs) - 1, -1, -1):
        v = (v << 32) | int(limbs[k])
    return -v if sign < 0 else v


def _as_matrix(a):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.int64))
    if a.ndim != 2 or a.shape[0] != a.shape[1]:
        raise ValueError("square matrix expected")
    return a


# ---------------------------------------------------------------- Eq. 1
def per_bruteforce(a) -> int:
    """Eq. 1: sum over all permutations sigma of prod_i a[i, sigma(i)]."""
    a = [[int(x) for x in row] for row in np.asarray(a)]
    n = len(a)
    if n > 9:
        raise ValueError("brute force is for n <= 9")
    total = 0
    for sigma in itertools.permutations(range(n)):
        p = 1
        for i in range(n):
            p *= a[i][sigma[i]]
            if p == 0:
                break
        total += p
    return total


def per_ryser_py(a) -> int:
    """Ryser's formula (Section 1) in Python integers, every subset S of the
    columns enumerated and every row sum taken afresh:
    per(A) = (-1)^n sum_S (-1)^|S| prod_i sum_{j in S} a_ij."""
    a = [[int(x) for x in row] for row in np.asarray(a)]
    n = len(a)
    if n > 16:
        raise ValueError("per_ryser_py is for n <= 16")
    if n == 0:
        return 1
    total = 0
    for mask in range(1, 1 << n):
        cols = [j for j in range(n) if mask >> j & 1]
        prod = 1
        for i in range(n):
            prod *= sum(a[i][j] for j in cols)
            if prod == 0:
                break
        total += (-1) ** (n - len(cols)) * prod
    return total


# ---------------------------------------------------------------- C oracle
def ryser(a) -> int:
    """Ryser's formula by the C oracle (n <= 30)."""
    a = _as_matrix(a)
    cap = 96
    limbs = np.zeros(cap, dtype=np.uint32)
    nl, sg = ctypes.c_int(0), ctypes.c_int(0)
    _check(_lib().oracle_ryser(a.shape[0], _ptr(a, ctypes.c_int64), _ptr(limbs, ctypes.c_uint32),
                               cap, ctypes.byref(nl), ctypes.byref(sg)))
    return _limbs_to_int(limbs, nl.value, sg.value)


def permanent(a, d: int = 0, L: int = 0, threads: int | None = None, three: bool = False) -> int:
    """per(A) by Algorithm PH: d levels of Eq. 2, then H_per on every job
    (leaf cut-off L; L <= 2 is the paper's own rule), then the sum.  three:
    split nodes with s >= 5 by Eq. 2's three children instead of sending
    them to Ryser."""
    a = _as_matrix(a)
    if threads is None:
        threads = os.cpu_count() or 1
    cap = 96
    limbs = np.zeros(cap, dtype=np.uint32)
    nl, sg = ctypes.c_int(0), ctypes.c_int(0)
    _check(_lib().oracle_permanent(a.shape[0], _ptr(a, ctypes.c_int64), int(d), int(L), int(three), int(threads),
                                   _ptr(limbs, ctypes.c_uint32), cap, ctypes.byref(nl),
                                   ctypes.byref(sg)))
    return _limbs_to_int(limbs, nl.value, sg.value)


def jobs(a, d: int, L: int = 0, three: bool = False):
    """Job list after d levels of Algorithm PH, Step 2, in natural order.

    Returns a list of (matrix, coefficient) pairs; the permanent of the input
    equals sum(coef * per(matrix)).
    """
    a = _as_matrix(a)
    lib = _lib()
    nj, ne = ctypes.c_int64(0), ctypes.c_int64(0)
    null32 = ctypes.POINTER(ctypes.c_int32)()
    null64 = ctypes.POINTER(ctypes.c_int64)()
    nullu = ctypes.POINTER(ctypes.c_uint32)()
    _check(lib.oracle_jobs(a.shape[0], _ptr(a, ctypes.c_int64), int(d), int(L), int(three), ctypes.byref(nj),
                           ctypes.byref(ne), null32, null64, nullu, 0, null32))
    nj, ne = nj.value, ne.value
    cap = 96
    sizes = np.zeros(max(nj, 1), dtype=np.int32)
    mats = np.zeros(max(ne, 1), dtype=np.int64)
    climbs = np.zeros(max(nj, 1) * cap, dtype=np.uint32)
    csign = np.zeros(max(nj, 1), dtype=np.int32)
    _check(lib.oracle_jobs(a.shape[0], _ptr(a, ctypes.c_int64), int(d), int(L), int(three),
                           ctypes.byref(ctypes.c_int64()),
                           ctypes.byref(ctypes.c_int64()), _ptr(sizes, ctypes.c_int32),
                           _ptr(mats, ctypes.c_int64), _ptr(climbs, ctypes.c_uint32), cap,
                           _ptr(csign, ctypes.c_int32)))
    out = []
    off = 0
    for w in range(nj):
        m = int(sizes[w])
        mat = mats[off:off + m * m].reshape(m, m).copy()
        off += m * m
        limbs = climbs[w * cap:(w + 1) * cap]
        nl = cap
        while nl > 0 and limbs[nl - 1] == 0:
            nl -= 1
        out.append((mat, _limbs_to_int(limbs, nl, int(csign[w]))))
    return out


def job_permanents(mats, L: int = 0, threads: int | None = None, three: bool = False):
    """per(M) for each dense matrix in ``mats`` by H_per (leaf cut-off L)."""
    if threads is None:
        threads = os.cpu_count() or 1
    mats = [_as_matrix(m) for m in mats]
    count = len(mats)
    sizes = np.array([m.shape[0] for m in mats] or [0], dtype=np.int32)
    flat = np.concatenate([m.ravel() for m in mats] or [np.zeros(1, np.int64)]).astype(np.int64)
    cap = 96
    limbs = np.zeros(max(count, 1) * cap, dtype=np.uint32)
    nl = np.zeros(max(count, 1), dtype=np.int32)
    sg = np.zeros(max(count, 1), dtype=np.int32)
    _check(_lib().oracle_job_permanents(count, _ptr(sizes, ctypes.c_int32), _ptr(flat, ctypes.c_int64),
                                        int(L), int(three), int(threads), _ptr(limbs, ctypes.c_uint32), cap,
                                        _ptr(nl, ctypes.c_int32), _ptr(sg, ctypes.c_int32)))
    return [_limbs_to_int(limbs[w * cap:(w + 1) * cap], nl[w], sg[w]) for w in range(count)]


# ---------------------------------------------------------------- bounds
def rowcol_bound(a) -> int:
    """|per(A)| <= min(prod_i sum_j |a_ij|, prod_j sum_i |a_ij|)."""
    b = np.abs(np.asarray(a, dtype=object))
    pr = 1
    for s in b.sum(axis=1):
        pr *= int(s)
    pc = 1
    for s in b.sum(axis=0):
        pc *= int(s)
    return min(pr, pc)


def bregman_bound(a) -> float:
    """Bregman's bound for a 0/1 matrix: per(A) <= prod_i (r_i!)^(1/r_i)."""
    r = np.asarray(a).astype(bool).sum(axis=1)
    return math.exp(sum(math.lgamma(int(k) + 1) / int(k) for k in r if k > 0)) if (r > 0).all() else 0.0


def schrijver_lower_bound(n: int, k: int) -> float:
    """Schrijver's bound for k-regular 0/1 matrices:
    per(A) >= ((k-1)^(k-1) / k^(k-2))^n; (4/3)^n for k = 3."""
    return ((k - 1) ** (k - 1) / k ** (k - 2)) ** n
