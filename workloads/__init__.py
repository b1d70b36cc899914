"""Seeded synthetic inputs shared by the oracle tests, the CUDA-path tests and the bench.

This module only draws matrices; it holds none of the permanent arithmetic.
Every generator takes an explicit integer seed and uses numpy's PCG64
(``numpy.random.default_rng``), so the same seed gives the same matrix on
any machine.

The workloads stand in for the paper's fullerene and sparse-collection
matrices (Section 4): random simple 3-regular graphs (fullerenes are
3-regular), the truncated icosahedron C60 itself, dense small-integer leaf
batches for the Ryser kernel, and rows holding 3 to 5 nonzeros for
"real sparse" inputs such as the dwt_66 matrix of Section 4.3, which is not
available here.
"""
from __future__ import annotations

import itertools

import numpy as np

__all__ = [
    "regular3",
    "c60_coordinates",
    "c60",
    "paper_adjacency",
    "shuffle_vertices",
    "leaf_batch",
    "sparse_rows",
    "mixed_batch",
    "random_small",
]


def regular3(n: int, seed: int) -> np.ndarray:
    """Adjacency matrix of a random simple 3-regular graph on ``n`` vertices.

    Configuration model: 3n stubs are shuffled and paired consecutively; a
    pairing with a loop or a repeated edge is rejected and redrawn from the
    same generator.  Returns an int64 0/1 symmetric matrix.
    """
    if n < 4 or (3 * n) % 2:
        raise ValueError("a simple 3-regular graph needs n >= 4 and 3n even")
    rng = np.random.default_rng(seed)
    while True:
        stubs = np.repeat(np.arange(n), 3)
        rng.shuffle(stubs)
        a = np.zeros((n, n), dtype=np.int64)
        ok = True
        for k in range(0, 3 * n, 2):
            u, v = int(stubs[k]), int(stubs[k + 1])
            if u == v or a[u, v]:
                ok = False
                break
            a[u, v] = a[v, u] = 1
        if ok:
            return a


def c60_coordinates() -> np.ndarray:
    """The 60 vertices of the truncated icosahedron.

    All even (cyclic) permutations of (0, +-1, +-3phi), (+-1, +-(2+phi), +-2phi)
    and (+-phi, +-2, +-(2phi+1)), phi the golden ratio.  Sorted
    lexicographically so that vertex ids are reproducible.
    """
    phi = (1.0 + 5.0 ** 0.5) / 2.0
    base = [(0.0, 1.0, 3 * phi), (1.0, 2 + phi, 2 * phi), (phi, 2.0, 2 * phi + 1)]
    pts = set()
    for b in base:
        for rot in ((0, 1, 2), (1, 2, 0), (2, 0, 1)):
            v = (b[rot[0]], b[rot[1]], b[rot[2]])
            for signs in itertools.product((1.0, -1.0), repeat=3):
                pts.add(tuple(round(v[i] * signs[i], 9) + 0.0 for i in range(3)))
    p = np.array(sorted(pts), dtype=np.float64)
    if p.shape != (60, 3):
        raise AssertionError("truncated icosahedron must have 60 vertices")
    return p


def c60(seed: int | None = None) -> np.ndarray:
    """60x60 0/1 adjacency of C60: vertices joined at the minimum distance.

    With ``seed`` given, the vertex order is shuffled by that seed (the same
    permutation applied to rows and columns).
    """
    p = c60_coordinates()
    d = np.linalg.norm(p[:, None, :] - p[None, :, :], axis=2)
    np.fill_diagonal(d, np.inf)
    dmin = d.min()
    a = (np.abs(d - dmin) < 1e-6).astype(np.int64)
    if seed is not None:
        a = shuffle_vertices(a, seed)
    return a


def paper_adjacency(name: str) -> np.ndarray:
    """The C100 or C60 adjacency matrix printed in the paper's Appendix
    (``name`` = "c100" or "c60"), read from the fixture under tests/golden."""
    import os

    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden",
                        f"{name}_adjacency.txt")
    rows = []
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            rows.append([int(x) for x in line.split()])
    n = len(rows)
    a = np.zeros((n, n), dtype=np.int64)
    for r in rows:
        for u in r[1:]:
            a[r[0] - 1, u - 1] = 1
    return a


def shuffle_vertices(a: np.ndarray, seed: int) -> np.ndarray:
    """Apply one seeded permutation to both the rows and the columns."""
    perm = np.random.default_rng(seed).permutation(a.shape[0])
    return np.ascontiguousarray(a[np.ix_(perm, perm)])


def leaf_batch(count: int, seed: int, nmin: int = 12, nmax: int = 24,
               p_nonzero: float = 0.35, vmax: int = 3):
    """Independent dense small-integer matrices for the leaf Ryser kernel.

    Sizes are uniform in [nmin, nmax]; each entry is nonzero with probability
    ``p_nonzero`` and a nonzero entry is uniform in {1, ..., vmax}.  Returns a
    list of int64 arrays.
    """
    rng = np.random.default_rng(seed)
    sizes = rng.integers(nmin, nmax + 1, size=count)
    out = []
    for n in sizes:
        n = int(n)
        nz = rng.random((n, n)) < p_nonzero
        vals = rng.integers(1, vmax + 1, size=(n, n))
        out.append(np.where(nz, vals, 0).astype(np.int64))
    return out


def sparse_rows(n: int, seed: int, kmin: int = 3, kmax: int = 5) -> np.ndarray:
    """n x n 0/1 matrix whose rows hold kmin..kmax nonzeros at random columns.

    Row counts are uniform in [kmin, kmax] and the columns of a row are
    distinct; the whole matrix is redrawn until every column holds at least
    one nonzero.
    """
    rng = np.random.default_rng(seed)
    while True:
        a = np.zeros((n, n), dtype=np.int64)
        for i in range(n):
            k = int(rng.integers(kmin, kmax + 1))
            cols = rng.choice(n, size=k, replace=False)
            a[i, cols] = 1
        if (a.sum(axis=0) > 0).all():
            return a


def mixed_batch(seed: int, count3: int = 128, countsp: int = 128,
                n3=(40, 90), nsp=(40, 70)):
    """Mixed batch: ``count3`` random 3-regular adjacencies with n uniform in
    ``n3`` (n even) and ``countsp`` sparse-row matrices with n uniform in
    ``nsp``.  Returns a list of int64 matrices."""
    rng = np.random.default_rng(seed)
    mats = []
    for _ in range(count3):
        n = int(rng.integers(n3[0], n3[1] + 1))
        if n % 2:
            n += 1 if n < n3[1] else -1
        mats.append(regular3(n, int(rng.integers(1 << 62))))
    for _ in range(countsp):
        n = int(rng.integers(nsp[0], nsp[1] + 1))
        mats.append(sparse_rows(n, int(rng.integers(1 << 62))))
    return mats


def random_small(n: int, seed: int, lo: int = -3, hi: int = 3,
                 density: float = 1.0) -> np.ndarray:
    """Small signed integer matrix for exactness tests: entries uniform in
    [lo, hi], each kept with probability ``density``."""
    rng = np.random.default_rng(seed)
    v = rng.integers(lo, hi + 1, size=(n, n))
    keep = rng.random((n, n)) < density
    return np.where(keep, v, 0).astype(np.int64)


def random01(n: int, nonzeros: int, seed: int) -> np.ndarray:
    """n x n 0/1 matrix with ``nonzeros`` ones at uniformly random distinct
    positions, redrawn until every row and every column holds a one (the
    random (n, S) groups of the paper's Section 3.1 with S = nonzeros)."""
    rng = np.random.default_rng(seed)
    while True:
        flat = rng.choice(n * n, size=nonzeros, replace=False)
        a = np.zeros(n * n, dtype=np.int64)
        a[flat] = 1
        a = a.reshape(n, n)
        if (a.sum(axis=0) > 0).all() and (a.sum(axis=1) > 0).all():
            return a
