"""The residue path (perm_opts.modulus) and perm_crt against the oracle.

Eq. 2 and Ryser's formula are identities over any commutative ring, so the
whole path run modulo a prime p gives per(A) mod p; residues for several
primes and the Chinese remainder theorem give per(A) itself, also beyond
the 256-bit ring.  Residues must equal the oracle's exact value mod p
(bit-exact); CRT values must equal the integers they came from; the
permanental polynomial per(xI - A) (Section 4.2, Eq. 11) must equal the
oracle's brute force, the oracle's values interpolated, and the closed
forms of a graph's low-order coefficients."""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from oracle import polynomial as OP

pytestmark = pytest.mark.gpu

pk = pytest.importorskip("paper_1112_6072_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)
from paper_1112_6072_gb300 import polynomial as PP  # noqa: E402

PRIMES = [3, 5, 65537, 2147483647]
DRIVERS = {"walk": dict(expand_walk=True), "fused": dict(expand_walk=False, fused_levels=True),
           "levels": dict(expand_walk=False, fused_levels=False)}


def residues(mats, p, natural=False, **kw):
    with pk.Plan(mats, modulus=p, **kw) as plan:
        plan.expand()
        if natural:
            plan.evaluate(order=np.arange(plan.njobs, dtype=np.uint32))
        else:
            plan.evaluate()
        got = plan.results()
        assert all(plan.result_bits(i) == 0 for i in range(len(mats)))
        assert all(0 <= v < p for v in got)
    return got


def leaf_mats():
    rng = np.random.default_rng(5)
    mats = [W.leaf_batch(1, int(rng.integers(1 << 30)), nmin=n, nmax=n)[0] for n in range(1, 25)]
    mats += [W.random_small(n, 90 + n, lo=-5, hi=5) for n in (2, 7, 13, 16)]
    mats += [np.ones((n, n), np.int64) for n in (20, 24)]
    # entries far beyond the exact path's 2^31 limit: reduced modulo p first
    mats += [rng.integers(-(1 << 40), 1 << 40, size=(9, 9)).astype(np.int64)]
    mats += [np.zeros((0, 0), np.int64), np.zeros((4, 4), np.int64)]
    return mats


def exact(m):
    n = m.shape[0]
    if n == 0:
        return 1
    if n >= 20 and (m == 1).all():
        return math.factorial(n)
    if np.abs(m).max() >= 1 << 31:
        return oracle.per_ryser_py(m)
    return oracle.permanent(m)


@pytest.fixture(scope="module")
def leaf_case():
    mats = leaf_mats()
    return mats, [exact(m) for m in mats]


@pytest.mark.parametrize("p", PRIMES)
def test_leaf_residues(p, leaf_case):
    mats, vals = leaf_case
    want = [v % p for v in vals]
    assert residues(mats, p, natural=True) == want
    assert residues(mats, p) == want  # the planned order


@pytest.mark.parametrize("driver", list(DRIVERS))
@pytest.mark.parametrize("p", [65537, 2147483647])
def test_hybrid_residues(driver, p):
    """Expansion (every driver), coefficients and leaves modulo p: C60 at
    leaf order 11 and a 36-vertex cubic graph split at depth 20."""
    assert residues([W.c60(60)], p, leaf_size=11, **DRIVERS[driver]) == [395974320 % p]
    a = W.regular3(36, 1)
    assert residues([a], p, split_depth=20, leaf_size=16, **DRIVERS[driver]) == [oracle.permanent(a) % p]


@pytest.mark.parametrize("p", [3, 65537, 2147483647])
def test_dense_split_and_depth_first_residues(p):
    """The three-child split and the depth-first evaluator (jobs above the
    leaf order) modulo p, signed entries."""
    rng = np.random.default_rng(17)
    a = W.sparse_rows(30, 3, kmin=4, kmax=6) * rng.choice([-2, -1, 1, 2], size=(30, 30))
    want = oracle.permanent(a) % p
    assert residues([a], p, split_depth=4, leaf_size=10, dense_split=True) == [want]
    assert residues([a], p, split_depth=0, leaf_size=12) == [want]
    assert residues([a], p, split_depth=2, leaf_size=20) == [want]


def block_matrix(sizes, bits, seed):
    """A block-diagonal matrix of dense signed blocks with rows and columns
    shuffled: per = the product of the blocks' permanents."""
    rng = np.random.default_rng(seed)
    n = sum(sizes)
    a = np.zeros((n, n), np.int64)
    want, o = 1, 0
    for s in sizes:
        b = rng.integers(-(1 << bits), 1 << bits, size=(s, s)).astype(np.int64)
        a[o:o + s, o:o + s] = b
        want *= oracle.per_ryser_py(b)
        o += s
    r, c = rng.permutation(n), rng.permutation(n)
    return a[r][:, c], want


@pytest.mark.parametrize("kw", [dict(leaf_size=12), dict(split_depth=3, leaf_size=6),
                                dict(split_depth=2, leaf_size=10, dense_split=True)])
def test_beyond_ring_by_crt(kw):
    """|per(A)| ~ 2^530: the exact path refuses (PERM_EOVERFLOW); the
    residues of 19 primes and perm_crt give per(A) exactly."""
    a, want = block_matrix([5, 6, 7], 28, seed=3)
    assert want.bit_length() > 400
    with pytest.raises(pk.PermError) as e:
        pk.Plan([a], **kw)
    assert e.value.status == 2
    primes = PP.primes_for(want.bit_length())
    res = np.array([[residues([a], p, **kw)[0] for p in primes]], dtype=np.uint32)
    assert pk.crt(res, primes) == [want]


def test_crt_round_trip():
    rng = np.random.default_rng(9)
    for k in (1, 2, 5, 17, 64):
        primes = PP.primes_below(1 << 31, k)
        half = math.prod(primes) // 2
        vals = [0, 1, -1, half, -half, half - 1]
        vals += [int.from_bytes(rng.bytes(4 * k), "little") % (2 * half + 1) - half for _ in range(200)]
        res = np.array([[v % p for p in primes] for v in vals], dtype=np.uint32)
        assert pk.crt(res, primes) == vals
    for bad in ([4, 7], [7, 7], [2, 7], [1 << 31, 7]):
        with pytest.raises(pk.PermError):
            pk.crt(np.zeros((1, 2), np.uint32), bad)
    with pytest.raises(pk.PermError):
        pk.crt(np.array([[7, 0]], np.uint32), [7, 11])  # residue not below its prime


def test_modulus_rejects_non_primes():
    for p in (1, 2, 9, 65535, 1 << 31):
        with pytest.raises(pk.PermError) as e:
            pk.Plan([np.eye(3, dtype=np.int64)], modulus=p)
        assert e.value.status == 1


# ------------------------------------------------- permanental polynomial
def test_polynomial_small_matrices_vs_brute_force():
    rng = np.random.default_rng(21)
    prism = np.zeros((6, 6), np.int64)
    for u, v in [(0, 1), (1, 2), (2, 0), (3, 4), (4, 5), (5, 3), (0, 3), (1, 4), (2, 5)]:
        prism[u, v] = prism[v, u] = 1
    cases = [prism, rng.integers(-3, 4, size=(7, 7)).astype(np.int64), np.ones((8, 8), np.int64),
             np.zeros((3, 3), np.int64), np.array([[5]], np.int64)]
    for a in cases:
        assert PP.permanental_polynomial(a) == OP.permanental_polynomial_bruteforce(a)
    assert PP.permanental_polynomial(np.zeros((0, 0), np.int64)) == [1]


@pytest.mark.parametrize("kw", [dict(), dict(split_depth=4, leaf_size=6)])
def test_polynomial_cubic16_vs_oracle_values(kw):
    """A 16-vertex cubic graph: the oracle's exact per(xI - A) at 17 points,
    interpolated, against the library (residues, interpolation modulo p,
    CRT), leaf-only and hybrid; and the exact values at the points."""
    a = W.regular3(16, 1)
    xs = list(range(-8, 9))
    ys = [oracle.permanent(x * np.eye(16, dtype=np.int64) - a) for x in xs]
    want = OP.interpolate(xs, ys)
    assert want[-1] == 1 and want[14] == 24
    assert PP.permanental_polynomial(a, **kw) == want
    assert PP.values(a, xs, **kw) == ys


def cycles(a, length):
    """Undirected cycles of the given length in a simple graph (brute force
    over paths that start at their smallest vertex)."""
    n = a.shape[0]
    nb = [np.flatnonzero(a[v]).tolist() for v in range(n)]
    count = 0

    def walk(start, v, seen, k):
        nonlocal count
        for w in nb[v]:
            if k == length and w == start:
                count += 1
            elif k < length and w > start and w not in seen:
                walk(start, w, seen | {w}, k + 1)

    for s in range(n):
        walk(s, s, {s}, 1)
    return count // 2  # each cycle in both directions


def graph_coefficient_pins(a, c):
    """The coefficient of x^(n-k) is the sum of per(-A_S) over the k-vertex
    subsets S: (-1)^k times the fixed-point-free permutations along edges of
    the induced subgraphs.  So x^n: 1; x^(n-1): 0; x^(n-2): the edges;
    x^(n-3): -2 triangles; x^(n-4): disjoint edge pairs + 2 four-cycles;
    x^(n-5): -2 five-cycles - 2 (triangle, disjoint edge) pairs (checked
    where there is no triangle)."""
    n = a.shape[0]
    edges = int(a.sum()) // 2
    deg = a.sum(axis=1)
    tri, c4, c5 = cycles(a, 3), cycles(a, 4), cycles(a, 5)
    assert c[n] == 1 and c[n - 1] == 0 and c[n - 2] == edges and c[n - 3] == -2 * tri
    assert c[n - 4] == math.comb(edges, 2) - sum(math.comb(int(d), 2) for d in deg) + 2 * c4
    if tri == 0:
        assert c[n - 5] == -2 * c5
    # A >= 0: the coefficient of x^k has the sign (-1)^(n-k) or is zero
    assert all((v > 0) == ((n - k) % 2 == 0) for k, v in enumerate(c) if v)
    return edges, tri, c4, c5


def test_polynomial_graph_pins_cubic24():
    a = W.regular3(24, 2)
    c = PP.permanental_polynomial(a, leaf_size=10)
    graph_coefficient_pins(a, c)
    assert c[0] == oracle.permanent(a)


def test_shifted_value_by_crt():
    """per(I - A) of a 36-vertex cubic graph from three primes' residues and
    perm_crt equals the exact path's value (|per(I - A)| <= 4^36)."""
    a = W.regular3(36, 1)
    with pk.Plan([np.eye(36, dtype=np.int64) - a], leaf_size=12) as plan:
        plan.expand()
        plan.evaluate()
        want = plan.results()[0]
    assert PP.values(a, [1], leaf_size=12) == [want]
    assert want != 0
