"""Pins of the CPU oracle against facts fixed by the paper and by mathematics
(closed forms, brute force on tiny inputs, invariances, bounds, printed data,
library routines for special cases).  No GPU needed."""
import math
import os

import numpy as np
import pytest

import oracle
import workloads as W
from conftest import GOLDEN


def perm_matrix(n, seed):
    p = np.random.default_rng(seed).permutation(n)
    m = np.zeros((n, n), dtype=np.int64)
    m[np.arange(n), p] = 1
    return m


def cyc(n):
    return np.eye(n, dtype=np.int64) + np.roll(np.eye(n, dtype=np.int64), 1, axis=1)


# ---------------------------------------------------------------- Eq. 1 closed forms
@pytest.mark.parametrize("n", range(1, 8))
def test_bruteforce_closed_forms(n):
    assert oracle.per_bruteforce(np.ones((n, n), np.int64)) == math.factorial(n)
    assert oracle.per_bruteforce(np.eye(n, dtype=np.int64)) == 1
    assert oracle.per_bruteforce(perm_matrix(n, n)) == 1
    if n >= 3:
        assert oracle.per_bruteforce(cyc(n)) == 2
    # one row scaled by c scales per by c (multilinearity)
    a = W.random_small(n, 100 + n)
    b = a.copy()
    b[0] *= 3
    assert oracle.per_bruteforce(b) == 3 * oracle.per_bruteforce(a)


def test_bruteforce_2x2_3x3_by_hand():
    assert oracle.per_bruteforce([[1, 2], [3, 4]]) == 1 * 4 + 2 * 3
    a = [[1, 2, 3], [4, 5, 6], [7, 8, 9]]
    # six permutation products of a 3x3 written out
    assert oracle.per_bruteforce(a) == 1*5*9 + 1*6*8 + 2*4*9 + 2*6*7 + 3*4*8 + 3*5*7


# ---------------------------------------------------------------- Ryser
@pytest.mark.parametrize("seed", range(12))
def test_ryser_matches_bruteforce(seed):
    n = 1 + seed % 8
    a = W.random_small(n, seed, lo=-4, hi=4, density=0.7)
    want = oracle.per_bruteforce(a)
    assert oracle.per_ryser_py(a) == want
    assert oracle.ryser(a) == want


@pytest.mark.parametrize("n", [8, 10, 12, 14])
def test_ryser_closed_forms(n):
    assert oracle.ryser(np.ones((n, n), np.int64)) == math.factorial(n)
    assert oracle.ryser(cyc(n)) == 2
    assert oracle.ryser(np.eye(n, dtype=np.int64)) == 1
    # per(c * J_n) = c^n n!
    assert oracle.ryser(3 * np.ones((n, n), np.int64)) == 3 ** n * math.factorial(n)


def test_ryser_large_values_exact():
    # per(J_20) = 20! needs more than 64 bits once multiplied out by entries 7
    n = 16
    a = 7 * np.ones((n, n), np.int64)
    assert oracle.ryser(a) == 7 ** n * math.factorial(n)


# ---------------------------------------------------------------- H_per / PH
@pytest.mark.parametrize("seed", range(16))
def test_hybrid_matches_bruteforce(seed):
    n = 2 + seed % 7
    dens = [0.3, 0.5, 0.8][seed % 3]
    a = W.random_small(n, 1000 + seed, lo=-3, hi=3, density=dens)
    want = oracle.per_bruteforce(a)
    for d, L in [(0, 0), (1, 0), (2, 0), (3, 3), (n, 0), (2, 5)]:
        assert oracle.permanent(a, d=d, L=L, threads=2) == want, (d, L)


@pytest.mark.parametrize("seed", range(10))
def test_e2_node_identity(seed):
    """Eq. 2: per(parent) = sum over children of coef * per(child), every
    child's permanent by brute force, one to three levels down."""
    n = 5 + seed % 4
    a = W.random_small(n, 2000 + seed, lo=0, hi=2, density=0.45)
    want = oracle.per_bruteforce(a)
    for d in (1, 2, 3):
        js = oracle.jobs(a, d)
        got = sum(c * oracle.per_bruteforce(m) for m, c in js)
        assert got == want, d
        for m, c in js:
            assert m.shape[0] >= n - d
            assert (m != 0).any(axis=0).all() and (m != 0).any(axis=1).all()


def test_e2_three_regular_children_shape():
    """On a 3-regular matrix every row has 3 nonzeros: the first pivot gives
    two (n-1)x(n-1) children, the second with coefficient a_{i,j3} = 1."""
    a = W.regular3(10, 5)
    js = oracle.jobs(a, 1)
    assert len(js) == 2
    assert all(m.shape == (9, 9) for m, _ in js)
    assert [c for _, c in js] == [1, 1]


# ---------------------------------------------------------------- Eq. 2 with three children (s >= 5)
@pytest.mark.parametrize("seed", range(12))
def test_three_child_split_matches_bruteforce(seed):
    """Dense nodes (s >= 5) split by Eq. 2's three children down to order
    2 give Eq. 1's value."""
    n = 5 + seed % 4
    a = W.random_small(n, 3000 + seed, lo=-2, hi=3, density=0.9)
    want = oracle.per_bruteforce(a)
    assert oracle.permanent(a, d=0, L=0, threads=2, three=True) == want
    assert oracle.permanent(a, d=3, L=2, threads=2, three=True) == want


@pytest.mark.parametrize("n", [5, 6, 7, 8])
def test_three_child_split_closed_form(n):
    assert oracle.permanent(np.ones((n, n), np.int64), three=True) == math.factorial(n)


@pytest.mark.parametrize("seed", range(6))
def test_three_child_node_identity(seed):
    """per(parent) = sum of coef * per(child) over the three-child job lists,
    children by brute force; a level never leaves s >= 5 nodes unsplit."""
    n = 6 + seed % 3
    a = W.random_small(n, 4000 + seed, lo=0, hi=2, density=0.85)
    want = oracle.per_bruteforce(a)
    for d in (1, 2, 3):
        js = oracle.jobs(a, d, three=True)
        assert sum(c * oracle.per_bruteforce(m) for m, c in js) == want, d


def test_three_child_first_level_shapes():
    """A 7x7 matrix whose sparsest line is row 0 with six nonzeros: A1 and A2
    lose a row and a column; A3 keeps the order with row 0's first four
    nonzeros cleared and everything else unchanged."""
    a = np.ones((7, 7), np.int64)
    a[0, 6] = 0
    a[1:, 0] = 2
    js = oracle.jobs(a, 1, three=True)
    assert [m.shape[0] for m, _ in js] == [6, 6, 7]
    a3 = js[2][0]
    assert (a3[0, :4] == 0).all() and (a3[0, 4:] == a[0, 4:]).all() and (a3[1:] == a[1:]).all()
    assert len(oracle.jobs(a, 1)) == 1  # without the option the node is a leaf, carried


def test_zero_line_and_empty():
    a = W.random_small(6, 3)
    a[2] = 0
    assert oracle.permanent(a) == 0
    assert oracle.jobs(a, 2) == []
    assert oracle.permanent(np.zeros((0, 0), np.int64)) == 1


def test_permutation_matrices_through_hybrid():
    for n in (5, 12, 30):
        assert oracle.permanent(perm_matrix(n, n)) == 1
        assert oracle.permanent(cyc(n)) == 2


# ---------------------------------------------------------------- invariances
@pytest.mark.parametrize("n,seed", [(20, 1), (24, 2), (30, 3)])
def test_invariances_three_regular(n, seed):
    a = W.regular3(n, seed)
    p = oracle.permanent(a)
    rng = np.random.default_rng(seed)
    r, c = rng.permutation(n), rng.permutation(n)
    assert oracle.permanent(a[np.ix_(r, c)]) == p
    assert oracle.permanent(a.T.copy()) == p
    # block diagonal: per(A (+) B) = per(A) per(B)
    b = W.regular3(12, seed + 7)
    blk = np.zeros((n + 12, n + 12), np.int64)
    blk[:n, :n] = a
    blk[n:, n:] = b
    assert oracle.permanent(blk) == p * oracle.permanent(b)


@pytest.mark.parametrize("n,seed", [(20, 11), (36, 1), (36, 2), (40, 3)])
def test_three_regular_bounds(n, seed):
    """Schrijver (4/3)^n <= per(A) <= Bregman 6^(n/3) for 3-regular 0/1."""
    a = W.regular3(n, seed)
    p = oracle.permanent(a, d=6)
    assert oracle.schrijver_lower_bound(n, 3) <= p <= 6 ** (n / 3) * (1 + 1e-12)
    assert p <= oracle.bregman_bound(a) * (1 + 1e-12)
    assert p <= oracle.rowcol_bound(a)


def test_depth_independence():
    a = W.regular3(36, 1)
    vals = {oracle.permanent(a, d=d, L=L) for d, L in [(0, 0), (5, 0), (12, 0), (20, 16), (20, 0)]}
    assert len(vals) == 1


# ---------------------------------------------------------------- printed data
def test_t12_fixture_sums_to_printed_total():
    vals = {}
    total = None
    with open(os.path.join(GOLDEN, "t12_c100_subpermanents.txt")) as f:
        for line in f:
            if line.startswith("#"):
                continue
            k, v = line.split()
            if k == "total":
                total = int(v)
            else:
                vals[int(k)] = int(v)
    assert sorted(vals) == list(range(1, 160))
    assert total == 149364113290700
    assert sum(vals.values()) == total
    # the total lies within the 3-regular bounds for n = 100
    assert (4 / 3) ** 100 <= total <= 6 ** (100 / 3)


def _pentagons(a):
    n = a.shape[0]
    nb = [set(np.flatnonzero(a[i])) for i in range(n)]
    cyc5 = set()
    for v in range(n):
        for u1 in nb[v]:
            for u2 in nb[u1] - {v}:
                for u3 in nb[u2] - {v, u1}:
                    for u4 in nb[u3] - {v, u1, u2}:
                        if v in nb[u4]:
                            cyc5.add(frozenset((v, u1, u2, u3, u4)))
    return len(cyc5)


def test_appendix_graphs_are_fullerenes(c100_adjacency, c60_paper_adjacency):
    for a, n in ((c100_adjacency, 100), (c60_paper_adjacency, 60)):
        assert a.shape == (n, n)
        assert (a == a.T).all() and (np.diag(a) == 0).all()
        assert (a.sum(axis=1) == 3).all()
        assert np.trace(a @ a @ a) == 0  # triangle-free
        assert _pentagons(a) == 12  # Euler: every fullerene has 12 pentagons


def test_c60_coordinates_match_paper_list(c60_paper_adjacency):
    """The truncated icosahedron built from its coordinates and the paper's
    C60 list are the same graph up to vertex order: equal spectra and equal
    permanents (different vertex orders give different expansion trees)."""
    a = W.c60(seed=7)
    assert (a.sum(axis=1) == 3).all() and _pentagons(a) == 12
    ev1 = np.sort(np.linalg.eigvalsh(a.astype(float)))
    ev2 = np.sort(np.linalg.eigvalsh(c60_paper_adjacency.astype(float)))
    assert np.allclose(ev1, ev2, atol=1e-9)
    p1 = oracle.permanent(a, d=12)
    p2 = oracle.permanent(c60_paper_adjacency, d=12)
    assert p1 == p2
    assert oracle.schrijver_lower_bound(60, 3) <= p1 <= 6 ** 20


# ---------------------------------------------------------------- KKLLL
@pytest.mark.parametrize("seed", range(6))
def test_kklll_unbiased_exact_enumeration(seed):
    """The paper's Theorem: E|det W|^2 = per(B), by enumerating all 3^nnz
    draws for a tiny pattern."""
    rng = np.random.default_rng(seed)
    n = 3 + seed % 2
    while True:
        b = (rng.random((n, n)) < 0.6).astype(np.int64)
        if 4 <= b.sum() <= 10:
            break
    assert abs(oracle.kklll_exact_mean(b) - oracle.per_bruteforce(b)) < 1e-8


@pytest.mark.parametrize("seed", range(5))
def test_det_partial_pivot_matches_library(seed):
    rng = np.random.default_rng(seed)
    m = 2 + 3 * seed
    w = rng.normal(size=(m, m)) + 1j * rng.normal(size=(m, m))
    la, zero = oracle.det_partial_pivot(w)
    d = np.linalg.det(w)
    assert not zero
    assert abs(la - math.log(abs(d) ** 2)) < 1e-9
    w[:, 1] = 0
    assert oracle.det_partial_pivot(w)[1]


def test_splitmix64_published_sequence():
    """SplitMix64 seeded with 0: the first three published outputs."""
    from oracle.kklll import splitmix64_mix
    g = 0x9E3779B97F4A7C15
    outs = [splitmix64_mix((k * g) & ((1 << 64) - 1)) for k in range(3)]
    assert outs == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_kklll_choice_uniform():
    counts = np.bincount([oracle.kklll_choice(5, 3, t, e) for t in range(60) for e in range(100)],
                         minlength=3)
    assert counts.sum() == 6000 and (abs(counts - 2000) < 200).all()


def test_kklll_estimate_near_permanent():
    """With many trials the mean is near per(B) (loose statistical check)."""
    a = W.regular3(10, 4)
    p = oracle.permanent(a)
    la = oracle.kklll_log_ap(a, seed=1, job=0, trials=2000)
    assert abs(la - math.log(p)) < 0.35


@pytest.mark.parametrize("perm,seed,job", [([1, 2, 0], 3, 0), ([4, 0, 3, 1, 2, 5], 11, 7),
                                           (list(range(9))[::-1], 2, 3)])
def test_kklll_permutation_pattern_is_exactly_one(perm, seed, job):
    """A permutation pattern has per(B) = 1 and |det W|^2 = prod |w|^2 = 1 in
    every trial (each w a cube root of unity), so log AP = 0 for any trial
    count and stream position."""
    m = len(perm)
    b = np.zeros((m, m), dtype=np.int64)
    b[np.arange(m), perm] = 1
    for trials in (1, 5, 40):
        assert abs(oracle.kklll_log_ap(b, seed=seed, job=job, trials=trials)) < 1e-12


def test_kklll_block_diagonal_permutation_blocks():
    """Block diagonal of 1x1 blocks and permutation blocks (again a
    permutation pattern, now with blocks of several orders): log AP = 0."""
    blocks = [np.ones((1, 1)), np.eye(3)[[2, 0, 1]], np.ones((1, 1)), np.eye(4)[[1, 3, 0, 2]]]
    m = sum(x.shape[0] for x in blocks)
    b = np.zeros((m, m), dtype=np.int64)
    k = 0
    for x in blocks:
        r = x.shape[0]
        b[k:k + r, k:k + r] = x
        k += r
    assert abs(oracle.kklll_log_ap(b, seed=9, job=4, trials=25)) < 1e-12


@pytest.mark.parametrize("seed,job,trials", [(1, 0, 4), (7, 3, 9), (1234, 11, 64), (5, 2, 1)])
def test_kklll_all_ones_2x2_exact_mean(seed, job, trials):
    """All-ones 2 x 2 pattern: det W = w00 w11 - w01 w10 = u^(c00+c11) - u^(c01+c10)
    with u = exp(2 pi i / 3), so |det W|^2 = 0 when c00 + c11 = c01 + c10 (mod 3)
    and |1 - u|^2 = 3 otherwise.  Reading each trial's draws back with
    kklll_choice gives the mean as an exact rational 3 k / T, which pins the
    log of the mean over trials (not a mean of logs) and the all-singular
    case (-inf)."""
    b = np.ones((2, 2), dtype=np.int64)
    k = 0
    for t in range(trials):
        c = [oracle.kklll_choice(seed, job, t, e) for e in range(4)]  # e = 2 i + j
        k += (c[0] + c[3] - c[1] - c[2]) % 3 != 0
    got = oracle.kklll_log_ap(b, seed=seed, job=job, trials=trials)
    if k == 0:
        assert got == -math.inf
    else:
        assert abs(got - math.log(3.0 * k / trials)) < 1e-12
    # a stream where trials differ, so a mean of logs would not agree
    if 0 < k < trials:
        assert abs(got - math.log(3.0)) > 1e-3


def test_kklll_all_ones_2x2_stream_has_both_outcomes():
    """The pin above sees both singular and regular trials on this stream."""
    ks = [(oracle.kklll_choice(1234, 11, t, 0) + oracle.kklll_choice(1234, 11, t, 3)
           - oracle.kklll_choice(1234, 11, t, 1) - oracle.kklll_choice(1234, 11, t, 2)) % 3 != 0
          for t in range(64)]
    assert 0 < sum(ks) < 64


# ---------------------------------------------------------------- scheduling
def test_efficiency_reproduces_table_t5():
    """Tables T5-T7 (C100): printed efficiency = T1 / (m Tm)."""
    t1 = 118413.21
    rows = [(2, 59265.87, 0.9990), (4, 29902.32, 0.9900), (8, 15243.71, 0.9710),
            (16, 7829.07, 0.9453), (32, 4387.49, 0.8434),  # T5
            (32, 3796.85, 0.9746), (32, 3911.22, 0.9461)]  # T6, T7
    for m, tm, eff in rows:
        assert abs(oracle.efficiency(t1, tm, m) - eff) < 1.5e-3


def test_list_schedule_small_cases():
    assert oracle.list_schedule([3, 3, 2, 2, 2], 2) == 7  # LS in given order
    order = oracle.lpt_order([3, 3, 2, 2, 2])
    assert order == [0, 1, 2, 3, 4]
    assert oracle.list_schedule([2, 2, 2, 3, 3], 2) == 7
    assert oracle.list_schedule([2, 2, 2, 3, 3], 2, oracle.lpt_order([2, 2, 2, 3, 3])) == 7
    # LPT worst case 4/3 - 1/(3m) against the brute-force optimum
    rng = np.random.default_rng(0)
    import itertools
    for _ in range(30):
        t = rng.integers(1, 20, size=7).tolist()
        m = 3
        opt = min(max(sum(t[j] for j in range(7) if assign[j] == k) for k in range(m))
                  for assign in itertools.product(range(m), repeat=7))
        lpt = oracle.list_schedule(t, m, oracle.lpt_order(t))
        assert lpt <= (4 / 3 - 1 / (3 * m)) * opt + 1e-9
        assert oracle.list_schedule(t, m) <= (2 - 1 / m) * opt + 1e-9


def test_kendall_tau_b_matches_library():
    scipy_stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(3)
    for _ in range(5):
        x = rng.integers(0, 6, size=40)
        y = x + rng.integers(0, 4, size=40)
        want = scipy_stats.kendalltau(x, y).statistic
        assert abs(oracle.kendall_tau_b(x.tolist(), y.tolist()) - want) < 1e-12
    assert oracle.kendall_tau_b([1, 2, 3], [1, 2, 3]) == 1.0
    assert oracle.kendall_tau_b([1, 2, 3], [3, 2, 1]) == -1.0
