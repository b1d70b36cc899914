"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Permanents, coefficients and job lists must agree bit for bit; the KKLLL
estimate within 1e-5 relative (FP32 against fp64); the cost-network
gradient within FP32 rounding of the fp64 oracle."""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu

pk = pytest.importorskip("paper_1112_6072_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

M256 = (1 << 256) - 1


def signed_low(v, bits):
    v &= (1 << bits) - 1
    return v - (1 << bits) if v >> (bits - 1) else v


# ---------------------------------------------------------------- leaf Ryser (K2)
def test_leaf_batch_small_sizes_all_paths():
    """n = 1..20 dense small-integer leaves, every register width, a ragged
    tail of tiny jobs, and the 128-bit ring."""
    mats = []
    rng = np.random.default_rng(11)
    for n in list(range(1, 21)) + [3, 7, 12, 17, 19]:
        mats.append(W.leaf_batch(1, int(rng.integers(1 << 30)), nmin=n, nmax=n)[0])
    with pk.Plan(mats) as plan:
        plan.expand()
        plan.evaluate(order=np.arange(plan.njobs, dtype=np.uint32))
        got = plan.results()
    want = [oracle.permanent(m) for m in mats]
    assert got == want


def test_leaf_batch_signed_and_wide():
    """Signed entries (cancellation), the 256-bit ring and bit classes 15 and
    31 of the row-product tree."""
    mats = [W.random_small(n, 50 + n, lo=-3, hi=3) for n in range(2, 17)]
    mats += [W.random_small(12, 7, lo=-900, hi=1000)]           # bit class 15, 256-bit ring
    mats += [W.random_small(6, 8, lo=-(1 << 20), hi=1 << 20)]   # bit class 31
    mats += [np.ones((n, n), np.int64) for n in (20, 22, 24)]    # n! beyond 64 bits
    with pk.Plan(mats) as plan:
        plan.expand()
        plan.evaluate(order=np.arange(plan.njobs, dtype=np.uint32))
        got = plan.results()
    want = [oracle.ryser(m) if m.shape[0] <= 16 else oracle.permanent(m) for m in mats]
    assert got[-3:] == [math.factorial(20), math.factorial(22), math.factorial(24)]
    assert got == want


def _column_supports(n, supports, seed):
    """n x n matrix whose column j holds supports[j] entries in 1..3 at random rows."""
    rng = np.random.default_rng(seed)
    a = np.zeros((n, n), dtype=np.int64)
    for j, k in enumerate(supports):
        rows = rng.choice(n, size=k, replace=False)
        a[rows, j] = rng.integers(1, 4, size=k)
    return a


def _sparsest_pair(a):
    """(union, |rows of a|, |rows of b|) of the column pair touching the
    fewest rows, the lowest pair on ties (the blocked walk's choice)."""
    nz = a != 0
    best = None
    for x in range(a.shape[0]):
        for y in range(x + 1, a.shape[0]):
            u = int((nz[:, x] | nz[:, y]).sum())
            if best is None or u < best[0]:
                best = (u, int(nz[:, x].sum()), int(nz[:, y].sum()))
    return best


def test_blocked_walk_orientation_and_fallback():
    """Leaves whose sparsest column pair touches 9-16 rows: with the lower
    column over 8 rows and the other within 8 (column 1 becomes Gray column
    0), and with both over 8 (the plain walk); every line holds >= 5 entries,
    so the depth-first evaluator also takes each matrix as one leaf."""
    swap = [_column_supports(20, [9] * 19 + [7], s) for s in (2, 4)]
    plain = [_column_supports(20, [9] * 20, s) for s in (1, 2, 4)]
    for a in swap:
        u, ka, kb = _sparsest_pair(a)
        assert 8 < u <= 16 and ka > 8 and kb <= 8
    for a in plain:
        u, ka, kb = _sparsest_pair(a)
        assert 8 < u <= 16 and ka > 8 and kb > 8
    mats = swap + plain
    assert min(int((m != 0).sum(axis=1).min()) for m in mats) >= 5
    want = [oracle.permanent(m) for m in mats]
    with pk.Plan(mats) as plan:  # leaf batch
        plan.expand()
        plan.evaluate()
        assert plan.results() == want
    with pk.Plan(mats, split_depth=0, leaf_size=12) as plan:  # depth-first, one leaf each
        plan.expand()
        plan.evaluate()
        assert plan.results() == want


def test_leaf_chunk_sizes_agree():
    mats = W.leaf_batch(24, seed=5, nmin=14, nmax=20)
    res = []
    for c in (1, 3, 6, 10):
        with pk.Plan(mats, chunk_log2=c) as plan:
            plan.expand()
            plan.evaluate(order=np.arange(plan.njobs, dtype=np.uint32))
            res.append(plan.results())
    assert all(r == res[0] for r in res)
    assert res[0] == [oracle.permanent(m) for m in mats]


def test_leaf_batch_full_size_sample():
    """Config-2 shape (n in [12, 24], P(nonzero) = 0.35, values 1..3): a
    seeded sample at full size, including the largest order."""
    mats = W.leaf_batch(10, seed=2024)
    mats += W.leaf_batch(1, seed=99, nmin=24, nmax=24)
    with pk.Plan(mats) as plan:
        plan.expand()
        plan.evaluate()
        got = plan.results()
    want = oracle.job_permanents(mats)
    assert got == want


def test_graph_replay_matches_eval():
    """The evaluation captured as a CUDA graph and replayed gives the same
    permanents and job values, replay after replay (leaf and depth-first)."""
    mats = W.leaf_batch(30, seed=8, nmin=10, nmax=20) + [W.regular3(30, 3)]
    with pk.Plan(mats, leaf_size=10) as plan:
        plan.expand()
        rec = plan.evaluate(records=True)
        want = plan.results()
        for _ in range(3):
            rec2 = plan.replay(records=True)
            assert plan.results() == want
            assert [r.value_mod for r in rec2] == [r.value_mod for r in rec]
    assert want[-1] == oracle.permanent(mats[-1])
    with pk.Plan([W.regular3(12, 1)]) as plan:
        plan.expand()
        with pytest.raises(pk.PermError):
            plan.replay()


def test_zero_and_empty_inputs():
    z = W.random_small(5, 1)
    z[:, 2] = 0
    with pk.Plan([z, np.zeros((0, 0), np.int64), np.eye(3, dtype=np.int64)]) as plan:
        plan.expand()
        plan.evaluate()
        assert plan.results() == [0, 1, 1]


def test_invalid_arguments_rejected():
    with pytest.raises(pk.PermError):
        pk.Plan([np.full((3, 3), 1 << 40, dtype=np.int64)])
    with pytest.raises(pk.PermError):
        pk.Plan([np.ones((130, 130), np.int64)])
    a = W.regular3(12, 1)
    with pk.Plan([a], split_depth=2, leaf_size=4) as plan:
        plan.expand()
        with pytest.raises(pk.PermError):
            plan.evaluate(order=np.zeros(plan.njobs, dtype=np.uint32) if plan.njobs > 1 else [5])


# ---------------------------------------------------------------- expansion (K1)
DRIVERS = {"walk": dict(expand_walk=True), "fused": dict(expand_walk=False, fused_levels=True),
           "levels": dict(expand_walk=False, fused_levels=False)}


def _driver_jobs(mats, driver, **kw):
    with pk.Plan(mats, **DRIVERS[driver], **kw) as plan:
        plan.expand()
        return plan.jobs_export(), plan.expand_driver


def _same_jobs(got, want):
    assert len(got) == len(want)
    for (gi, gm, gc), (wi, wm, wc) in zip(got, want):
        assert gi == wi and gm.shape == wm.shape and (gm == wm).all() and gc == wc


@pytest.mark.parametrize("driver", list(DRIVERS))
@pytest.mark.parametrize("n,seed,d,L", [(10, 1, 3, 2), (16, 2, 6, 4), (24, 3, 10, 8), (36, 1, 20, 16)])
def test_job_list_matches_oracle(n, seed, d, L, driver):
    a = W.regular3(n, seed)
    got, used = _driver_jobs([a], driver, split_depth=d, leaf_size=L)
    if driver == "walk":
        assert used == "walk"
    want = oracle.jobs(a, d, L)
    assert len(got) == len(want)
    for (mi, gm, gc), (wm, wc) in zip(got, want):
        assert mi == 0
        assert gm.shape == wm.shape and (gm == wm).all()
        assert gc == wc % (1 << 256)


@pytest.mark.parametrize("driver", list(DRIVERS))
def test_job_list_signed_sparse(driver):
    a = W.random_small(14, 77, lo=-2, hi=2, density=0.25)
    a[np.arange(14), np.arange(14)] = 1  # no zero line
    got, _ = _driver_jobs([a], driver, split_depth=5, leaf_size=3)
    want = oracle.jobs(a, 5, 3)
    assert len(got) == len(want)
    for (_, gm, gc), (wm, wc) in zip(got, want):
        assert (gm == wm).all() and gc == wc % (1 << 256)


@pytest.mark.parametrize("driver", list(DRIVERS))
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_dense_split_job_list_matches_oracle(seed, driver):
    """Eq. 2 with the third child (s >= 5): the expansion's job list equals
    the oracle's, and some jobs kept their order through a level."""
    a = W.random_small(12, 500 + seed, lo=1, hi=2, density=0.75)
    # every line holds at least five nonzeros, so the root takes three children
    assert min((a != 0).sum(axis=0).min(), (a != 0).sum(axis=1).min()) >= 5
    got, used = _driver_jobs([a], driver, split_depth=4, leaf_size=3, dense_split=True)
    if driver == "walk":
        assert used == "walk"
    want = oracle.jobs(a, 4, 3, three=True)
    assert len(got) == len(want) > 0
    for (_, gm, gc), (wm, wc) in zip(got, want):
        assert gm.shape == wm.shape and (gm == wm).all() and gc == wc % (1 << 256)
    assert any(m.shape[0] > 12 - 4 for _, m, _ in got)


@pytest.mark.parametrize("case", ["c60", "batch", "regular80", "signed30"])
def test_drivers_same_jobs(case):
    """The traversal, the single-launch multi-level expansion (with its
    buffer growth and hand-over to per-level launches) and the per-level
    launches yield one job list."""
    if case == "c60":
        mats, kw = [W.c60(60)], dict(leaf_size=12)
    elif case == "batch":
        mats = [W.regular3(n, s) for n, s in ((20, 1), (28, 2), (40, 3), (12, 4))] + [W.sparse_rows(24, 5)]
        kw = dict(split_depth=9, leaf_size=6)
    elif case == "regular80":  # frontier beyond the first buffers: growth and copies
        mats, kw = [W.regular3(80, 3)], dict(split_depth=19, leaf_size=10)
    else:
        a = W.random_small(30, 9, lo=-3, hi=3, density=0.15)
        a[np.arange(30), (np.arange(30) * 7) % 30] = 2
        mats, kw = [a], dict(split_depth=12, leaf_size=5)
    want, _ = _driver_jobs(mats, "levels", **kw)
    assert len(want) > 0
    for driver in ("fused", "walk"):
        got, used = _driver_jobs(mats, driver, **kw)
        if driver == "walk":
            # roots above the traversal's 64-wide tile go level by level
            assert used == ("fused" if case == "regular80" else "walk")
        _same_jobs(got, want)


@pytest.mark.parametrize("case,expect", [("c60_L12", "walk"), ("c60_L8", "walk"), ("same_order_batch", "walk"),
                                         ("mixed_orders", "fused"), ("regular80", "fused")])
def test_walk_automatic_depth(case, expect):
    """Automatic depth: the traversal runs to the end of the tree and replays
    the level rule on its per-depth counts -- accepted when the rule reaches
    the end (C60, leaf order 12: 78,425 jobs), run again at the depth the
    rule stops at (leaf order 8: the count passes 2^17 one level above the
    end), or handed to the level-by-level driver (its buffers fill for
    n = 80; matrices of several orders need the waiting band).  The job list
    is the per-level driver's in every case."""
    if case == "c60_L12":
        mats, kw = [W.c60(60)], dict(leaf_size=12)
    elif case == "c60_L8":
        mats, kw = [W.c60(60)], dict(leaf_size=8)
    elif case == "same_order_batch":
        mats, kw = [W.regular3(30, s) for s in (1, 2, 3)], dict(leaf_size=10)
    elif case == "mixed_orders":
        mats, kw = [W.regular3(n, 1) for n in (24, 30)], dict(leaf_size=10)
    else:
        mats, kw = [W.regular3(80, 2)], dict(leaf_size=12)
    want, _ = _driver_jobs(mats, "levels", **kw)
    got, used = _driver_jobs(mats, "walk", **kw)
    assert used == expect
    _same_jobs(got, want)


# ---------------------------------------------------------------- hybrid end to end (K1+K3+K2+K6)
def test_config1_regular36_d20_L16():
    a = W.regular3(36, 1)
    with pk.Plan([a], split_depth=20, leaf_size=16) as plan:
        plan.expand()
        rec = plan.evaluate(records=True)
        got = plan.result(0)
        bits = plan.result_bits(0)
    assert got == oracle.permanent(a)
    # every job's coef * per(job) against the oracle's job values
    jobs = oracle.jobs(a, 20, 16)
    pj = oracle.job_permanents([m for m, _ in jobs])
    for r, (m, c), p in zip(rec, jobs, pj):
        assert signed_low(r.value_mod, bits) == c * p


@pytest.mark.parametrize("d,L", [(0, 8), (6, 8), (10, 12), (14, 6), (4, 2)])
def test_depth_first_evaluator(d, L):
    """Jobs above the leaf order go through the depth-first evaluator."""
    a = W.regular3(36, 2)
    with pk.Plan([a], split_depth=d, leaf_size=L) as plan:
        plan.expand()
        rec = plan.evaluate(records=True)
        got = plan.result(0)
    assert got == oracle.permanent(a)
    assert sum(r.nodes for r in rec) >= len(rec)


def test_depth_first_signed_and_column_pivots():
    for seed in range(4):
        a = W.random_small(18, 300 + seed, lo=-2, hi=3, density=0.3)
        a[np.arange(18), (np.arange(18) + seed) % 18] = 1
        with pk.Plan([a], split_depth=3, leaf_size=6) as plan:
            plan.expand()
            plan.evaluate()
            assert plan.result(0) == oracle.permanent(a)


def test_depth_first_wide_retry_dense_block():
    """A dense 17 x 17 block reached inside a depth-first job is a leaf of
    17 rows (s >= 5): the narrow kernel hands the job to the wide one."""
    sp = W.regular3(20, 3)
    n = 37
    a = np.zeros((n, n), np.int64)
    a[:20, :20] = sp
    a[20:, 20:] = 1
    with pk.Plan([a], split_depth=2, leaf_size=12) as plan:
        plan.expand()
        rec = plan.evaluate(records=True)
        got = plan.result(0)
    assert got == oracle.permanent(sp) * math.factorial(17)
    assert all(r.status == 0 for r in rec)


@pytest.mark.parametrize("rows,cols", [([0], []), ([7], [3]), ([2, 9], [5])])
def test_depth_first_big_entries_exact_or_overflow(rows, cols):
    """Rows and columns scaled by s = 2^29 + 7 scale the permanent by s per
    line (multilinearity).  Merged entries outgrow int32 (the narrow kernel
    hands the job on) and may outgrow the leaf's range: the result is then
    PERM_EOVERFLOW -- never a wrong value."""
    base = W.regular3(30, 5)
    s = (1 << 29) + 7
    a = base.copy()
    for r in rows:
        a[r] *= s
    for c in cols:
        a[:, c] *= s
    want = oracle.permanent(base) * s ** (len(rows) + len(cols))
    try:
        with pk.Plan([a], split_depth=4, leaf_size=10) as plan:
            plan.expand()
            plan.evaluate()
            got = plan.result(0)
        assert got == want
    except pk.PermError as e:
        assert e.status == 2


def test_c60_both_constructions():
    from conftest import read_adjacency
    mats = [W.c60(seed=3), read_adjacency("c60_adjacency.txt")]
    want = oracle.permanent(mats[0], d=12)
    for order in ("natural", "lpt"):
        with pk.Plan(mats, leaf_size=12, order=order) as plan:
            plan.expand()
            plan.evaluate()
            assert plan.results() == [want, want]


def test_packed_plan_matches_list_plan():
    """Plan.packed (one buffer, matrices back to back) gives the same plan as
    the list form: same results, equal to the oracle on sampled matrices;
    orders 0 and 1 included."""
    mats = (W.leaf_batch(300, seed=99, nmin=4, nmax=14) + [np.zeros((0, 0), dtype=np.int64), np.array([[5]])]
            + [W.regular3(20, 3)])
    data = np.concatenate([np.asarray(m, dtype=np.int64).ravel() for m in mats])
    orders = [m.shape[0] for m in mats]
    with pk.Plan(mats, order="natural") as a, pk.Plan.packed(data, orders, order="natural") as b:
        assert a.expand() == b.expand()
        a.evaluate()
        b.evaluate()
        ra, rb = a.results(), b.results()
    assert ra == rb
    for i in (0, 1, 150, 299, 300, 301, 302):
        assert rb[i] == oracle.permanent(mats[i]), i


def test_batch_of_matrices_one_launch():
    mats = [W.regular3(n, n) for n in (20, 24, 28, 30)] + [W.sparse_rows(22, 5)]
    with pk.Plan(mats, leaf_size=10) as plan:
        plan.expand()
        plan.order("lpt")
        plan.evaluate()
        got = plan.results()
    assert got == [oracle.permanent(m) for m in mats]


# ---------------------------------------------------------------- estimator (K4) and order
@pytest.mark.parametrize("n,d,trials", [(30, 14, 0), (20, 12, 0), (26, 14, 0), (28, 17, 40), (40, 16, 0),
                                         (46, 14, 100), (38, 20, 0), (80, 40, 60), (50, 8, 300), (70, 6, 40),
                                         (80, 0, 12), (96, 10, 6)])
def test_kklll_matches_oracle(n, d, trials):
    """Thread kernels for job orders <= 8 and 12 (order 11 with 40 trials: a
    partial last chunk of 32), the several-rows-per-lane register kernel up
    to 16, the tiled kernels for 24, 32, 40, 48 and 64 (parts of 32 trials,
    the last one partial), the shared-memory kernel above 64 (two pattern
    words per row); relative 1e-5 on the mean (FP32 against fp64)."""
    a = W.regular3(n, 4)
    with pk.Plan([a], split_depth=d, leaf_size=4, kklll_trials=trials, seed=1234) as plan:
        plan.expand()
        la = plan.estimate()
        jobs = plan.jobs_export()
    rng = np.random.default_rng(0)
    for j in rng.choice(len(jobs), size=min(8, len(jobs)), replace=False):
        want = oracle.kklll_log_ap(jobs[j][1], seed=1234, job=int(j), trials=trials or None)
        assert abs(float(la[j]) - want) < 1e-5, (j, la[j], want)


def test_kklll_dense_job_matches_oracle():
    """A job with more nonzeros than the tiled kernel's nonzero list (700 >
    512) fills its trial matrices row by row from the CSR block."""
    a = W.random01(36, 700, 11)
    with pk.Plan([a], split_depth=0, leaf_size=4, kklll_trials=40, seed=77) as plan:
        plan.expand()
        la = plan.estimate()
        jobs = plan.jobs_export()
    assert len(jobs) == 1 and int(np.count_nonzero(jobs[0][1])) == 700
    want = oracle.kklll_log_ap(jobs[0][1], seed=77, job=0, trials=40)
    assert abs(float(la[0]) - want) < 1e-5, (la[0], want)


def test_lpt_order_is_stable_sort_of_estimate():
    a = W.regular3(32, 9)
    with pk.Plan([a], split_depth=12, leaf_size=8) as plan:
        plan.expand()
        la = plan.estimate()
        q = plan.order("lpt")
    want = sorted(range(len(la)), key=lambda i: (-float(la[i]), i))
    assert list(q) == want


# ---------------------------------------------------------------- cost network (K5)
def test_mlp_gradient_matches_oracle():
    rng = np.random.default_rng(3)
    p = pk.mlp_init(3)
    x = rng.normal(size=(300, pk.MLP_FEATURES)).astype(np.float32)
    y = rng.normal(size=300).astype(np.float32)
    loss, g = pk.mlp_grad(p, x, y)
    wl, wg = omlp.loss_and_grad(p.astype(np.float64), x.astype(np.float64), y.astype(np.float64))
    assert abs(loss - wl) <= 1e-5 * max(1.0, abs(wl))
    assert np.allclose(g, wg, rtol=1e-3, atol=1e-5 * np.abs(wg).max())
    pred = pk.mlp_predict(p, x)
    assert np.allclose(pred, omlp.forward(p, x)[0], rtol=1e-4, atol=1e-5)


def test_mlp_training_reduces_loss():
    rng = np.random.default_rng(4)
    x = rng.normal(size=(2000, pk.MLP_FEATURES)).astype(np.float32)
    y = (x[:, 0] * 2 - x[:, 3] + 0.5 * x[:, 10]).astype(np.float32)
    p0 = pk.mlp_init(0)
    l0, _ = pk.mlp_grad(p0, x, y)
    p1, l1 = pk.mlp_train(p0, x, y, steps=300, lr=3e-3)
    assert l1 < 0.1 * l0
