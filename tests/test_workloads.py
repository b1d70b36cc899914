"""The seeded input generators follow their stated recipes (CPU only)."""
import numpy as np
import pytest

import workloads as W


def _is_simple_cubic(a):
    return (a.dtype == np.int64 and np.array_equal(a, a.T) and not a.diagonal().any()
            and set(np.unique(a)) <= {0, 1} and (a.sum(axis=1) == 3).all())


@pytest.mark.parametrize("n,seed", [(4, 1), (36, 1), (80, 1), (96, 1), (60, 9)])
def test_regular3_is_a_simple_cubic_graph(n, seed):
    a = W.regular3(n, seed)
    assert a.shape == (n, n) and _is_simple_cubic(a)
    assert np.array_equal(a, W.regular3(n, seed))           # seeded
    if n > 4:
        assert not np.array_equal(a, W.regular3(n, seed + 1))


def test_regular3_rejects_impossible_orders():
    for n in (3, 5, 7):
        with pytest.raises(ValueError):
            W.regular3(n, 1)


def test_c60_is_the_truncated_icosahedron_graph():
    """60 vertices of degree 3 and 90 edges, all at the minimum distance; no
    triangles and exactly 12 pentagons: with girth 5 every closed walk of
    length 5 runs around a 5-cycle (5 starting points, 2 directions), so
    trace(A^5) = 10 * 12."""
    a = W.c60()
    assert a.shape == (60, 60) and _is_simple_cubic(a) and int(a.sum()) == 180
    p = W.c60_coordinates()
    d = np.linalg.norm(p[:, None] - p[None], axis=2)
    assert np.allclose(d[a == 1], d[a == 1].min())
    a3 = np.linalg.matrix_power(a, 3)
    assert np.trace(a3) == 0
    assert np.trace(a3 @ a @ a) == 120
    s = W.c60(seed=60)
    perm = np.random.default_rng(60).permutation(60)
    assert _is_simple_cubic(s) and not np.array_equal(s, a)
    assert np.array_equal(s, a[np.ix_(perm, perm)])  # one vertex permutation on rows and columns


def test_leaf_batch_recipe():
    mats = W.leaf_batch(3000, seed=20240601)
    sizes = np.array([m.shape[0] for m in mats])
    assert sizes.min() == 12 and sizes.max() == 24
    counts = np.bincount(sizes, minlength=25)[12:]
    assert counts.min() > 3000 / 13 * 0.7                    # uniform over the 13 orders
    vals = np.concatenate([m.ravel() for m in mats])
    assert set(np.unique(vals)) == {0, 1, 2, 3}
    p = float((vals != 0).mean())
    assert abs(p - 0.35) < 0.01
    nzv = vals[vals != 0]
    assert all(abs(float((nzv == v).mean()) - 1 / 3) < 0.02 for v in (1, 2, 3))
    # seeded: the same count and seed give the same batch (the sizes are drawn
    # first, so a shorter batch is not a prefix of a longer one)
    x, y = W.leaf_batch(50, seed=7), W.leaf_batch(50, seed=7)
    assert all(np.array_equal(u, v) for u, v in zip(x, y))


@pytest.mark.parametrize("n,seed", [(40, 1), (55, 2), (70, 3)])
def test_sparse_rows_recipe(n, seed):
    a = W.sparse_rows(n, seed)
    r = a.sum(axis=1)
    assert set(np.unique(a)) <= {0, 1} and r.min() >= 3 and r.max() <= 5
    assert (a.sum(axis=0) > 0).all()


def test_mixed_batch_composition():
    mats = W.mixed_batch(seed=5, count3=16, countsp=16)
    assert len(mats) == 32
    for a in mats[:16]:
        n = a.shape[0]
        assert 40 <= n <= 90 and n % 2 == 0 and _is_simple_cubic(a)
    for a in mats[16:]:
        n = a.shape[0]
        r = a.sum(axis=1)
        assert 40 <= n <= 70 and r.min() >= 3 and r.max() <= 5 and (a.sum(axis=0) > 0).all()


def test_random01_exact_count_and_no_empty_line():
    a = W.random01(60, 240, 3)
    assert int(a.sum()) == 240 and set(np.unique(a)) == {0, 1}
    assert (a.sum(axis=0) > 0).all() and (a.sum(axis=1) > 0).all()


def test_autotune_cache_key_tells_matrices_apart():
    """The tuner's cache key: equal matrices share it, a different pattern
    with the same order and row counts does not."""
    from paper_1112_6072_gb300 import autotune
    a = W.regular3(36, 1)
    b = W.regular3(36, 2)  # same order, every row with 3 nonzeros
    assert autotune._key(a) == autotune._key(a.copy())
    assert autotune._key(a) != autotune._key(b)
    assert autotune._key(a) != autotune._key(2 * a)
