"""The evaluation in one persistent launch (perm_opts.single_launch):
results equal to the oracle and to the grouped evaluation on leaf-only,
depth-first, mixed, residue and wide-ring workloads; the launch count; the
queue order holding across leaf and depth-first jobs (Algorithm PH, Step 3
as list scheduling over one queue)."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

pk = pytest.importorskip("paper_1112_6072_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def run(mats, order="natural", single=True, records=False, **kw):
    with pk.Plan(mats, single_launch=single, **kw) as p:
        p.expand()
        q = p.order(order)
        rec = p.evaluate(order=q, records="array" if records else False)
        out = dict(res=p.results(), launches=p.last_launches, njobs=p.njobs, q=q, rec=rec,
                   bits=[p.result_bits(i) for i in range(len(mats))])
        if records:
            p.replay()
            out["replay"] = p.results()
    return out


CASES = {
    # leaf jobs only, one variant
    "c60_L11": ([W.c60(60)], dict(leaf_size=11)),
    # big leaf jobs: many Gray-code tasks each, shared through the board
    "leaf_batch_21": ([W.leaf_batch(1, s, nmin=18, nmax=21)[0] for s in range(8)], dict()),
    # leaf jobs of several variants and depth-first jobs of order <= 32 in one queue
    "mixed_orders": ([W.regular3(n, n) for n in (24, 30, 36)] + [W.sparse_rows(28, 5)], dict(split_depth=3, leaf_size=10)),
    # depth-first jobs only (orders 26..34: tile 32 in the launch, tile 64 before it)
    "dfs_only": ([W.regular3(36, 2), W.regular3(34, 3)], dict(split_depth=2, leaf_size=12)),
    # the three-child split in the depth-first walk
    "dense_split": ([W.sparse_rows(26, 3, kmin=4, kmax=6)], dict(split_depth=3, leaf_size=8, dense_split=True)),
    # dense jobs of order 20 above the leaf order: the narrow tile hands them to the wide kernel
    "retry_wide": ([(np.random.default_rng(8).random((20, 20)) < 0.5).astype(np.int64),
                    W.regular3(30, 4)], dict(split_depth=1, leaf_size=12)),
}


_WANT = {}


def oracle_values(case):
    if case not in _WANT:
        _WANT[case] = [oracle.permanent(m, d=8) if m.shape[0] > 24 else oracle.permanent(m) for m in CASES[case][0]]
    return _WANT[case]


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("order", ["natural", "lpt"])
def test_single_launch_matches_grouped_and_oracle(case, order):
    mats, kw = CASES[case]
    one = run(mats, order, True, records=True, **kw)
    grp = run(mats, order, False, **kw)
    assert one["res"] == grp["res"]
    assert one["replay"] == one["res"]
    assert one["res"] == oracle_values(case)
    rec = one["rec"]
    assert (rec["status"] == 0).all() and (rec["queue_pos"] >= 0).all()
    # the persistent launch, the status summary, and the tile-64 launch when a job is above
    # order 32; jobs the narrow tile hands on add their wide rerun and a second summary
    assert one["launches"] <= (3 if case != "retry_wide" else 5)


def test_single_launch_residues_and_wide_ring():
    rng = np.random.default_rng(4)
    dense = rng.integers(-900, 1000, size=(12, 12)).astype(np.int64)
    mats = [W.regular3(30, 1), dense]
    want = [oracle.permanent(mats[0]), oracle.ryser(dense)]
    for p in (65537, 2147483647):
        one = run(mats, "natural", True, modulus=p, split_depth=3, leaf_size=10)
        grp = run(mats, "natural", False, modulus=p, split_depth=3, leaf_size=10)
        assert one["res"] == grp["res"] == [v % p for v in want]
    # a 256-bit matrix next to a 128-bit one: the launch runs in the wider ring
    one = run(mats, "natural", True, split_depth=3, leaf_size=10)
    assert one["bits"][1] > one["bits"][0]
    assert one["res"] == want


def test_single_launch_overflow_status():
    """A leaf whose row sums leave the exact leaf's range reports
    PERM_EOVERFLOW in single-launch mode too."""
    a = np.full((6, 6), (1 << 29) + 7, dtype=np.int64)
    for single in (False, True):
        with pk.Plan([a], single_launch=single) as p:
            p.expand()
            with pytest.raises(pk.PermError) as e:
                p.evaluate()
            assert e.value.status == 2


def test_single_launch_follows_queue_order():
    """Warps take queue positions in order: jobs early in the queue start
    before jobs late in it, across leaf and depth-first jobs."""
    mats = [W.regular3(n, n) for n in (40, 44, 48)]
    one = run(mats, "lpt", True, records=True, split_depth=6, leaf_size=12)
    rec, q = one["rec"], one["q"]
    start = rec["t_start_ns"][q].astype(np.float64)
    k = max(len(q) // 10, 1)
    assert np.median(start[:k]) <= np.median(start[-k:])
    assert one["launches"] <= 3
