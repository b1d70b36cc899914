"""The allocation-free leaf batch, for callers that cannot allocate device
memory while they run (a host framework whose allocator owns every device
allocation, or a loop that may not allocate after start-up): it must return
the oracle's permanents, and the same as the planning entry point, call
after call, using only the buffers the caller passes in.

This file is named so that pytest collects it last."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

pk = pytest.importorskip("paper_1112_6072_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def words_to_ints(words):
    out = []
    for row in words.reshape(-1, 4):
        v = 0
        for k in range(3, -1, -1):
            v = (v << 64) | int(row[k])
        out.append(v - (1 << 256) if v >> 255 else v)
    return out


def planned_results(mats):
    with pk.Plan(mats) as plan:
        plan.expand()
        plan.evaluate(order=np.arange(plan.njobs, dtype=np.uint32))
        return plan.results()


def run_noalloc(mats, n, calls=2):
    """Results and statuses of `calls` calls in a row on the same buffers."""
    dev = torch.device("cuda", 0)
    count = len(mats)
    a = torch.from_numpy(np.stack(mats).astype(np.int64).reshape(count, n, n)).to(dev)
    stream = torch.cuda.current_stream()
    outs = []
    for _ in range(calls):
        out = torch.full((count, 4), -1, dtype=torch.int64, device=dev)
        status = torch.full((count,), -1, dtype=torch.int32, device=dev)
        pk.leaf_batch_noalloc(a.data_ptr(), n, count, out.data_ptr(), status.data_ptr(), stream)
        torch.cuda.synchronize()
        outs.append((words_to_ints(out.cpu().numpy().view(np.uint64)), status.cpu().numpy()))
    return outs


@pytest.mark.parametrize("n,count,kind", [(14, 96, "leaf"), (20, 12, "leaf"), (9, 200, "signed"),
                                          (1, 50, "signed"), (24, 1, "leaf"), (30, 2, "ones")])
def test_noalloc_matches_oracle_and_planned_path_twice(n, count, kind):
    """Orders 1 (no Gray walk), 9, 14 and 20, 24 (the 24-row register
    width) and 30 (the 32-row width, every entry 1: per = 30!)."""
    if kind == "signed":
        mats = [W.random_small(n, 7000 + k, lo=-3, hi=3) for k in range(count)]
    elif kind == "ones":
        mats = [np.ones((n, n), dtype=np.int64) for _ in range(count)]
    else:
        mats = W.leaf_batch(count, seed=4242 + n, nmin=n, nmax=n)
    if kind == "ones":
        import math
        want = [math.factorial(n)] * count
    elif n <= 20:
        want = oracle.job_permanents(mats)
    else:
        want = [oracle.permanent(m) for m in mats]
    assert planned_results(mats) == want
    for call, (got, status) in enumerate(run_noalloc(mats, n)):
        assert (status == 0).all(), call
        assert got == want, call


def test_noalloc_rejects_sizes_beyond_the_limit():
    dev = torch.device("cuda", 0)
    a = torch.zeros((1, 4, 4), dtype=torch.int64, device=dev)
    out = torch.zeros((1, 4), dtype=torch.int64, device=dev)
    st = torch.zeros((1,), dtype=torch.int32, device=dev)
    with pytest.raises(pk.PermError):
        pk.leaf_batch_noalloc(a.data_ptr(), 4, 5000, out.data_ptr(), st.data_ptr())
    with pytest.raises(pk.PermError):
        pk.leaf_batch_noalloc(a.data_ptr(), 40, 1, out.data_ptr(), st.data_ptr())
    with pytest.raises(pk.PermError):
        pk.leaf_batch_noalloc(a.data_ptr(), 0, 1, out.data_ptr(), st.data_ptr())


def test_noalloc_flags_out_of_range_entries_and_bounds():
    """Matrix 1 has an entry of 2^31 (out of range); matrix 2 has every
    entry 2^27 -- each row's sum of |a_ij| (10 * 2^27) is in range, but the
    bound (10 * 2^27)^10 ~ 2^303 exceeds 2^(254 - 10): PERM_EOVERFLOW with the
    output cleared, never a wrong value.  Matrix 0 is per(J_10) = 10!."""
    n = 10
    m = np.ones((3, n, n), dtype=np.int64)
    m[1, 2, 3] = 1 << 31
    m[2] = 1 << 27
    got, status = run_noalloc(list(m), n, calls=1)[0]
    assert status.tolist() == [0, 2, 2]
    assert got == [3628800, 0, 0]
