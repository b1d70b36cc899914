"""The allocation-free leaf batch, for callers that cannot allocate device
memory while they run (for instance while recording a CUDA graph): it must
return the same permanents as the planning entry point, call after call,
using only the buffers the caller passes in.

This file is named so that pytest collects it last."""
import numpy as np
import pytest

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


def reference_results(mats):
    with pk.Plan(mats) as plan:
        plan.expand()
        plan.evaluate(order=np.arange(plan.njobs, dtype=np.uint32))
        return plan.results()


@pytest.mark.parametrize("n,count,signed", [(14, 96, False), (20, 12, False), (9, 200, True)])
def test_noalloc_matches_planned_path_twice(n, count, signed):
    if signed:
        mats = [W.random_small(n, 7000 + k, lo=-3, hi=3) for k in range(count)]
    else:
        mats = W.leaf_batch(count, seed=4242 + n, nmin=n, nmax=n)
    want = reference_results(mats)
    dev = torch.device("cuda", 0)
    a = torch.from_numpy(np.stack(mats).astype(np.int64)).to(dev)
    stream = torch.cuda.current_stream()
    for call in range(2):
        out = torch.full((count, 4), -1, dtype=torch.int64, device=dev)
        status = torch.full((count,), -1, dtype=torch.int32, device=dev)
        pk.leaf_batch_noalloc(a.data_ptr(), n, count, out.data_ptr(), status.data_ptr(), stream)
        torch.cuda.synchronize()
        assert (status.cpu().numpy() == 0).all(), call
        got = words_to_ints(out.cpu().numpy().view(np.uint64))
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


def test_noalloc_flags_out_of_range_entries():
    dev = torch.device("cuda", 0)
    m = np.ones((2, 6, 6), dtype=np.int64)
    m[1, 2, 3] = 1 << 31
    a = torch.from_numpy(m).to(dev)
    out = torch.zeros((2, 4), dtype=torch.int64, device=dev)
    st = torch.zeros((2,), dtype=torch.int32, device=dev)
    pk.leaf_batch_noalloc(a.data_ptr(), 6, 2, out.data_ptr(), st.data_ptr())
    torch.cuda.synchronize()
    s = st.cpu().numpy()
    assert s[0] == 0 and s[1] == 2
    assert words_to_ints(out.cpu().numpy().view(np.uint64))[0] == 720
