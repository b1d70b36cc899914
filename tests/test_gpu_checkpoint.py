"""Checkpoint and resume at job boundaries (checkpoint.py) on the GPU: a run
stopped after some chunks and resumed by a new process-like start (a new
plan of the same matrices, the snapshot read back) equals the single pass
and the oracle; another job list is refused; the residue path and
matrices without jobs."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

pk = pytest.importorskip("paper_1112_6072_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)
from paper_1112_6072_gb300 import checkpoint as C  # noqa: E402


def single_pass(mats, **kw):
    with pk.Plan(mats, **kw) as p:
        p.expand()
        p.evaluate()
        return p.results()


@pytest.mark.parametrize("order", ["natural", "lpt"])
def test_stop_and_resume_equals_single_pass(tmp_path, order):
    mats = [W.c60(60), W.regular3(36, 1), np.zeros((0, 0), np.int64), np.zeros((5, 5), np.int64)]
    kw = dict(leaf_size=12)
    path = str(tmp_path / "c60.snap")
    with pk.Plan(mats, **kw) as p:
        run = C.CheckpointedRun(p, path, chunks=5, order=order)
        assert run.run(stop_after=2) is None
    # a new start: a new plan of the same matrices, the snapshot read back
    with pk.Plan(mats, **kw) as p:
        run = C.CheckpointedRun(p, path)
        assert run.state["chunk"] == 2 and 0 < run.state["done"].sum() < p.njobs
        got = run.run()
    want = single_pass(mats, **kw)
    assert got == want
    assert got[:2] == [395974320, oracle.permanent(mats[1])] and got[2:] == [1, 0]


def test_resume_refuses_another_job_list(tmp_path):
    path = str(tmp_path / "snap")
    with pk.Plan([W.c60(60)], leaf_size=12) as p:
        C.CheckpointedRun(p, path, chunks=4).run(stop_after=1)
    with pk.Plan([W.c60(60)], leaf_size=11) as p:  # another split: another job list
        with pytest.raises(C.CheckpointError):
            C.CheckpointedRun(p, path)


def test_resume_on_the_residue_path(tmp_path):
    p_ = 2147483647
    a = W.regular3(40, 3)
    path = str(tmp_path / "snap")
    with pk.Plan([a], modulus=p_, split_depth=6, leaf_size=10) as p:
        C.CheckpointedRun(p, path, chunks=3).run(stop_after=1)
    with pk.Plan([a], modulus=p_, split_depth=6, leaf_size=10) as p:
        got = C.CheckpointedRun(p, path).run()
    assert got == [oracle.permanent(a, d=8) % p_]
