"""Full-size workloads on the GPU, checked against the oracle where it can
follow: the oracle evaluates sampled jobs one by one (each job's
coef * per(job) must match bit for bit), the job values must add up to the
reported permanent, and 3-regular permanents must lie within Schrijver's
and Bregman's bounds.  Small members of the mixed batch are checked whole."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

pk = pytest.importorskip("paper_1112_6072_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def signed_low(v, bits):
    v &= (1 << bits) - 1
    return v - (1 << bits) if v >> (bits - 1) else v


def _sampled_job_check(a, plan_kw, samples, seed):
    with pk.Plan([a], **plan_kw) as p:
        nj = p.expand()
        rec = p.evaluate(records=True)
        per = p.result(0)
        bits = p.result_bits(0)
        rng = np.random.default_rng(seed)
        pick = [int(j) for j in rng.choice(nj, size=min(samples, nj), replace=False)]
        jobs = p.jobs_select(pick)
    assert all(r.status == 0 for r in rec)
    vals = [signed_low(r.value_mod, bits) for r in rec]
    assert sum(vals) == per
    want = oracle.job_permanents([m for _, m, _ in jobs])
    for j, (_, m, c), w in zip(pick, jobs, want):
        assert vals[j] == signed_low(c, bits) * w, j
    return per, nj


def test_config4_orderings_agree():
    a = W.regular3(80, 2)
    vals = set()
    for order in ("natural", "lpt"):
        with pk.Plan([a], leaf_size=12, order=order) as p:
            p.expand()
            p.evaluate()
            vals.add(p.result(0))
    assert len(vals) == 1


def test_mixed_batch_one_plan():
    """Config-5 shape at reduced sizes: 3-regular and 3-5-nonzero rows
    matrices of different orders in one plan and one set of launches."""
    mats = W.mixed_batch(seed=5, count3=6, countsp=6, n3=(24, 40), nsp=(20, 30))
    with pk.Plan(mats, leaf_size=12) as p:
        p.expand()
        p.order("lpt")
        p.evaluate()
        got = p.results()
    want = [oracle.permanent(m) for m in mats]
    assert got == want


def test_sparse_rows_sampled_jobs():
    a = W.sparse_rows(60, 5)
    per, nj = _sampled_job_check(a, {"leaf_size": 12}, samples=6, seed=3)
    assert per <= oracle.bregman_bound(a) * (1 + 1e-12)
