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
        p.expand()
        rec = p.evaluate(records=True)
        per = p.result(0)
        bits = p.result_bits(0)
        jobs = p.jobs_export()
    assert all(r.status == 0 for r in rec)
    vals = [signed_low(r.value_mod, bits) for r in rec]
    assert sum(vals) == per
    rng = np.random.default_rng(seed)
    pick = rng.choice(len(jobs), size=min(samples, len(jobs)), replace=False)
    want = oracle.job_permanents([jobs[j][1] for j in pick])
    for j, w in zip(pick, want):
        assert vals[j] == signed_low(jobs[j][2], bits) * w, j
    return per, len(jobs)


@pytest.mark.parametrize("n", [80, 96])
def test_config4_regular(n):
    a = W.regular3(n, 1)
    per, nj = _sampled_job_check(a, {"leaf_size": 12}, samples=6, seed=n)
    assert nj > 10_000
    assert oracle.schrijver_lower_bound(n, 3) <= per <= 6 ** (n / 3)
    assert per <= oracle.bregman_bound(a) * (1 + 1e-12)


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
