"""The Kendall study pipeline on a small group: exact permanents of the
group against the oracle, estimates per matrix, and tau-b of the measured
times computed by the study module."""
import numpy as np
import pytest

import oracle
import workloads as W
from paper_1112_6072_gb300 import kendall

pk = pytest.importorskip("paper_1112_6072_gb300")

pytestmark = pytest.mark.gpu


def test_random01_group_study():
    mats = [W.random01(14, 42, 300 + i) for i in range(12)]
    times, pers = [], []
    for a in mats:
        with pk.Plan([a], leaf_size=6, order="natural") as p:
            p.expand()
            rec = p.evaluate(records="array")
            pers.append(p.result(0))
            times.append(int((rec["t_end_ns"].max() - rec["t_start_ns"].min())) if len(rec) else 0)
    assert pers == [oracle.permanent(a) for a in mats]
    with pk.Plan(mats, split_depth=0, leaf_size=6, seed=99) as p:
        assert p.expand() == len(mats)
        ap = p.estimate()
    for k in (0, 5, 11):
        assert abs(float(ap[k]) - oracle.kklll_log_ap(mats[k], seed=99, job=k)) < 1e-5
    row = kendall.table(times, per=pers, ap=ap.tolist())
    assert row["n"] == 12
    assert abs(row["per"]["tau"] - oracle.kendall_tau_b(times, pers)) < 1e-12


def test_job_permanents_from_records():
    """per(job) recovered from the records' coef * per(job) equals the
    oracle's per of each exported job."""
    a = W.regular3(24, 3)
    with pk.Plan([a], split_depth=8, leaf_size=6) as p:
        p.expand()
        jobs = p.jobs_export()
        _, coefs, _ = p.job_coefs()
        rec = p.evaluate(records="array")
        bits = p.result_bits(0)
    vals = kendall.words_to_ints(rec["value"])
    got = kendall.exact_job_permanents(vals, coefs, bits)
    assert got == [oracle.permanent(m) for _, m, _ in jobs]
