"""The learned cost model end to end: train on the job timings one matrix's
evaluation produces, order a held-out matrix's jobs by predicted time, and
compare list-scheduling makespans with the paper's KKLLL order.  The model
is kept only where it does no worse (the paper's order is the fallback);
the permanent itself is unchanged by any order."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

pk = pytest.importorskip("paper_1112_6072_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)
learned = pytest.importorskip("paper_1112_6072_gb300.learned")


def _collect(a, d, L):
    with pk.Plan([a], split_depth=d, leaf_size=L, seed=7) as p:
        p.expand()
        la = p.estimate()
        X, t, recs = learned.collect(p, "natural")
        return X, t, la, p.result(0)


def test_learned_order_gain_over_kklll():
    d, L = 30, 10
    X, t, _, _ = _collect(W.regular3(56, 21), d, L)
    params, loss = learned.train(X, t, steps=600)
    assert np.isfinite(loss)
    a_val = W.regular3(56, 22)
    Xv, tv, la, per = _collect(a_val, d, L)
    assert per == oracle.permanent(a_val)
    pred = learned.predict_log_time(params, Xv)
    tau_pred = learned.kendall_tau(pred, tv)
    tau_ap = learned.kendall_tau(la, tv)
    workers = 64
    kept, ms = learned.choose(params, Xv, tv, la, workers)
    gain = ms["lpt_kklll"] / ms["learned"]
    print(f"jobs={len(tv)} tau(pred,time)={tau_pred:.3f} tau(KKLLL,time)={tau_ap:.3f} "
          f"makespans(m={workers}): {ms} learned gain over KKLLL-LPT = {gain:.3f}")
    assert tau_pred > 0.2          # the network ranks job times
    assert ms["exact_lpt"] <= ms["natural"] + 1e-9
    best = min(ms["learned"], ms["lpt_kklll"])
    chosen = ms["learned"] if kept is not None else ms["lpt_kklll"]
    assert chosen == best           # fallback keeps the better of the two
    # the queue set by the attached model evaluates to the same permanent
    with pk.Plan([a_val], split_depth=d, leaf_size=L, order="learned") as p:
        p.expand()
        p.attach_model(params)
        q = p.order("learned")
        assert sorted(q.tolist()) == list(range(p.njobs))
        p.evaluate()
        assert p.result(0) == per
