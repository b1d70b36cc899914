"""What the trained cost model gains over the method without it.

The network is trained, on the GPU by the library's own forward, backward
and Adam kernels, on job timings that the method logs in configurations
1-3 only: the n = 36 3-regular matrix and C60 split at several depths
(jobs of order 20-40), and matrices of the leaf batch.  It does not use the
KKLLL feature, so ordering by it costs one feature pass and one forward
pass.  On a held-out configuration-4 matrix (random 3-regular n = 80, split
to depth 40: 11,841 jobs of order 40 -- few jobs per warp, where the order
matters) the test compares device makespans: the learned order (plus its
ordering time) against natural order, and against the paper's KKLLL-LPT
order plus the estimator's time.  Every order gives the same permanent."""
import time

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

pk = pytest.importorskip("paper_1112_6072_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)
learned = pytest.importorskip("paper_1112_6072_gb300.learned")


def _timings(mats, **kw):
    with pk.Plan(mats, model_uses_estimate=False, **kw) as p:
        p.expand()
        X, t, _ = learned.collect(p, "natural")
    return X, t


def train_on_configs_1_to_3():
    Xs, ts = [], []
    for d in (4, 8, 12, 16, 20):                       # configuration 1: n = 36, leaf order 14
        X, t = _timings([W.regular3(36, 1)], split_depth=d, leaf_size=14)
        Xs.append(X)
        ts.append(t)
    for d in (20, 24, 28):                             # configuration 3: C60 (another vertex shuffle)
        X, t = _timings([W.c60(seed=61)], split_depth=d, leaf_size=14)
        Xs.append(X)
        ts.append(t)
    X, t = _timings(W.leaf_batch(1500, seed=777))      # configuration 2: leaf-batch matrices
    Xs.append(X)
    ts.append(t)
    return learned.train(np.concatenate(Xs), np.concatenate(ts), steps=800)


def _makespan(a, order, params=None, reps=2):
    with pk.Plan([a], split_depth=40, leaf_size=14, order=order, model_uses_estimate=False) as p:
        p.expand()
        if params is not None:
            p.attach_model(params)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        p.order(order)
        torch.cuda.synchronize()
        order_ms = (time.perf_counter() - t0) * 1e3
        p.evaluate()
        evs = [p.last_eval_ms]
        for _ in range(reps - 1):
            p.replay()
            evs.append(p.last_eval_ms)
        return min(evs), order_ms, p.result(0), p.njobs


def test_learned_order_gain_on_held_out_configuration_4():
    params, loss = train_on_configs_1_to_3()
    assert np.isfinite(loss)
    a = W.regular3(80, 1)
    nat, nat_o, per_n, nj = _makespan(a, "natural")
    lpt, lpt_o, per_l, _ = _makespan(a, "lpt")
    lrn, lrn_o, per_m, _ = _makespan(a, "learned", params)
    print(f"jobs={nj} loss={loss:.4f} natural {nat:.1f} ms; KKLLL-LPT {lpt:.1f} + {lpt_o:.1f} ms; "
          f"learned {lrn:.1f} + {lrn_o:.2f} ms")
    assert per_n == per_l == per_m
    assert nj == 11841
    # the learned order, ordering included, beats the paper's order with its estimator ...
    assert lrn + lrn_o < lpt + lpt_o
    # ... and the unordered queue
    assert lrn + lrn_o < nat
