"""Learned job-cost model around the library's own kernels.

The method itself generates the training data: every evaluation logs each
job's device start and end time.  The network (12 -> 64 -> 64 -> 1, ReLU,
FP32) learns log(job time) from the job's features on the GPU
(``perm_mlp_train``); its predictions re-order the queue
(``PERM_ORDER_LEARNED``, an LPT order on predicted times, Section 2.4).
The paper's own order -- non-increasing KKLLL estimate (Section 3.3) --
stays the fallback: a model is kept only if its list-scheduling makespan on
held-out jobs is no worse than the estimate's.
"""
from __future__ import annotations

import heapq

import numpy as np

from . import Plan, mlp_init, mlp_predict, mlp_train


def job_times_ns(records) -> np.ndarray:
    """Device time of each job: last worker's end minus first worker's start."""
    return np.array([max(1, r.t_end_ns - r.t_start_ns) for r in records], dtype=np.float64)


def collect(plan: Plan, order="natural"):
    """Features (njobs x 12), job times (ns) and records of one evaluation."""
    feats = plan.features()
    q = plan.order(order)
    recs = plan.evaluate(order=q, records=True)
    return feats, job_times_ns(recs), recs


def train(feats, times_ns, steps=800, lr=3e-3, seed=0):
    """Fit log(time) on the GPU with the library's forward/backward/Adam kernels."""
    y = np.log(np.asarray(times_ns, dtype=np.float64)).astype(np.float32)
    p0 = mlp_init(seed)
    # start the output bias at the mean target so Adam fits the spread
    p0[-1] = float(y.mean())
    params, loss = mlp_train(p0, feats, y, steps=steps, lr=lr)
    return params, loss


def predict_log_time(params, feats) -> np.ndarray:
    return mlp_predict(params, feats)


def list_makespan(times, order, workers: int) -> float:
    """Graham's list scheduling: jobs in `order`, each to the least-loaded
    of `workers` identical workers; returns the finishing time."""
    heap = [(0.0, k) for k in range(workers)]
    for j in order:
        load, k = heapq.heappop(heap)
        heapq.heappush(heap, (load + float(times[j]), k))
    return max(load for load, _ in heap)


def order_by(keys) -> np.ndarray:
    """Non-increasing key, equal keys in natural order."""
    keys = np.asarray(keys, dtype=np.float64)
    idx = np.arange(len(keys))
    return np.lexsort((idx, -keys))


def kendall_tau(x, y) -> float:
    from scipy.stats import kendalltau

    return float(kendalltau(x, y).statistic)


def compare_orders(times, log_ap, pred, workers: int):
    """Makespans of natural, KKLLL-LPT, learned and exact-time LPT orders."""
    n = len(times)
    out = {
        "natural": list_makespan(times, np.arange(n), workers),
        "lpt_kklll": list_makespan(times, order_by(log_ap), workers),
        "exact_lpt": list_makespan(times, order_by(times), workers),
        "lower_bound": max(float(np.sum(times)) / workers, float(np.max(times))),
    }
    if pred is not None:
        out["learned"] = list_makespan(times, order_by(pred), workers)
    return out


def choose(params, feats_val, times_val, log_ap_val, workers: int):
    """Keep the model only if it schedules held-out jobs no worse than the
    paper's KKLLL order; returns (params or None, makespans)."""
    pred = predict_log_time(params, feats_val)
    ms = compare_orders(times_val, log_ap_val, pred, workers)
    return (params if ms["learned"] <= ms["lpt_kklll"] else None), ms
