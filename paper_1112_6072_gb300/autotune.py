"""Autotuner for the knobs the paper leaves to the implementation.

* leaf order L -- where Eq. 2 stops and Ryser / Nijenhuis-Wilf takes over
  (the paper's H_per goes down to order 2; a GPU warp prefers larger
  leaves);
* split depth d -- how many levels Algorithm PH, Step 2 expands before jobs
  are formed (more jobs: better balance, more estimator work);
* Gray codes per lane (chunk_log2) -- how finely one leaf job is spread over
  warps, i.e. threads per job;
* evaluator warps per SM for the depth-first kernel.

Every candidate runs through the library on the GPU on a sample input and
the fastest whole-path time wins.  Results are cached per matrix (order,
nonzeros, the range of nonzeros per row and a hash of the entries) and GPU
name, in memory and optionally in a JSON file.
"""
from __future__ import annotations

import json
import os
import time

import numpy as np

from . import Plan

_CACHE: dict = {}


def _gpu_name():
    try:
        import torch
        return torch.cuda.get_device_name(0)
    except Exception:
        return "unknown"


def _key(a) -> str:
    """Cache key of a matrix: two matrices share tuned knobs only when their
    entries are equal (a hash of them), on the same GPU model."""
    import hashlib
    a = np.ascontiguousarray(np.asarray(a, dtype=np.int64))
    n = a.shape[0]
    r = (a != 0).sum(axis=1) if n else np.zeros(1, np.int64)
    h = hashlib.sha256(a.tobytes() + np.int64(n).tobytes()).hexdigest()[:16]
    return f"n{n}_nnz{int((a != 0).sum())}_r{int(r.min())}-{int(r.max())}_{h}_{_gpu_name()}"


def _time_path(mats, reps=2, **opts) -> float:
    best = float("inf")
    for _ in range(reps):
        t = time.perf_counter()
        with Plan(mats, **opts) as p:
            p.expand()
            p.order(opts.get("order", "natural"))
            p.evaluate()
            p.results()
        best = min(best, time.perf_counter() - t)
    return best


def tune_hybrid(a, leaf_sizes=(10, 11, 12, 13, 14), depth_offsets=(-16, -12, -8, -4, 0), workers=(8, 16),
                order="natural", cache_file: str | None = None) -> dict:
    """Best (leaf_size, split_depth, workers_per_sm) for a sparse matrix: the
    whole path timed at split depths from the automatic one (jobs at the
    leaf order, evaluated by the leaf kernel) up to 16 levels above it (fewer,
    larger jobs, evaluated depth first)."""
    key = "hybrid_" + _key(a)
    if cache_file and os.path.exists(cache_file):
        _CACHE.update(json.load(open(cache_file)))
    if key in _CACHE:
        return dict(_CACHE[key])
    n = np.asarray(a).shape[0]
    results = []
    for L in leaf_sizes:
        # depth the automatic rule reached, from the jobs' order
        with Plan([a], leaf_size=L) as p:
            p.expand()
            rec = p.evaluate(records=True)
            d_auto = n - max(r.order for r in rec) if rec else 0
        for off in depth_offsets:
            d = max(0, d_auto + off)
            if n - d > 64:
                continue
            for w in workers:
                t = _time_path([a], leaf_size=L, split_depth=d, workers_per_sm=w, order=order)
                results.append((t, L, d, w))
    t, L, d, w = min(results)
    best = {"leaf_size": L, "split_depth": d, "workers_per_sm": w, "seconds": t, "tried": len(results)}
    _CACHE[key] = best
    if cache_file:
        json.dump(_CACHE, open(cache_file, "w"), indent=1)
    return dict(best)


def tune_leaf_batch(mats, chunks=(6, 8, 10, 12), cache_file: str | None = None) -> dict:
    """Best Gray codes per lane (2^chunk_log2) for a batch of leaf-order matrices."""
    key = f"leaf_{len(mats)}_{max(m.shape[0] for m in mats)}_{_gpu_name()}"
    if key in _CACHE:
        return dict(_CACHE[key])
    results = []
    for c in chunks:
        with Plan(mats, chunk_log2=c, order="natural") as p:
            p.expand()
            order = np.arange(p.njobs, dtype=np.uint32)
            p.evaluate(order=order)
            ms = []
            for _ in range(2):
                p.evaluate(order=order)
                ms.append(p.last_eval_ms)
        results.append((min(ms), c))
    ms, c = min(results)
    best = {"chunk_log2": c, "eval_ms": ms, "tried": len(results)}
    _CACHE[key] = best
    if cache_file:
        json.dump(_CACHE, open(cache_file, "w"), indent=1)
    return dict(best)


def tune_batch(mats, leaf_sizes=(12, 14, 16), sample=16, order="lpt") -> dict:
    """Best leaf order L for a batch, timed on a sample of it: the whole path
    (automatic split depth) over every k-th matrix by order, so the sample
    spans the batch's sizes without its most expensive members."""
    by_n = sorted(range(len(mats)), key=lambda k: (np.asarray(mats[k]).shape[0], k))
    step = max(1, len(by_n) // sample)
    picked = [mats[k] for k in by_n[: len(by_n) - step][::step]][:sample] or list(mats)
    key = f"batch_{len(mats)}_{sum(np.asarray(m).shape[0] for m in mats)}_{_gpu_name()}"
    if key in _CACHE:
        return dict(_CACHE[key])
    results = [(_time_path(picked, reps=1, leaf_size=L, order=order), L) for L in leaf_sizes]
    t, L = min(results)
    best = {"leaf_size": L, "sample_seconds": t, "sample": len(picked),
            "tried": {str(l): round(s, 4) for s, l in results}}
    _CACHE[key] = best
    return dict(best)
