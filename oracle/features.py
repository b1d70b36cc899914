"""ORACLE -- test infrastructure only.  The job features of the learned cost
model, in fp64, written from their definition.

The cost model is not in the paper (it is an addition to the ordering step
of Section 3.3: jobs are queued by non-increasing predicted time instead of
the KKLLL estimate).  Its inputs are twelve numbers per job of order m with
nnz nonzeros:

    f[0]      m / 64
    f[1]      nnz / m^2
    f[2..9]   the fraction of the m rows holding 1, 2, 3, 4, 5-6, 7-9,
              10-14 and >= 15 nonzeros (a row without nonzeros, which a job
              never has, counts with the rows holding one)
    f[10]     log AP / 64, AP the KKLLL approximate permanent of the job
              (Section 2.3); -1 when log AP is not finite (every trial
              singular); 0 when the model is used without the estimate
    f[11]     log2(m * 2^(m-1)) / 64 = (log2 m + m - 1) / 64, the size of
              the job's Ryser / Nijenhuis-Wilf evaluation (Section 1)

A job of order 0 has all twelve features 0.
"""
from __future__ import annotations

import math

import numpy as np

NFEAT = 12
# upper ends of the row-count bins 1, 2, 3, 4, 5-6, 7-9, 10-14, >= 15
BIN_TOP = (1, 2, 3, 4, 6, 9, 14)


def row_bin(k: int) -> int:
    """Histogram bin of a row holding k nonzeros (k = 0 joins the first)."""
    for b, top in enumerate(BIN_TOP):
        if k <= top:
            return b
    return len(BIN_TOP)


def job_features(a, log_ap: float | None = None) -> np.ndarray:
    """The twelve features of one job matrix ``a``; ``log_ap`` is its log
    KKLLL estimate, or None when the model does not use the estimate."""
    a = np.asarray(a)
    m = int(a.shape[0])
    f = np.zeros(NFEAT, dtype=np.float64)
    if m == 0:
        return f
    nz = a != 0
    nnz = int(nz.sum())
    f[0] = m / 64.0
    f[1] = nnz / float(m * m)
    for k in nz.sum(axis=1):
        f[2 + row_bin(int(k))] += 1.0 / m
    if log_ap is None:
        f[10] = 0.0
    elif math.isfinite(log_ap):
        f[10] = log_ap / 64.0
    else:
        f[10] = -1.0
    f[11] = (math.log2(m) + (m - 1)) / 64.0
    return f


def features(mats, log_aps=None) -> np.ndarray:
    """Features of a list of jobs (rows in the list's order)."""
    if log_aps is None:
        log_aps = [None] * len(mats)
    return np.array([job_features(m, la) for m, la in zip(mats, log_aps)], dtype=np.float64).reshape(-1, NFEAT)
