"""ORACLE -- test infrastructure only.  Scheduling arithmetic of Section 2.4
and the rank statistic of Section 3.2.

``list_schedule`` is Graham's list scheduling: jobs, taken in the given
order, each go to the machine that is currently least loaded (Algorithm PH,
Step 3).  Feeding the jobs in non-increasing processing time gives LPT.
"""
from __future__ import annotations

import heapq
import math


def list_schedule(times, m: int, order=None) -> float:
    """Makespan of list scheduling of ``times`` on ``m`` identical machines;
    the least-loaded machine takes the next job (lowest index on ties)."""
    if m < 1:
        raise ValueError("m >= 1")
    idx = range(len(times)) if order is None else order
    heap = [(0.0, k) for k in range(m)]
    heapq.heapify(heap)
    for j in idx:
        load, k = heapq.heappop(heap)
        heapq.heappush(heap, (load + float(times[j]), k))
    return max(load for load, _ in heap)


def lpt_order(keys):
    """Indices by non-increasing key; equal keys keep their natural order."""
    return sorted(range(len(keys)), key=lambda i: (-keys[i], i))


def efficiency(t1: float, tm: float, m: int) -> float:
    """Parallel efficiency T1 / (m * Tm), as in Tables T5-T17."""
    return t1 / (m * tm)


def kendall_tau_b(x, y) -> float:
    """Kendall's tau with ties (Eq. 10): S / sqrt((N0 - T)(N0 - U)),
    N0 = n(n-1)/2, T and U the tied pairs in x and in y (Eq. 8, 9)."""
    n = len(x)
    s = 0
    tx = ty = 0
    for i in range(n):
        for j in range(i + 1, n):
            a = (x[j] > x[i]) - (x[j] < x[i])
            b = (y[j] > y[i]) - (y[j] < y[i])
            s += a * b
            tx += a == 0
            ty += b == 0
    n0 = n * (n - 1) / 2
    den = math.sqrt((n0 - tx) * (n0 - ty))
    return s / den if den > 0 else 0.0
