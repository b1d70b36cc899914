"""Kendall tau-b of the study module (Eq. 10, O(n log n)) against the
oracle's pair-by-pair statement and against brute force on small inputs."""
import math

import numpy as np
import pytest

import oracle
from paper_1112_6072_gb300 import kendall


@pytest.mark.parametrize("seed", range(6))
def test_tau_b_matches_oracle_with_ties(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 120))
    x = rng.integers(0, 6, size=n).tolist()
    y = (np.array(x) * rng.integers(-1, 2) + rng.integers(0, 5, size=n)).tolist()
    assert abs(kendall.tau_b(x, y) - oracle.kendall_tau_b(x, y)) < 1e-12


def test_tau_b_extremes_and_big_ints():
    assert kendall.tau_b([1, 2, 3, 4], [10, 20, 30, 40]) == 1.0
    assert kendall.tau_b([1, 2, 3, 4], [4, 3, 2, 1]) == -1.0
    big = [10**30 + k for k in range(50)]
    assert kendall.tau_b(big, list(range(50))) == 1.0
    assert kendall.tau_b([1, 1, 1], [1, 2, 3]) == 0.0


def test_inversions_brute_force():
    rng = np.random.default_rng(3)
    for _ in range(20):
        a = rng.integers(0, 10, size=int(rng.integers(0, 40))).tolist()
        want = sum(1 for i in range(len(a)) for j in range(i + 1, len(a)) if a[i] > a[j])
        assert kendall._inversions(a) == want


def test_p_value_normal_limit():
    # z = 1.96 gives p = 0.05
    n = 100
    sd = math.sqrt(2 * (2 * n + 5) / (9 * n * (n - 1)))
    assert abs(kendall.p_value(1.959963985 * sd, n) - 0.05) < 1e-6
    assert kendall.p_value(0.0, n) == 1.0


def test_exact_job_permanents():
    bits = 120
    coefs = [3, (1 << 256) - 2, 1]          # 3, -2, 1
    pers = [7, 11, -(1 << 100)]
    vals = [(c if c < (1 << 255) else c - (1 << 256)) * p % (1 << 256) for c, p in zip(coefs, pers)]
    assert kendall.exact_job_permanents(vals, coefs, bits) == pers
