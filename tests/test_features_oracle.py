"""Pins of the job-feature oracle (oracle/features.py): rows computed by
hand for small matrices, the bin edges, and the estimate feature's
special cases."""
import math

import numpy as np
import pytest

from oracle import features as F


def test_identity_3x3_by_hand():
    f = F.job_features(np.eye(3, dtype=np.int64), log_ap=0.0)
    want = np.zeros(12)
    want[0] = 3 / 64           # order
    want[1] = 3 / 9            # nnz / m^2
    want[2] = 1.0              # every row holds one nonzero
    want[10] = 0.0             # log AP = log 1
    want[11] = (math.log2(3) + 2) / 64   # log2(3 * 2^2) / 64
    assert np.array_equal(f, want)


def test_5x5_mixed_rows_by_hand():
    a = np.array([[1, 0, 0, 0, 0],      # 1 nonzero
                  [2, -1, 0, 0, 0],     # 2
                  [1, 1, 1, 0, 0],      # 3
                  [1, 1, 1, 1, 1],      # 5 -> bin "5-6"
                  [0, 0, 3, 0, 7]])     # 2
    f = F.job_features(a, log_ap=math.log(12.0))
    assert f[0] == 5 / 64
    assert f[1] == 13 / 25
    assert np.array_equal(f[2:10], np.array([1, 2, 1, 0, 1, 0, 0, 0]) / 5)
    assert f[10] == math.log(12.0) / 64
    assert f[11] == (math.log2(5) + 4) / 64
    assert abs(f[2:10].sum() - 1.0) < 1e-15


def test_bins_edges():
    assert [F.row_bin(k) for k in range(0, 20)] == [0, 0, 1, 2, 3, 4, 4, 5, 5, 5, 6, 6, 6, 6, 6, 7, 7, 7, 7, 7]


def test_wide_rows_fill_the_last_bins():
    a = np.zeros((16, 16), dtype=np.int64)
    a[:8, :] = 1        # 16 nonzeros
    a[8:, :10] = 1      # 10 nonzeros
    f = F.job_features(a)
    assert f[9] == 0.5 and f[8] == 0.5 and f[10] == 0.0


@pytest.mark.parametrize("la,want", [(None, 0.0), (-math.inf, -1.0), (math.nan, -1.0), (64.0, 1.0)])
def test_estimate_feature(la, want):
    assert F.job_features(np.eye(2, dtype=np.int64), log_ap=la)[10] == want


def test_empty_job_and_batch_shape():
    assert np.array_equal(F.job_features(np.zeros((0, 0))), np.zeros(12))
    X = F.features([np.eye(2), np.ones((3, 3))], [0.0, math.log(6.0)])
    assert X.shape == (2, 12) and X[1, 1] == 1.0 and X[1, 4] == 1.0
