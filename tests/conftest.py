import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU oracle runs")


def read_adjacency(name):
    """Read a golden adjacency fixture (1-based neighbour lists) as a 0/1 matrix."""
    import numpy as np

    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            rows.append([int(x) for x in line.split()])
    n = len(rows)
    a = np.zeros((n, n), dtype=np.int64)
    for r in rows:
        for u in r[1:]:
            a[r[0] - 1, u - 1] = 1
    return a


@pytest.fixture(scope="session")
def c100_adjacency():
    return read_adjacency("c100_adjacency.txt")


@pytest.fixture(scope="session")
def c60_paper_adjacency():
    return read_adjacency("c60_adjacency.txt")
