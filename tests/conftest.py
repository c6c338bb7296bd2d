import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the CUDA library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def csr_from_edges(n, edges):
    import numpy as np
    rows, cols = [], []
    for a, b in edges:
        rows += [a, b]
        cols += [b, a]
    for i in range(n):
        rows.append(i)
        cols.append(i)
    order = np.lexsort((cols, rows))
    rows = np.asarray(rows)[order]
    cols = np.asarray(cols, dtype=np.int32)[order]
    rp = np.zeros(n + 1, np.int32)
    np.cumsum(np.bincount(rows, minlength=n), out=rp[1:])
    return rp, cols


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle
    oracle.lib()
    return oracle
