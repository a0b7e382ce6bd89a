import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")


def bsr_dense(row_ptr, col, vals, nrows=None, ncols=None):
    """Dense matrix of a block-CSR matrix (test helper)."""
    vals = np.asarray(vals)
    b = vals.shape[-1]
    nr = len(row_ptr) - 1 if nrows is None else nrows
    nc = (int(np.max(col)) + 1 if len(col) else 0) if ncols is None else ncols
    A = np.zeros((nr * b, nc * b))
    for i in range(len(row_ptr) - 1):
        for p in range(row_ptr[i], row_ptr[i + 1]):
            j = col[p]
            A[i * b:(i + 1) * b, j * b:(j + 1) * b] = vals[p]
    return A


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle
    oracle.build()
    return oracle
