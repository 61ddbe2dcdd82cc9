import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")


@pytest.fixture(scope="session")
def small_a():
    """Config A shape at reduced size: 4000 vectors, D=128, nlist=16, M=16."""
    from workloads import make_dataset, train_ivfpq
    d = make_dataset("A", n=4000, nq=24)
    ix = train_ivfpq(d["base"], 16, 16, seed=1, device="cpu")
    return d, ix


def int_dataset(n=600, dim=8, nlist=4, hi=15, seed=7):
    """Tiny integer data whose PQ (dsub = 1) reconstructs every vector exactly."""
    r = np.random.Generator(np.random.PCG64(seed))
    base = r.integers(0, hi + 1, size=(n, dim)).astype(np.float32)
    cent = base[r.permutation(n)[:nlist]].copy()
    d2 = ((base[:, None, :] - cent[None]) ** 2).sum(-1)
    list_of = np.argmin(d2, axis=1).astype(np.int32)
    res = base - cent[list_of]
    vals = np.arange(-hi, hi + 1, dtype=np.float32)          # every residual value
    books = np.zeros((dim, 256, 1), dtype=np.float32)
    books[:, :len(vals), 0] = vals[None, :]
    books[:, len(vals):, 0] = 1000.0                          # unused, far away
    codes = (res + hi).astype(np.uint8)
    return base, dict(centroids=cent, codebooks=books, codes=codes, list_of=list_of)
