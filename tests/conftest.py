import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the library's kernels)")


@pytest.fixture(scope="session")
def cfg1_small():
    """The plain FP32 L2 parity workload: 10,000 x 128 Gaussian mixture (32
    clusters, centres U[0,100], sigma 5), M=16, efConstruction=100, seed 1,
    with 1,000 queries (the first 100 are the 100-query set)."""
    import oracle as O
    from paper_2501_06121_b300 import datagen as G
    X, Q = G.gaussian_mixture(10000, 1000, d=128, clusters=32, sigma=5.0, seed=1)
    g = O.build_dense(X, O.L2, 16, 100, 1)
    return X, Q, g


@pytest.fixture(scope="session")
def int_small():
    """Integer-valued mixture at reduced size (20,000 x 128, values 0..255),
    M=16, efConstruction=100: distances are exact in FP32/FP16/BF16."""
    import oracle as O
    from paper_2501_06121_b300 import datagen as G
    X, Q = G.integer_mixture(20000, 300, d=128, clusters=64, sigma=20.0, seed=2)
    g = O.build_dense(X, O.L2, 16, 100, 2)
    return X, Q, g
