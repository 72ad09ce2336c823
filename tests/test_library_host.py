"""Host-side logic of the library (no GPU needed): the graph builder's
levels and invariants."""
import numpy as np
import pytest

import oracle as O
from helpers import graph_problems
from paper_2501_06121_b300 import datagen as G


def test_product_levels_equal_oracle_levels():
    from paper_2501_06121_b300 import kann as K
    for M in (16, 32):
        lv, L, nu = K.kann_hnsw_levels(100_000, M, 99)
        ref = O.levels(100_000, M, 99)
        assert np.array_equal(lv, ref)
        assert L == ref.max() and nu == int(np.sum(ref >= 1))


@pytest.mark.parametrize("nthreads", [1, 4])
def test_library_builder_invariants(nthreads):
    from paper_2501_06121_b300 import kann as K
    X, _ = G.gaussian_mixture(5000, 1, d=32, clusters=16, seed=11)
    g = K.kann_hnsw_build_dense(X, K.KANN_L2, 12, 80, 11, nthreads=nthreads)
    assert graph_problems(g) == []
    base, _ = G.sparse_zipf(1500, 1, vocab=400, lam_doc=15, lam_query=5, seed=12)
    gs = K.kann_hnsw_build_sparse(base, 8, 60, 12, nthreads=nthreads)
    assert graph_problems(gs, max_unreachable=1.0) == []


def test_library_builder_single_thread_deterministic():
    from paper_2501_06121_b300 import kann as K
    X, _ = G.gaussian_mixture(3000, 1, d=32, clusters=16, seed=13)
    a = K.kann_hnsw_build_dense(X, K.KANN_L2, 12, 80, 13, nthreads=1)
    b = K.kann_hnsw_build_dense(X, K.KANN_L2, 12, 80, 13, nthreads=1)
    assert np.array_equal(a["l0"], b["l0"]) and np.array_equal(a["upper"], b["upper"])
