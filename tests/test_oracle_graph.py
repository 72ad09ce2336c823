"""Graph invariants of HNSW construction (Malkov & Yashunin Alg. 1/4) for the
oracle's builder and for the library's host builder."""
import numpy as np
import pytest

import oracle as O
from helpers import graph_problems
from paper_2501_06121_b300 import datagen as G


def _unit(rng, n, d):
    x = rng.standard_normal((n, d)).astype(np.float32)
    return x / np.linalg.norm(x, axis=1, keepdims=True)


def test_oracle_graph_dense_l2_invariants(cfg1_small):
    X, Q, g = cfg1_small
    ga = g.arrays()
    assert graph_problems(ga) == []
    assert ga["M"] == 16 and ga["M0"] == 32
    assert np.array_equal(ga["level"], O.levels(len(X), 16, 1))


def test_oracle_graph_ip_invariants():
    rng = np.random.default_rng(5)
    X = _unit(rng, 3000, 32)
    g = O.build_dense(X, O.IP, 8, 60, 3)
    assert graph_problems(g.arrays()) == []


def test_oracle_graph_sparse_invariants():
    base, _ = G.sparse_zipf(2000, 1, vocab=500, lam_doc=20, lam_query=5, seed=9)
    g = O.build_sparse(*base, M=8, efC=60, seed=4)
    # -IP is not a metric: under a Zipf term law the heuristic prunes the
    # back-links of many documents (hubs win every comparison), so layer-0
    # reachability is not bounded here; every other invariant still holds.
    assert graph_problems(g.arrays(), max_unreachable=1.0) == []


def test_oracle_graph_simple_rule_invariants():
    rng = np.random.default_rng(6)
    X = rng.standard_normal((2000, 16)).astype(np.float32)
    g = O.build_dense(X, O.L2, 8, 40, 3, simple=True)
    ga = g.arrays()
    # the nearest-M rule keeps clustered lists, so a few more nodes lose all in-edges
    assert graph_problems(ga, max_unreachable=0.1) == []


def test_oracle_build_deterministic():
    rng = np.random.default_rng(7)
    X = rng.standard_normal((1500, 16)).astype(np.float32)
    a = O.build_dense(X, O.L2, 8, 40, 3).arrays()
    b = O.build_dense(X, O.L2, 8, 40, 3).arrays()
    for key in ("level", "l0", "upper_slot", "upper"):
        assert np.array_equal(a[key], b[key])
    assert a["entry"] == b["entry"]
