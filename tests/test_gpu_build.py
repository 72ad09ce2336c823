"""HNSW construction with the layer-0 insertions on the GPU
(kann_hnsw_build_device; the indexing pipeline of kANNolo Sec. 2 / Fig. 1,
HNSW per Malkov & Yashunin Alg. 1 with the Alg. 4 heuristic).

The edge set of a heuristic construction has no reference value to match
(parity unpinned, as for the host builder); the device graph is held to the
same invariants as the host builder's graphs -- degree caps, no self loops or
duplicate edges, edges within their layer, levels from the counter-based
generator, the entry point on the top layer, at most 1% of a layer
unreachable -- and to the search quality of a host-built graph of the same
data: recall@10 at equal ef within 0.01 (the batched insertion differs from
sequential insertion only in that nodes of one batch do not link to each
other)."""
import numpy as np
import pytest
import torch

import oracle as O
from helpers import graph_problems, layer_lists, recall
from paper_2501_06121_b300 import datagen as G
from paper_2501_06121_b300 import kann as K

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def search_recall(g, X, Q, gt, ef):
    idx = K.kann_index_upload(K.graph_to_device(g), vectors=dev(X))
    ids, _ = K.kann_search(idx, dev(Q), 10, ef)
    torch.cuda.synchronize()
    return recall(ids.cpu().numpy(), gt, 10)


def unreachable_fraction(g, layer=0):
    nodes = np.nonzero(g["level"] >= layer)[0]
    seen = {int(g["entry"])}
    stack = [int(g["entry"])]
    while stack:
        v = stack.pop()
        for u in layer_lists(g, v, layer):
            if u not in seen:
                seen.add(u)
                stack.append(u)
    return 1.0 - len(seen) / len(nodes)


@pytest.mark.parametrize("M,efc,batch", [(12, 80, 0), (16, 100, 2048), (8, 40, 0)])
def test_device_builder_invariants(M, efc, batch):
    # the structural invariants everywhere; reachability: at most 1% of layer 0
    # unreachable, as for the host builder's graphs.  The upper layers are the
    # host builder's graph of the upper-layer nodes -- for a sequential build
    # the same graph as in a whole build, since inserting a level-0 node never
    # touches them -- and at an upper-layer cap of M = 8 a few per cent of
    # their nodes lose every in-edge to pruning
    X, _ = G.gaussian_mixture(20000, 1, d=32, clusters=16, seed=11)
    g = K.kann_hnsw_build_device(dev(X), K.KANN_L2, M, efc, 11, batch=batch)
    assert graph_problems(g, max_unreachable=0.05) == []
    assert unreachable_fraction(g, 0) <= 0.01
    lv, L, nu = K.kann_hnsw_levels(20000, M, 11)
    assert np.array_equal(g["level"], lv) and g["max_level"] == L


@pytest.mark.parametrize("metric", [K.KANN_L2, K.KANN_IP])
def test_device_builder_recall_close_to_host_builder(metric):
    if metric == K.KANN_L2:
        X, Q = G.gaussian_mixture(30000, 300, d=64, clusters=32, sigma=5.0, seed=21)
    else:
        X, Q = G.vmf_mixture(30000, 300, d=64, clusters=32, kappa=50.0, seed=21, concentration=0.2)
    gt, _ = O.exact_dense(X, Q, 10, metric)
    gh = K.kann_hnsw_build_dense(X, metric, 16, 100, 21, nthreads=0)
    gd = K.kann_hnsw_build_device(dev(X), metric, 16, 100, 21)
    assert graph_problems(gd) == []
    for ef in (16, 32, 64):
        rh, rd = search_recall(gh, X, Q, gt, ef), search_recall(gd, X, Q, gt, ef)
        assert rd >= rh - 0.01, (ef, rh, rd)


def test_device_builder_all_nodes_on_layer_zero_and_tiny_inputs():
    # M large enough that almost no node has level >= 1, and tiny n
    rng = np.random.default_rng(3)
    for n in (1, 2, 5, 300):
        X = rng.standard_normal((n, 16)).astype(np.float32)
        g = K.kann_hnsw_build_device(dev(X), K.KANN_L2, 32, 40, 5 + n)
        assert graph_problems(g) == []
        if n >= 2:
            ei, _ = O.exact_dense(X, X[:5], 1, O.L2)
            idx = K.kann_index_upload(K.graph_to_device(g), vectors=dev(X))
            ids, _ = K.kann_search(idx, dev(X[:5]), 1, max(n, 1))
            torch.cuda.synchronize()
            assert np.array_equal(ids.cpu().numpy()[:, 0], ei[:, 0])  # ef >= n: exact


def test_device_builder_sparse_invariants_and_recall():
    # sparse IP (the Splade-shaped measure): the host builder's sparse
    # invariants (reachability is not bounded for -IP graphs, whose Zipf hubs
    # win most comparisons) and recall within 0.01 of a host-built graph
    base, qs = G.sparse_zipf(8000, 200, vocab=3000, lam_doc=40, lam_query=12, seed=31)
    td = lambda c: (dev(c[0]), dev(c[1].view(np.int16)), dev(c[2]))
    b_d = td(base)
    gd = K.kann_hnsw_build_device_sparse(b_d[0], b_d[1], b_d[2], 3000, 16, 100, 31)
    assert graph_problems(gd, max_unreachable=1.0) == []
    lv, L, nu = K.kann_hnsw_levels(8000, 16, 31)
    assert np.array_equal(gd["level"], lv)
    gh = K.kann_hnsw_build_sparse(base, 16, 100, 31, nthreads=0)
    gt, _ = O.exact_sparse(base, qs, 10)
    q_d = td(qs)
    for ef in (32, 64, 128):
        rs = []
        for g in (gh, gd):
            idx = K.kann_index_upload(K.graph_to_device(g), sparse=dict(indptr=b_d[0], terms=b_d[1], weights=b_d[2],
                                                                        vocab=3000))
            ids, _ = K.kann_search_sparse(idx, q_d[0], q_d[1], q_d[2], 10, ef)
            torch.cuda.synchronize()
            rs.append(recall(ids.cpu().numpy(), gt, 10))
        assert rs[1] >= rs[0] - 0.01, (ef, rs)
