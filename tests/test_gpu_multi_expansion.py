"""The multi-expansion layer-0 search (kann_search_opts.expand = p > 1) against
its oracle form.

HNSW's layer-0 step (Malkov & Yashunin Alg. 2, the index of kANNolo Sec. 2)
expands one entry at a time.  The batched variant marks the p best
unexpanded entries of W expanded together, evaluates all their unvisited
neighbours in one batch and keeps the ef best; it is a different search, so
its contract is twofold:
  * against the oracle's implementation of the same rule
    (oracle.search_dense_multi): the parity contract of the other tests --
    bit for bit on integer data, >= 99.9% identical ID sets and distances
    within 1e-5 * max(|d|, sum |terms|) on real-valued data;
  * against the one-expansion search at equal ef: recall@10 within 0.005.
"""
import numpy as np
import pytest
import torch

import oracle as O
from helpers import golden_graph, id_set_match_fraction, load_golden, recall
from paper_2501_06121_b300 import kann as K

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def search(idx, Q, k, ef, **opts):
    ids, d = K.kann_search_ex(idx, dev(Q.astype(np.float32)), k, ef, **opts)
    torch.cuda.synchronize()
    return ids.cpu().numpy(), d.cpu().numpy()


@pytest.mark.parametrize("p", [2, 3, 4])
@pytest.mark.parametrize("dtype", [K.KANN_F32, K.KANN_F16])
def test_multi_expansion_integer_bit_exact_with_work_counts(int_small, p, dtype):
    X, Q, g = int_small
    Xd = dev(X)
    data = Xd if dtype == K.KANN_F32 else K.kann_quantize(Xd, dtype)[0]
    idx = K.kann_index_upload(K.graph_to_device(g.arrays()), vectors=data, dtype=dtype)
    for ef in (16, 64, 300):
        oi, od, oc = O.search_dense_multi(g, X, Q, 10, ef, O.L2, p)
        cnt = torch.zeros((len(Q), 4), dtype=torch.int32, device="cuda")
        gi, gd = search(idx, Q, 10, ef, expand=p, hash_bits=15, counters=cnt)
        assert np.array_equal(gi, oi), (p, ef)
        assert np.array_equal(gd.astype(np.float64), od), (p, ef)
        assert np.array_equal(cnt.cpu().numpy().astype(np.int64), oc), (p, ef)


@pytest.mark.parametrize("fmt", [K.KANN_VISITED_COMPACT, K.KANN_VISITED_WIDE])
def test_multi_expansion_forgetful_table_changes_nothing(int_small, fmt):
    # the forgetting argument holds per batch too: a forgotten id is either in
    # W (caught by the merge) or worse than worst(W), which only improves
    X, Q, g = int_small
    idx = K.kann_index_upload(K.graph_to_device(g.arrays()), vectors=dev(X))
    bi, bd = search(idx, Q, 10, 128, expand=3, hash_bits=15, visited_format=fmt)
    gi, gd = search(idx, Q, 10, 128, expand=3, hash_bits=5, visited_format=fmt)
    assert np.array_equal(gi, bi) and np.array_equal(gd, bd)


@pytest.mark.parametrize("p", [2, 4])
def test_multi_expansion_real_valued_parity_and_recall_contract(cfg1_small, p):
    X, Q, g = cfg1_small
    idx = K.kann_index_upload(K.graph_to_device(g.arrays()), vectors=dev(X))
    ei, _ = O.exact_dense(X, Q, 10, O.L2)
    for ef in (16, 32, 64, 128):
        oi, od, _ = O.search_dense_multi(g, X, Q, 10, ef, O.L2, p)
        gi, gd = search(idx, Q, 10, ef, expand=p)
        assert id_set_match_fraction(gi, oi) >= 0.999, ef
        ref = O.dist_dense(X, Q, gi, O.L2)
        assert np.all(np.abs(gd - ref) <= 1e-5 * np.abs(ref) + 1e-30)
        # the recall contract against the one-expansion (parity) search
        si, _ = search(idx, Q, 10, ef)
        assert recall(gi, ei, 10) >= recall(si, ei, 10) - 0.005, ef


def test_multi_expansion_with_rerank_and_mixed_batch(cfg1_small):
    X, Q, g = cfg1_small
    Xd = dev(X)
    idx = K.kann_index_upload(K.graph_to_device(g.arrays()), vectors=K.kann_quantize(Xd, K.KANN_F16)[0],
                              dtype=K.KANN_F16, rerank=Xd)
    th = K.kann_quantize(Xd, K.KANN_F16)[0].cpu().view(torch.int16).numpy().view(np.uint16)
    ti, _, _ = O.search_dense_multi(g, th, Q, 64, 64, O.L2, 2, dtype=O.DT_F16)
    oi, od = O.rerank_dense(X, Q, ti, 10, O.L2)
    gi, gd = search(idx, Q, 10, 64, expand=2, rerank=-1)
    assert id_set_match_fraction(gi, oi) >= 0.999
    # a mixed-k/ef batch in the persistent launch equals single calls
    rng = np.random.default_rng(4)
    n = 200
    ks = rng.choice([1, 10, 50], n).astype(np.int32)
    efs = rng.integers(16, 200, n).astype(np.int32)
    ctr = torch.zeros(1, dtype=torch.int32, device="cuda")
    bi, bd = K.kann_search_batch(idx, dev(Q[:n]), dev(ks), dev(efs), kmax=50, efmax=200, expand=3,
                                 work_counter=ctr)
    torch.cuda.synchronize()
    bi, bd = bi.cpu().numpy(), bd.cpu().numpy()
    for q in range(0, n, 9):
        si, sd = search(idx, Q[q:q + 1], int(ks[q]), int(efs[q]), expand=3)
        assert np.array_equal(bi[q, :ks[q]], si[0]) and np.array_equal(bd[q, :ks[q]], sd[0])


def test_multi_expansion_option_checks(cfg1_small):
    X, Q, g = cfg1_small
    idx = K.kann_index_upload(K.graph_to_device(g.arrays()), vectors=dev(X))
    with pytest.raises(K.KannError):
        search(idx, Q[:4], 10, 32, expand=K.KANN_MAX_EXPAND + 1)
    st = torch.zeros(4, dtype=torch.int32, device="cuda")
    gi, _ = search(idx, Q[:4], 10, 64, expand=4, max_hops=3, status=st)
    assert np.all((st.cpu().numpy() & K.KANN_QSTAT_HOPCAP) != 0) and np.all(gi[:, 0] >= 0)
    # multi-expansion is a dense-index option
    rng = np.random.default_rng(1)
    cb = rng.standard_normal((16, 256, 8)).astype(np.float32)
    codes = rng.integers(0, 256, (len(X), 16)).astype(np.uint8)
    ip = K.kann_index_upload(K.graph_to_device(g.arrays()), pq=dict(codes=dev(codes), codebooks=dev(cb),
                                                                    metric=K.KANN_L2))
    with pytest.raises(K.KannError):
        search(ip, Q[:4], 10, 32, expand=2)


def test_multi_expansion_hand_worked_golden_on_gpu():
    # the hand-worked multi-expansion cases (ids, distances and work counters)
    gold = {c["name"]: c for c in load_golden("hand_search.json")["cases"]}
    multi = load_golden("hand_search_multi.json")
    for mc in multi["cases"]:
        case = gold[mc["name"]]
        X = np.zeros((len(case["x"]), 4), np.float32)
        X[:, 0] = case["x"]  # padded to 16 bytes per row; L2 unchanged
        q = np.zeros((1, 4), np.float32)
        q[0, 0] = case["q"]
        idx = K.kann_index_upload(K.graph_to_device(golden_graph(case)), vectors=dev(X))
        for run in mc["runs"]:
            cnt = torch.zeros((1, 4), dtype=torch.int32, device="cuda")
            gi, gd = search(idx, q, run["k"], run["ef"], expand=multi["p"], counters=cnt)
            assert gi[0].tolist() == run["ids"] and gd[0].tolist() == run["dists"], (mc["name"], run)
            assert cnt.cpu().numpy()[0].tolist() == run["counters"], (mc["name"], run)
