"""Batching and serving patterns: the persistent work-stealing launch, CUDA
graph replay with a device-side batch size, and the continuous-batching
server.  A query's result depends only on the query, its k and ef: the same
bits alone, in a mixed batch, in any launch form, and in the server's mix."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2501_06121_b300 import datagen as G
from paper_2501_06121_b300 import kann as K
from paper_2501_06121_b300 import serving as S

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def two_indices(cfg1_small):
    X, Q, g = cfg1_small
    Xd = dev(X)
    idx_a = K.kann_index_upload(K.graph_to_device(g.arrays()), vectors=Xd)
    # second index: E4M3 traversal + FP32 re-rank over a different data set
    X2, Q2 = G.gaussian_mixture(8000, 300, d=64, clusters=16, sigma=3.0, seed=77)
    g2 = O.build_dense(X2, O.L2, 16, 100, 77)
    X2d = dev(X2)
    c8, s8 = K.kann_quantize(X2d, K.KANN_E4M3)
    idx_b = K.kann_index_upload(K.graph_to_device(g2.arrays()), vectors=c8, dtype=K.KANN_E4M3, scale=s8, rerank=X2d)
    return dict(a=(idx_a, Q, Xd), b=(idx_b, Q2, (X2d, c8, s8)))


def single(idx, q, k, ef, **o):
    ids, d = K.kann_search_ex(idx, dev(q[None]), k, ef, **o)
    torch.cuda.synchronize()
    return ids.cpu().numpy()[0], d.cpu().numpy()[0]


def test_persistent_equals_plain(two_indices):
    idx, Q, _ = two_indices["a"]
    rng = np.random.default_rng(1)
    n = 700
    ks = rng.choice([10, 100], n).astype(np.int32)
    efs = rng.integers(64, 513, n).astype(np.int32)
    a_i, a_d = K.kann_search_batch(idx, dev(Q[:n]), dev(ks), dev(efs), kmax=100, efmax=512)
    ctr = torch.zeros(1, dtype=torch.int32, device="cuda")
    b_i, b_d = K.kann_search_batch(idx, dev(Q[:n]), dev(ks), dev(efs), kmax=100, efmax=512, work_counter=ctr)
    torch.cuda.synchronize()
    assert torch.equal(a_i, b_i) and torch.equal(a_d, b_d)
    assert int(ctr.item()) >= n


def test_device_side_count_and_graph_replay(two_indices):
    idx, Q, _ = two_indices["a"]
    cap, kmax, efmax = 256, 10, 128
    q = torch.zeros((cap, 128), device="cuda")
    k = torch.full((cap,), 10, dtype=torch.int32, device="cuda")
    ef = torch.full((cap,), 64, dtype=torch.int32, device="cuda")
    n = torch.zeros(1, dtype=torch.int32, device="cuda")
    ctr = torch.zeros(1, dtype=torch.int32, device="cuda")
    ids = torch.full((cap, kmax), -7, dtype=torch.int32, device="cuda")
    dd = torch.zeros((cap, kmax), device="cuda")
    s = torch.cuda.Stream()
    launch = lambda: K.kann_search_batch(idx, q, k, ef, kmax=kmax, efmax=efmax, ids=ids, dists=dd, stream=s,
                                         work_counter=ctr, n_device=n)
    with torch.cuda.stream(s):
        launch()
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s, capture_error_mode="relaxed"):
        launch()
    for rep, nn in enumerate((37, 256, 1)):
        ids.fill_(-7)
        q.copy_(dev(Q[rep * 256:rep * 256 + cap]))
        n.fill_(nn)
        torch.cuda.synchronize()
        with torch.cuda.stream(s):
            g.replay()
        s.synchronize()
        ref_i, ref_d = K.kann_search_ex(idx, q[:nn], 10, 64)
        torch.cuda.synchronize()
        assert torch.equal(ids[:nn], ref_i) and torch.equal(dd[:nn], ref_d)
        assert bool((ids[nn:] == -7).all())  # rows past the device-side count are untouched


@pytest.mark.parametrize("tuned", [False, True])
def test_server_results_equal_alone_and_in_the_mix(two_indices, tuned):
    # tuned: the server picks each index's launch settings with the
    # autotuner (team size, visited table, ...), which never changes results
    idx_a, Qa, _ = two_indices["a"]
    idx_b, Qb, _ = two_indices["b"]
    indices = {"a": dict(index=idx_a, d=128, kmax=100, efmax=512),
               "b": dict(index=idx_b, d=64, kmax=100, efmax=512, opts=dict(rerank=-1))}
    tq = {"a": dev(Qa[:300]), "b": dev(Qb[:300])} if tuned else None
    srv = S.SearchServer(indices, page_capacity=128, max_pages=6, tune_queries=tq)
    assert set(srv.tuned) == ({"a", "b"} if tuned else set())
    reqs = S.poisson_requests(20000.0, 0.05, {"a": Qa, "b": Qb}, seed=5)
    done = srv.run(reqs, time_limit=30.0)
    assert len(done) == len(reqs)
    for r in done[::7]:
        idx = idx_a if r["index"] == "a" else idx_b
        o = dict(rerank=-1) if r["index"] == "b" else {}
        si, sd = single(idx, r["query"], r["k"], r["ef"], **o)
        assert np.array_equal(si, r["ids"]) and np.array_equal(sd, r["dists"])
    assert all(r["status"] & K.KANN_QSTAT_BAD_ID == 0 for r in done)
    summ = S.latency_summary(done, 0.05)
    assert summ["completed"] == len(reqs) and summ["p99_ms"] >= summ["p50_ms"] > 0


def test_server_admits_by_memory_as_it_frees(two_indices):
    # a budget with room for two pages in all: bursts on two indices take the
    # memory in turn (pages of the idle index are released), and every result
    # still equals a single call
    idx_a, Qa, _ = two_indices["a"]
    idx_b, Qb, _ = two_indices["b"]
    spec = {"a": dict(index=idx_a, d=128, kmax=10, efmax=128), "b": dict(index=idx_b, d=64, kmax=10, efmax=128)}
    pa = K.kann_search_workspace_bytes(idx_a, 64, 10, 128)
    pb = K.kann_search_workspace_bytes(idx_b, 64, 10, 128)
    srv = S.SearchServer(spec, page_capacity=64, memory_budget=max(pa, pb) * 2, max_pages=8)
    ra = S.poisson_requests(200000.0, 0.01, {"a": Qa}, k_choices=(10,), ef_range=(16, 128), seed=7)
    rb = S.poisson_requests(200000.0, 0.01, {"b": Qb}, k_choices=(10,), ef_range=(16, 128), seed=8)
    for r in rb:
        r["t"] += 0.03  # b's burst after a's
    done = srv.run(ra + rb, time_limit=60.0)
    assert len(done) == len(ra) + len(rb)
    assert srv.stats["peak_bytes"] <= max(pa, pb) * 2
    assert srv.stats["admissions_waited_for_memory"] > 0 and srv.stats["pages_released"] > 0
    for r in done[::11]:
        si, sd = single(idx_a if r["index"] == "a" else idx_b, r["query"], r["k"], r["ef"])
        assert np.array_equal(si, r["ids"]) and np.array_equal(sd, r["dists"])
    assert S.status_counts(done)["bad_id"] == 0


def test_autotuner_returns_result_preserving_settings(two_indices, tmp_path):
    from paper_2501_06121_b300 import autotune as A
    idx, Q, _ = two_indices["a"]
    Qd = dev(Q[:500])
    cache = str(tmp_path / "tune.json")
    opts = A.tune(idx, Qd, 10, 64, reps=2, cache_path=cache)
    assert set(opts) == {"lanes_per_row", "hash_bits", "visited_format", "warps_per_block", "lean", "team",
                         "persistent"}
    a_i, a_d = A.search_with(idx, Qd, 10, 64, opts)
    b_i, b_d = K.kann_search_ex(idx, Qd, 10, 64)
    torch.cuda.synchronize()
    assert torch.equal(a_i, b_i) and torch.equal(a_d, b_d)
    assert A.tune(idx, Qd, 10, 64, reps=2, cache_path=cache) == opts  # served from the cache


def test_admission_bytes_follow_the_settings(two_indices):
    idx_a, Qa, _ = two_indices["a"]
    idx_b, _, _ = two_indices["b"]
    assert K.kann_search_workspace_bytes(idx_a, 100, 10, 64) == 100 * 128 * 4 + 100 * 8 + 100 * 10 * 8 + 100 * 4 + 8
    assert K.kann_search_workspace_bytes(idx_b, 7, 100, 512) == 7 * 64 * 4 + 7 * 8 + 7 * 100 * 8 + 7 * 4 + 8
    assert K.kann_search_workspace_bytes(idx_a, 0, 10, 64) == 8
    assert K.kann_search_workspace_bytes(idx_a, 10, 10, K.KANN_MAX_EF + 1) == 0
    assert K.kann_search_workspace_bytes(idx_a, 10, 0, 64) == 0
    assert K.kann_search_workspace_bytes(idx_a, -1, 10, 64) == 0
    # the server sizes its pages with it, halving the capacity until one fits
    # the budget, and never lets the live pages exceed the budget
    spec = {"a": dict(index=idx_a, d=128, kmax=10, efmax=64)}
    per_page = K.kann_search_workspace_bytes(idx_a, 64, 10, 64)
    srv = S.SearchServer(spec, page_capacity=256, memory_budget=per_page)
    assert srv.caps["a"] == 64 and srv.page_bytes["a"] == per_page
    reqs = S.poisson_requests(100000.0, 0.01, {"a": Qa}, k_choices=(10,), ef_range=(16, 64), seed=2)
    done = srv.run(reqs, time_limit=60.0)
    assert len(done) == len(reqs) and srv.stats["peak_bytes"] <= per_page and len(srv.pages) == 1
    with pytest.raises(ValueError):
        S.SearchServer({"a": dict(index=idx_a, d=128, kmax=10, efmax=K.KANN_MAX_EF + 1)})


def test_host_batch_pipeline_equals_single_calls(two_indices):
    # batches from pinned host memory with copies overlapped on two copy
    # streams: each batch's results equal one kann_search_ex call's
    idx, Q, _ = two_indices["a"]
    n = 200
    pipe = S.HostBatchPipeline(idx, n, 128, 10, 64)
    outs = []
    for b in range(5):
        qh = torch.from_numpy(np.ascontiguousarray(Q[b * n:(b + 1) * n])).pin_memory()
        ih = torch.empty((n, 10), dtype=torch.int32).pin_memory()
        dh = torch.empty((n, 10), dtype=torch.float32).pin_memory()
        pipe.submit(qh, ih, dh)
        outs.append((qh, ih, dh))
    pipe.synchronize()
    for qh, ih, dh in outs:
        ri, rd = K.kann_search_ex(idx, qh.cuda(), 10, 64)
        torch.cuda.synchronize()
        assert torch.equal(ih, ri.cpu()) and torch.equal(dh, rd.cpu())
