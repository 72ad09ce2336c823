"""Pins for the oracle's HNSW search (Malkov & Yashunin Alg. 2 / Alg. 5, the
index of kANNolo Sec. 2): a hand-worked golden, brute force at ef >= n, the
equivalence of the two-heap and flag-buffer forms, the forgetful visited set,
integer closed forms and edge cases."""
import numpy as np
import pytest

import oracle as O
from helpers import golden_graph, load_golden, recall


@pytest.mark.parametrize("form", [O.FORM_TWO_HEAP, O.FORM_FLAGS])
def test_hand_worked_golden(form):
    gold = load_golden("hand_search.json")
    for case in gold["cases"]:
        g = O.import_graph(golden_graph(case))
        X = np.array(case["x"], np.float32).reshape(-1, 1)
        q = np.array([[case["q"]]], np.float32)
        for run in case["runs"]:
            ids, d, cnt = O.search_dense(g, X, q, run["k"], run["ef"], O.L2, form=form)
            assert ids[0].tolist() == run["ids"], (case["name"], run)
            assert d[0].tolist() == run["dists"]
            assert cnt[0, :2].tolist() == run["counters"][:2]
            if form == O.FORM_FLAGS:
                assert cnt[0].tolist() == run["counters"]
        kk = "exact_k2" if "exact_k2" in case else "exact_k3"
        k = len(case[kk]["ids"])
        ei, ed = O.exact_dense(X, q, k, O.L2)
        assert ei[0].tolist() == case[kk]["ids"] and ed[0].tolist() == case[kk]["dists"]


@pytest.mark.parametrize("metric", [O.L2, O.IP])
def test_brute_force_when_ef_covers_n(metric):
    rng = np.random.default_rng(21)
    X = rng.standard_normal((400, 8)).astype(np.float32)
    if metric == O.IP:
        X /= np.linalg.norm(X, axis=1, keepdims=True)
    Q = rng.standard_normal((40, 8)).astype(np.float32)
    g = O.build_dense(X, metric, 8, 50, 5)
    ids, d, _ = O.search_dense(g, X, Q, 10, 400, metric)
    ei, ed = O.exact_dense(X, Q, 10, metric)
    assert np.array_equal(ids, ei)
    assert np.array_equal(d, ed)
    # exact distances against an independent library evaluation
    if metric == O.L2:
        ref = ((Q.astype(np.float64)[:, None, :] - X.astype(np.float64)[None]) ** 2).sum(-1)
    else:
        ref = -(Q.astype(np.float64) @ X.astype(np.float64).T)
    assert np.allclose(np.take_along_axis(ref, ei, 1), ed, rtol=1e-12, atol=1e-12)


def test_two_heap_and_flag_forms_agree(cfg1_small):
    X, Q, g = cfg1_small
    for ef in (10, 32, 64, 200):
        a = O.search_dense(g, X, Q[:200], 10, ef, O.L2, form=O.FORM_TWO_HEAP)
        b = O.search_dense(g, X, Q[:200], 10, ef, O.L2, form=O.FORM_FLAGS)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
        assert np.array_equal(a[2][:, :2], b[2][:, :2])  # same layer-0 work


@pytest.mark.parametrize("cap", [1, 7, 64, 1000])
def test_forgetful_visited_set_changes_nothing(cfg1_small, cap):
    X, Q, g = cfg1_small
    a = O.search_dense(g, X, Q[:100], 10, 64, O.L2, form=O.FORM_FLAGS, visited_cap=0)
    b = O.search_dense(g, X, Q[:100], 10, 64, O.L2, form=O.FORM_FLAGS, visited_cap=cap)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert np.all(b[2][:, 0] >= a[2][:, 0])  # forgetting only adds work


@pytest.mark.parametrize("cap", [1, 3])
def test_forgetful_visited_set_changes_nothing_on_tied_integer_data(cap):
    # a table that forgets almost everything re-evaluates ids over and over;
    # the search must still return W's ids once each (equal (d, id) keys are
    # caught before they enter W twice), on data with many exact ties
    rng = np.random.default_rng(31)
    X = rng.integers(0, 6, (600, 6)).astype(np.float32)
    Q = rng.integers(0, 6, (60, 6)).astype(np.float32)
    g = O.build_dense(X, O.L2, 6, 40, 31)
    a = O.search_dense(g, X, Q, 10, 48, O.L2, visited_cap=0)
    b = O.search_dense(g, X, Q, 10, 48, O.L2, visited_cap=cap)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert all(len(set(r)) == len(r) for r in b[0])
    assert np.all(b[2][:, 0] >= a[2][:, 0])


def test_recall_reaches_one_and_grows_with_ef(cfg1_small):
    X, Q, g = cfg1_small
    ei, _ = O.exact_dense(X, Q[:100], 10, O.L2)
    rs = [recall(O.search_dense(g, X, Q[:100], 10, ef, O.L2)[0], ei, 10) for ef in (10, 20, 64, 400)]
    assert rs[-1] >= 0.999
    assert rs[0] <= rs[2] + 1e-9


def test_integer_data_distances_are_exact(int_small):
    X, Q, g = int_small
    ids, d, _ = O.search_dense(g, X, Q[:50], 10, 32, O.L2)
    xi, qi = X.astype(np.int64), Q[:50].astype(np.int64)
    ref = ((qi[:, None, :] - xi[ids]) ** 2).sum(-1)
    assert np.array_equal(ref.astype(np.float64), d)


def test_k_larger_than_ef_uses_k_and_pads():
    gold = load_golden("hand_search.json")
    case = gold["cases"][1]
    g = O.import_graph(golden_graph(case))
    X = np.array(case["x"], np.float32).reshape(-1, 1)
    q = np.array([[case["q"]]], np.float32)
    ids, d, _ = O.search_dense(g, X, q, 3, 1, O.L2)
    assert ids[0].tolist() == [3, 2, 4]  # ef_eff = max(ef, k) = 3
    ids, d, _ = O.search_dense(g, X, q, 8, 8, O.L2)
    assert ids[0].tolist()[:5] == [3, 2, 4, 1, 0] and ids[0].tolist()[5:] == [-1, -1, -1]
    assert np.all(np.isinf(d[0, 5:]))


def test_duplicates_ordered_by_id_and_self_query():
    rng = np.random.default_rng(3)
    base = rng.standard_normal((50, 4)).astype(np.float32)
    X = np.concatenate([base, base[:10]])  # ids 50..59 duplicate 0..9
    g = O.build_dense(X, O.L2, 6, 40, 9)
    ids, d, _ = O.search_dense(g, X, base[:10], 2, 60, O.L2)
    assert ids[:, 0].tolist() == list(range(10))
    assert ids[:, 1].tolist() == list(range(50, 60))
    assert np.all(d == 0.0)


def test_nan_query_does_not_fail():
    rng = np.random.default_rng(4)
    X = rng.standard_normal((200, 4)).astype(np.float32)
    g = O.build_dense(X, O.L2, 6, 40, 9)
    q = np.full((1, 4), np.nan, np.float32)
    ids, d, _ = O.search_dense(g, X, q, 5, 10, O.L2)
    assert np.all(np.isnan(d)) and np.all(ids >= 0)


# ------------------------------------------------------------------ multi-expansion form
def test_multi_expansion_hand_worked_golden():
    gold = load_golden("hand_search.json")
    multi = load_golden("hand_search_multi.json")
    cases = {c["name"]: c for c in gold["cases"]}
    for mc in multi["cases"]:
        case = cases[mc["name"]]
        g = O.import_graph(golden_graph(case))
        X = np.array(case["x"], np.float32).reshape(-1, 1)
        q = np.array([[case["q"]]], np.float32)
        for run in mc["runs"]:
            ids, d, cnt = O.search_dense_multi(g, X, q, run["k"], run["ef"], O.L2, multi["p"])
            assert ids[0].tolist() == run["ids"], (mc["name"], run)
            assert d[0].tolist() == run["dists"]
            assert cnt[0].tolist() == run["counters"]


def test_multi_expansion_with_one_entry_per_step_is_the_flag_search():
    # p = 1: the batched step reduces to the one-at-a-time step (the merge of
    # a whole neighbour list at once is the bounded top-ef insertion, which
    # does not depend on order): same ids, distances and work counts
    rng = np.random.default_rng(23)
    X = rng.integers(0, 50, (2500, 16)).astype(np.float32)
    Q = rng.integers(0, 50, (120, 16)).astype(np.float32)
    g = O.build_dense(X, O.L2, 10, 60, 23)
    for ef in (10, 40, 150):
        a = O.search_dense(g, X, Q, 10, ef, O.L2)
        b = O.search_dense_multi(g, X, Q, 10, ef, O.L2, 1)
        for x, y in zip(a, b):
            assert np.array_equal(x, y), ef


@pytest.mark.parametrize("p", [2, 4])
def test_multi_expansion_brute_force_when_ef_covers_n(p):
    rng = np.random.default_rng(29)
    X = rng.standard_normal((400, 8)).astype(np.float32)
    Q = rng.standard_normal((40, 8)).astype(np.float32)
    g = O.build_dense(X, O.L2, 8, 50, 5)
    ids, d, cnt = O.search_dense_multi(g, X, Q, 10, 400, O.L2, p)
    ei, ed = O.exact_dense(X, Q, 10, O.L2)
    assert recall(ids, ei, 10) == 1.0
    assert np.allclose(d, ed, rtol=1e-12)
    # with ef >= n every reachable node is evaluated and expanded exactly once
    assert np.all(cnt[:, 1] == cnt[:, 0] + 1)


@pytest.mark.parametrize("p", [2, 3, 4])
def test_multi_expansion_recall_near_the_one_at_a_time_search(p):
    # the batched step is a different search (not HNSW's): it may expand an
    # entry that the one-at-a-time step would evict first, so it does at
    # least as much work and finds a superset-or-equal quality W in practice
    from paper_2501_06121_b300 import datagen as G
    X, Q = G.gaussian_mixture(6000, 300, d=32, clusters=16, sigma=5.0, seed=31)
    g = O.build_dense(X, O.L2, 12, 80, 31)
    ei, _ = O.exact_dense(X, Q, 10, O.L2)
    for ef in (16, 32, 64):
        a = O.search_dense(g, X, Q, 10, ef, O.L2)
        b = O.search_dense_multi(g, X, Q, 10, ef, O.L2, p)
        assert recall(b[0], ei, 10) >= recall(a[0], ei, 10) - 0.005, (p, ef)
        assert b[2][:, 1].sum() >= a[2][:, 1].sum()
