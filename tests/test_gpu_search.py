"""Parity of the CUDA search path (through the C ABI) with the FP64 oracle.

Contract (HNSW search, the index of kANNolo Sec. 2): with the oracle's
graph and the same seeded inputs, the FP32 GPU search returns the same ID
set as the oracle on >= 99.9% of queries, every returned distance agrees
with the oracle's FP64 distance of that id within
1e-5 * max(|d|, sum |terms|), and recall@k against exact k-NN stays within
0.002 of the oracle's at every ef.  On integer-valued data every distance
is exact in FP32/FP16/BF16, so there the results are identical bit for bit.
"""
import numpy as np
import pytest
import torch

import oracle as O
from helpers import golden_graph, id_set_match_fraction, load_golden, recall
from paper_2501_06121_b300 import datagen as G
from paper_2501_06121_b300 import kann as K

pytestmark = pytest.mark.gpu

DT_O = {K.KANN_F32: O.DT_F32, K.KANN_F16: O.DT_F16, K.KANN_BF16: O.DT_BF16, K.KANN_E4M3: O.DT_E4M3}


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def upload(garr, X, dtype=K.KANN_F32, metric=K.KANN_L2, rerank=False):
    Xd = dev(X.astype(np.float32))
    scale = None
    data = Xd
    if dtype != K.KANN_F32:
        data, scale = K.kann_quantize(Xd, dtype)
    idx = K.kann_index_upload(K.graph_to_device(garr), vectors=data, dtype=dtype, metric=metric, scale=scale,
                              rerank=Xd if rerank else None)
    return idx, data, scale


def search(idx, Q, k, ef, **opts):
    ids, d = K.kann_search_ex(idx, dev(Q.astype(np.float32)), k, ef, **opts)
    torch.cuda.synchronize()
    return ids.cpu().numpy(), d.cpu().numpy()


def check_dists(X, Q, ids, d_gpu, metric, dtype=O.DT_F32, scale=None):
    """Every returned distance vs the oracle's FP64 distance of that id."""
    ref = O.dist_dense(X, Q, np.maximum(ids, 0), metric, dtype=dtype, scale=scale)
    if metric == O.L2:
        mag = np.abs(ref)
    else:
        Xv = X.astype(np.float64) if dtype == O.DT_F32 else None
        if Xv is None:
            mag = np.abs(ref) + 1.0
        else:
            mag = np.einsum("qd,qkd->qk", np.abs(Q.astype(np.float64)), np.abs(Xv[np.maximum(ids, 0)]))
    ok = ids >= 0
    err = np.abs(d_gpu.astype(np.float64) - ref)
    assert np.all(err[ok] <= 1e-5 * np.maximum(np.abs(ref[ok]), mag[ok]) + 1e-30), err[ok].max()


# ------------------------------------------------------------------ FP32 parity
def test_fp32_l2_parity_cfg1(cfg1_small):
    X, Q, g = cfg1_small
    idx, _, _ = upload(g.arrays(), X)
    ei, _ = O.exact_dense(X, Q, 10, O.L2)
    for ef in (16, 32, 64, 128):
        oi, od, _ = O.search_dense(g, X, Q, 10, ef, O.L2)
        gi, gd = search(idx, Q, 10, ef)
        assert id_set_match_fraction(gi, oi) >= 0.999, ef
        check_dists(X, Q, gi, gd, O.L2)
        assert abs(recall(gi, ei, 10) - recall(oi, ei, 10)) <= 0.002
    # the 100-query set at ef = 64, k = 10
    oi, _, _ = O.search_dense(g, X, Q[:100], 10, 64, O.L2)
    gi, _ = search(idx, Q[:100], 10, 64)
    assert id_set_match_fraction(gi, oi) >= 0.999


def test_counters_match_oracle_work(int_small):
    # integer data: identical decisions, so identical work (expansions and
    # upper-layer evaluations always; layer-0 evaluations when the visited
    # table never forgot)
    X, Q, g = int_small
    idx, _, _ = upload(g.arrays(), X)
    oi, _, oc = O.search_dense(g, X, Q, 10, 64, O.L2)
    cnt = torch.zeros((len(Q), 4), dtype=torch.int32, device="cuda")
    st = torch.zeros(len(Q), dtype=torch.int32, device="cuda")
    gi, _ = search(idx, Q, 10, 64, counters=cnt, status=st, hash_bits=14)
    c = cnt.cpu().numpy()
    assert np.array_equal(gi, oi)
    assert np.array_equal(c[:, 1:], oc[:, 1:])
    noforget = (st.cpu().numpy() & K.KANN_QSTAT_FORGOT) == 0
    assert noforget.mean() > 0.9
    assert np.array_equal(c[noforget, 0], oc[noforget, 0])
    assert np.all(c[:, 0] >= oc[:, 0])


# ------------------------------------------------------------------ exact integer closed form
@pytest.mark.parametrize("dtype", [K.KANN_F32, K.KANN_F16, K.KANN_BF16])
def test_integer_data_bit_exact(int_small, dtype):
    X, Q, g = int_small
    idx, _, _ = upload(g.arrays(), X, dtype=dtype)
    for ef in (16, 64, 200):
        oi, od, oc = O.search_dense(g, X, Q, 10, ef, O.L2)
        gi, gd = search(idx, Q, 10, ef)
        assert np.array_equal(gi, oi)
        assert np.array_equal(gd.astype(np.float64), od)


# Row widths that tile the lanes exactly (compile-time lane mapping) and widths
# that do not (general kernels), plus lane-mapping overrides at d = 128: on
# integer data every form must reproduce the oracle bit for bit.
@pytest.fixture(scope="module")
def int_dims():
    out = {}
    for d in (48, 64, 96, 256):
        X, Q = G.integer_mixture(4000, 120, d=d, clusters=16, sigma=20.0, seed=40 + d)
        out[d] = (X, Q, O.build_dense(X, O.L2, 16, 64, 40 + d))
    return out


@pytest.mark.parametrize("d", [48, 64, 96, 256])
@pytest.mark.parametrize("dtype", [K.KANN_F32, K.KANN_F16, K.KANN_BF16])
def test_integer_bit_exact_across_row_widths(int_dims, d, dtype):
    X, Q, g = int_dims[d]
    idx, _, _ = upload(g.arrays(), X, dtype=dtype)
    oi, od, _ = O.search_dense(g, X, Q, 10, 48, O.L2)
    gi, gd = search(idx, Q, 10, 48)
    assert np.array_equal(gi, oi)
    assert np.array_equal(gd.astype(np.float64), od)


@pytest.mark.parametrize("dtype,lpr", [(K.KANN_F16, 4), (K.KANN_F16, 16), (K.KANN_F16, 32), (K.KANN_F32, 4),
                                       (K.KANN_F32, 16), (K.KANN_BF16, 16)])
def test_lane_mapping_overrides_bit_exact(int_small, dtype, lpr):
    X, Q, g = int_small
    idx, _, _ = upload(g.arrays(), X, dtype=dtype)
    oi, od, _ = O.search_dense(g, X, Q, 10, 64, O.L2)
    gi, gd = search(idx, Q, 10, 64, lanes_per_row=lpr)
    assert np.array_equal(gi, oi)
    assert np.array_equal(gd.astype(np.float64), od)


@pytest.mark.parametrize("dtype", [K.KANN_F16, K.KANN_BF16])
@pytest.mark.parametrize("d", [64, 128, 256])
def test_lean_form_bit_exact(int_dims, int_small, dtype, d):
    X, Q, g = int_small if d == 128 else int_dims[d]
    idx, _, _ = upload(g.arrays(), X, dtype=dtype)
    oi, od, _ = O.search_dense(g, X, Q, 10, 48, O.L2)
    gi, gd = search(idx, Q, 10, 48, lean=1)
    assert np.array_equal(gi, oi)
    assert np.array_equal(gd.astype(np.float64), od)


@pytest.mark.parametrize("d", [64, 96, 256])
def test_e4m3_parity_across_row_widths(int_dims, d):
    X, Q, g = int_dims[d]
    idx, codes, scale = upload(g.arrays(), X, dtype=K.KANN_E4M3)
    c, s = codes.cpu().numpy(), scale.cpu().numpy()
    oi, od, _ = O.search_dense(g, c, Q, 10, 48, O.L2, dtype=O.DT_E4M3, scale=s)
    gi, gd = search(idx, Q, 10, 48)
    assert id_set_match_fraction(gi, oi) >= 0.999
    check_dists(c, Q, gi, gd, O.L2, dtype=O.DT_E4M3, scale=s)


@pytest.mark.parametrize("fmt", [K.KANN_VISITED_COMPACT, K.KANN_VISITED_WIDE])
def test_forgetful_table_changes_nothing(int_small, fmt):
    # a table of 32 slots forgets almost everything (full buckets or probe
    # windows, and a clear after nearly every expansion): the results stay
    # those of a table that never forgets
    X, Q, g = int_small
    idx, _, _ = upload(g.arrays(), X)
    base_i, base_d = search(idx, Q, 10, 128, hash_bits=14, visited_format=fmt)
    st = torch.zeros(len(Q), dtype=torch.int32, device="cuda")
    cnt = torch.zeros((len(Q), 4), dtype=torch.int32, device="cuda")
    gi, gd = search(idx, Q, 10, 128, hash_bits=5, status=st, counters=cnt, visited_format=fmt)
    assert np.array_equal(gi, base_i) and np.array_equal(gd, base_d)
    assert np.all((st.cpu().numpy() & K.KANN_QSTAT_FORGOT) != 0)


@pytest.mark.parametrize("ef", [16, 64, 300])
def test_visited_formats_and_sizes_agree_bit_for_bit(int_small, ef):
    # compact (16-bit slots, ids split into bucket and slot value) and wide
    # (32-bit id slots) tables of several sizes: the same results, and with a
    # table that never forgets, the oracle's work counts
    X, Q, g = int_small
    idx, _, _ = upload(g.arrays(), X, dtype=K.KANN_F16)
    oi, od, oc = O.search_dense(g, X, Q, 10, ef, O.L2)
    for fmt, hb in ((K.KANN_VISITED_COMPACT, 0), (K.KANN_VISITED_COMPACT, 9), (K.KANN_VISITED_COMPACT, 16),
                    (K.KANN_VISITED_WIDE, 0), (K.KANN_VISITED_WIDE, 15)):
        cnt = torch.zeros((len(Q), 4), dtype=torch.int32, device="cuda")
        gi, gd = search(idx, Q, 10, ef, hash_bits=hb, visited_format=fmt, counters=cnt)
        assert np.array_equal(gi, oi), (fmt, hb)
        assert np.array_equal(gd.astype(np.float64), od), (fmt, hb)
        if hb >= 15:
            assert np.array_equal(cnt.cpu().numpy().astype(np.int64), oc), (fmt, hb)


def test_compact_table_needs_room_for_the_ids(int_small):
    # 2^5 compact slots hold ids of at most 5 + 12 bits: a 20,000-node index
    # fits, and an explicit request that cannot fit is refused
    X, Q, g = int_small
    idx, _, _ = upload(g.arrays(), X)
    search(idx, Q[:4], 10, 32, hash_bits=5, visited_format=K.KANN_VISITED_COMPACT)
    big = dict(g.arrays())
    n = 1 << 18
    Xb = np.zeros((n, 128), np.float32)
    garr = dict(n=n, M=big["M"], M0=big["M0"], max_level=0, entry=0, level=np.zeros(n, np.int8),
                l0=np.full((n, big["M0"]), -1, np.int32), upper_slot=np.full(n, -1, np.int32),
                upper=np.full((1, 1, big["M"]), -1, np.int32))
    ib = K.kann_index_upload(K.graph_to_device(garr), vectors=dev(Xb))
    with pytest.raises(K.KannError):
        search(ib, Q[:4], 10, 32, hash_bits=5, visited_format=K.KANN_VISITED_COMPACT)
    gi, _ = search(ib, Q[:4], 10, 32, hash_bits=5)  # automatic: falls back to the wide table
    assert np.all(gi[:, 0] == 0) and np.all(gi[:, 1:] == -1)


# ------------------------------------------------------------------ other measures / formats
def test_ip_parity():
    X, Q = G.vmf_mixture(6000, 1000, d=64, clusters=16, kappa=50.0, seed=31)
    g = O.build_dense(X, O.IP, 16, 100, 31)
    idx, _, _ = upload(g.arrays(), X, metric=K.KANN_IP)
    oi, od, _ = O.search_dense(g, X, Q, 10, 64, O.IP)
    gi, gd = search(idx, Q, 10, 64)
    assert id_set_match_fraction(gi, oi) >= 0.999
    check_dists(X, Q, gi, gd, O.IP)


def test_quantize_matches_oracle_codecs():
    rng = np.random.default_rng(8)
    X = (rng.standard_normal((777, 64)) * 10.0 ** rng.integers(-3, 4, (777, 1))).astype(np.float32)
    X[5] = 0.0
    Xd = dev(X)
    h, _ = K.kann_quantize(Xd, K.KANN_F16)
    b, _ = K.kann_quantize(Xd, K.KANN_BF16)
    e, s = K.kann_quantize(Xd, K.KANN_E4M3)
    torch.cuda.synchronize()
    assert np.array_equal(h.cpu().view(torch.int16).numpy().view(np.uint16), O.encode_f16(X))
    assert np.array_equal(b.cpu().view(torch.int16).numpy().view(np.uint16), O.encode_bf16(X))
    oc, os_ = O.encode_e4m3_rows(X)
    assert np.array_equal(e.cpu().numpy(), oc)
    assert np.array_equal(s.cpu().numpy(), os_)


def test_e4m3_traversal_parity(cfg1_small):
    X, Q, g = cfg1_small
    idx, codes, scale = upload(g.arrays(), X, dtype=K.KANN_E4M3)
    c, s = codes.cpu().numpy(), scale.cpu().numpy()
    oi, od, _ = O.search_dense(g, c, Q, 10, 64, O.L2, dtype=O.DT_E4M3, scale=s)
    gi, gd = search(idx, Q, 10, 64)
    assert id_set_match_fraction(gi, oi) >= 0.999
    check_dists(c, Q, gi, gd, O.L2, dtype=O.DT_E4M3, scale=s)


@pytest.mark.parametrize("dtype", [K.KANN_F16, K.KANN_BF16, K.KANN_E4M3])
def test_reduced_precision_traversal_plus_rerank(cfg1_small, dtype):
    X, Q, g = cfg1_small
    idx, data, scale = upload(g.arrays(), X, dtype=dtype, rerank=True)
    ef, k = 64, 10
    if dtype == K.KANN_E4M3:
        tdata, tscale = data.cpu().numpy(), scale.cpu().numpy()
    else:
        tdata = data.cpu().view(torch.int16).numpy().view(np.uint16)
        tscale = None
    # oracle: traverse on the stored format, keep all ef, re-rank in FP64 on FP32
    ti, _, _ = O.search_dense(g, tdata, Q, ef, ef, O.L2, dtype=DT_O[dtype], scale=tscale)
    oi, od = O.rerank_dense(X, Q, ti, k, O.L2)
    gi, gd = search(idx, Q, k, ef, rerank=-1)
    assert id_set_match_fraction(gi, oi) >= 0.999
    check_dists(X, Q, gi, gd, O.L2)
    # re-ranked distances equal the FP32 traversal's distances bit for bit
    idx32, _, _ = upload(g.arrays(), X)
    fi, fd = search(idx32, Q, k, 400)
    for q in range(0, len(Q), 7):
        common = set(fi[q]) & set(gi[q])
        for i in common:
            assert fd[q][list(fi[q]).index(i)] == gd[q][list(gi[q]).index(i)]


# ------------------------------------------------------------------ batch, golden, edge cases
def test_mixed_batch_equals_single_calls(cfg1_small):
    X, Q, g = cfg1_small
    idx, _, _ = upload(g.arrays(), X)
    rng = np.random.default_rng(3)
    n = 257
    ks = rng.choice([1, 10, 100], n).astype(np.int32)
    efs = rng.integers(16, 300, n).astype(np.int32)
    Qd = dev(Q[:n])
    bi, bd = K.kann_search_batch(idx, Qd, dev(ks), dev(efs), kmax=100, efmax=300)
    torch.cuda.synchronize()
    bi, bd = bi.cpu().numpy(), bd.cpu().numpy()
    for q in range(0, n, 5):
        si, sd = search(idx, Q[q:q + 1], int(ks[q]), int(efs[q]))
        assert np.array_equal(bi[q, :ks[q]], si[0]) and np.array_equal(bd[q, :ks[q]], sd[0])
        assert np.all(bi[q, ks[q]:] == -1)


def test_hand_worked_golden_on_gpu():
    gold = load_golden("hand_search.json")
    for case in gold["cases"]:
        garr = golden_graph(case)
        X = np.zeros((len(case["x"]), 4), np.float32)
        X[:, 0] = case["x"]  # padded to 16 bytes per row; L2 unchanged
        q = np.zeros((1, 4), np.float32)
        q[0, 0] = case["q"]
        idx, _, _ = upload(garr, X)
        for run in case["runs"]:
            cnt = torch.zeros((1, 4), dtype=torch.int32, device="cuda")
            gi, gd = search(idx, q, run["k"], run["ef"], counters=cnt)
            assert gi[0].tolist() == run["ids"] and gd[0].tolist() == run["dists"]
            assert cnt.cpu().numpy()[0].tolist() == run["counters"]


@pytest.mark.parametrize("nq", [0, 1, 3, 5, 33])
def test_ragged_and_empty_batches(cfg1_small, nq):
    X, Q, g = cfg1_small
    idx, _, _ = upload(g.arrays(), X)
    if nq == 0:
        ids, d = K.kann_search(idx, torch.empty((0, 128), device="cuda"), 10, 64)
        assert ids.shape == (0, 10)
        return
    oi, _, _ = O.search_dense(g, X, Q[:nq], 10, 64, O.L2)
    gi, _ = search(idx, Q[:nq], 10, 64)
    assert id_set_match_fraction(gi, oi) == 1.0


def test_k_over_ef_padding_and_max_ef():
    gold = load_golden("hand_search.json")
    case = gold["cases"][1]
    garr = golden_graph(case)
    X = np.zeros((5, 4), np.float32)
    X[:, 0] = case["x"]
    q = np.zeros((1, 4), np.float32)
    q[0, 0] = case["q"]
    idx, _, _ = upload(garr, X)
    gi, gd = search(idx, q, 3, 1)
    assert gi[0].tolist() == [3, 2, 4]
    gi, gd = search(idx, q, 8, 1024)
    assert gi[0].tolist() == [3, 2, 4, 1, 0, -1, -1, -1] and np.all(np.isinf(gd[0, 5:]))
    with pytest.raises(K.KannError):
        search(idx, q, 8, 1025)


def test_duplicates_self_queries_and_nan():
    rng = np.random.default_rng(3)
    base = rng.standard_normal((60, 8)).astype(np.float32)
    X = np.concatenate([base, base[:10]])
    g = O.build_dense(X, O.L2, 6, 40, 9)
    idx, _, _ = upload(g.arrays(), X)
    gi, gd = search(idx, base[:10], 2, 70)
    assert gi[:, 0].tolist() == list(range(10)) and gi[:, 1].tolist() == list(range(60, 70))
    assert np.all(gd == 0.0)
    qn = np.full((2, 8), np.nan, np.float32)
    oi, _, _ = O.search_dense(g, X, qn, 5, 10, O.L2)
    gi, gd = search(idx, qn, 5, 10)
    assert np.array_equal(gi, oi) and np.all(np.isinf(gd))


def test_bad_ids_are_reported_not_followed(cfg1_small):
    X, Q, g = cfg1_small
    garr = g.arrays()
    garr["l0"] = garr["l0"].copy()
    # one edge in five points past the end of the index
    garr["l0"][garr["l0"] >= 0] = np.where(garr["l0"][garr["l0"] >= 0] % 5 == 0, 10**6,
                                          garr["l0"][garr["l0"] >= 0])
    with pytest.raises(K.KannError) as e:
        upload(garr, X)
    assert e.value.status == K.KANN_EFORMAT
    Xd = dev(X)
    idx = K.kann_index_upload(K.graph_to_device(garr), vectors=Xd, validate_ids=False)
    st = torch.zeros(50, dtype=torch.int32, device="cuda")
    gi, gd = search(idx, Q[:50], 10, 64, status=st)
    assert np.all((st.cpu().numpy() & K.KANN_QSTAT_BAD_ID) != 0)
    assert np.all((gi >= 0) & (gi < len(X)))


def test_hop_cap_sets_status(cfg1_small):
    X, Q, g = cfg1_small
    idx, _, _ = upload(g.arrays(), X)
    st = torch.zeros(20, dtype=torch.int32, device="cuda")
    gi, gd = search(idx, Q[:20], 10, 64, max_hops=3, status=st)
    assert np.all((st.cpu().numpy() & K.KANN_QSTAT_HOPCAP) != 0)
    assert np.all(gi[:, 0] >= 0)


# ------------------------------------------------------------------ exact k-NN
@pytest.mark.parametrize("metric", [K.KANN_L2, K.KANN_IP])
def test_exact_knn_matches_oracle(cfg1_small, metric):
    X, Q, _ = cfg1_small
    Qs = Q[:200]
    ei, ed = O.exact_dense(X, Qs, 10, metric)
    gi, gd = K.kann_exact_knn(dev(Qs), dev(X), 10, metric)
    torch.cuda.synchronize()
    gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
    assert id_set_match_fraction(gi, ei) >= 0.995
    check_dists(X, Qs, gi, gd, metric)


def test_exact_knn_integer_exact(int_small):
    X, Q, _ = int_small
    ei, ed = O.exact_dense(X, Q, 20, O.L2)
    gi, gd = K.kann_exact_knn(dev(Q), dev(X), 20, K.KANN_L2)
    torch.cuda.synchronize()
    assert np.array_equal(gi.cpu().numpy(), ei) and np.array_equal(gd.cpu().numpy().astype(np.float64), ed)



def test_bf16_rerank_copy(cfg1_small):
    X, Q, g = cfg1_small
    Xd = dev(X)
    Xb, _ = K.kann_quantize(Xd, K.KANN_BF16)
    Xh, _ = K.kann_quantize(Xd, K.KANN_F16)
    idx = K.kann_index_upload(K.graph_to_device(g.arrays()), vectors=Xh, dtype=K.KANN_F16, rerank=Xb)
    gi, gd = search(idx, Q, 10, 64, rerank=-1)
    th = Xh.cpu().view(torch.int16).numpy().view(np.uint16)
    tb = Xb.cpu().view(torch.int16).numpy().view(np.uint16)
    ti, _, _ = O.search_dense(g, th, Q, 64, 64, O.L2, dtype=O.DT_F16)
    oi, od = O.rerank_dense(tb, Q, ti, 10, O.L2, dtype=O.DT_BF16)
    assert id_set_match_fraction(gi, oi) >= 0.999
    check_dists(tb, Q, gi, gd, O.L2, dtype=O.DT_BF16)
