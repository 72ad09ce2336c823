"""Parity of the PQ (ADC) and sparse-IP search back-ends with the FP64 oracle
(kANNolo Sec. 2: PQ quantizer, citing Jegou et al.; Sec. 3 / Table 1: sparse
inner product).  Same contract as the dense path: >= 99.9% identical ID sets,
distances within 1e-5 * max(|d|, sum |terms|) of the oracle's FP64 value."""
import numpy as np
import pytest
import torch

import oracle as O
from helpers import id_set_match_fraction
from paper_2501_06121_b300 import datagen as G
from paper_2501_06121_b300 import kann as K

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def pq_setup():
    X, Q = G.vmf_mixture(6000, 1000, d=64, clusters=16, kappa=50.0, seed=41)
    g = O.build_dense(X, O.IP, 16, 100, 41)          # graph on the original vectors
    cb, _ = O.pq_train(X, m=16, ksub=256, iters=8, seed=41)
    codes = O.pq_encode(X, cb)
    return X, Q, g, cb, codes


def adc_mag(cb, codes, Q, ids, metric):
    out = np.zeros(ids.shape)
    m = cb.shape[0]
    for qi in range(len(Q)):
        lut = O.pq_lut(cb, Q[qi], metric)
        c = codes[np.maximum(ids[qi], 0)].astype(int)
        out[qi] = np.abs(lut[np.arange(m)[None, :], c]).sum(1)
    return out


@pytest.mark.parametrize("metric", [K.KANN_IP, K.KANN_L2])
def test_pq_parity(pq_setup, metric):
    X, Q, g, cb, codes = pq_setup
    idx = K.kann_index_upload(K.graph_to_device(g.arrays()),
                              pq=dict(codes=dev(codes), codebooks=dev(cb), metric=metric))
    oi, od, _ = O.search_pq(g, codes, cb, Q, 10, 64, metric)
    gi, gd = K.kann_search(idx, dev(Q), 10, 64)
    torch.cuda.synchronize()
    gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
    assert id_set_match_fraction(gi, oi) >= 0.999
    # every returned distance against the oracle's ADC value of that id
    ref = np.zeros(gi.shape)
    for qi in range(len(Q)):
        lut = O.pq_lut(cb, Q[qi], metric)
        ref[qi] = lut[np.arange(16)[None, :], codes[gi[qi]].astype(int)].sum(1)
    mag = adc_mag(cb, codes, Q, gi, metric)
    assert np.all(np.abs(gd - ref) <= 1e-5 * np.maximum(np.abs(ref), mag) + 1e-30)


@pytest.mark.parametrize("metric", [K.KANN_IP, K.KANN_L2])
def test_pq_fp16_table_parity(pq_setup, metric):
    # the FP16 table (power-of-two scale, entries rounded to nearest) against
    # the oracle's search with the same reading of the table
    X, Q, g, cb, codes = pq_setup
    idx = K.kann_index_upload(K.graph_to_device(g.arrays()),
                              pq=dict(codes=dev(codes), codebooks=dev(cb), metric=metric))
    oi, od, _ = O.search_pq(g, codes, cb, Q, 10, 64, metric, lut_f16=True)
    gi, gd = K.kann_search_ex(idx, dev(Q), 10, 64, pq_lut_f16=1)
    torch.cuda.synchronize()
    gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
    assert id_set_match_fraction(gi, oi) >= 0.999
    ref = np.zeros(gi.shape)
    mag = np.zeros(gi.shape)
    for qi in range(len(Q)):
        lut = O.pq_lut(cb, Q[qi], metric, lut_f16=True)
        terms = lut[np.arange(16)[None, :], codes[gi[qi]].astype(int)]
        ref[qi] = terms.sum(1)
        mag[qi] = np.abs(terms).sum(1)
    # FP32 arithmetic as in the FP32-table contract, plus: the GPU rounds its
    # FP32 entry and the oracle its FP64 entry to FP16, so an entry that lies
    # next to a rounding boundary may land one FP16 step (2^-10 relative, or
    # 2^-9 if the scale's power of two flips too) away
    tol = 1e-5 * np.maximum(np.abs(ref), mag) + 2.0 ** -9 * mag + 1e-30
    assert np.all(np.abs(gd - ref) <= tol)
    assert np.mean(np.abs(gd - ref) <= 1e-5 * np.maximum(np.abs(ref), mag) + 1e-30) >= 0.99
    # and the search it drives stays close to the FP32-table search
    fi, _ = K.kann_search(idx, dev(Q), 10, 64)
    torch.cuda.synchronize()
    assert id_set_match_fraction(gi, fi.cpu().numpy()) >= 0.95


def test_pq_rerank(pq_setup):
    X, Q, g, cb, codes = pq_setup
    Xd = dev(X)
    idx = K.kann_index_upload(K.graph_to_device(g.arrays()), pq=dict(codes=dev(codes), codebooks=dev(cb),
                                                                     metric=K.KANN_IP), rerank=Xd)
    ti, _, _ = O.search_pq(g, codes, cb, Q, 100, 100, O.IP)
    oi, od = O.rerank_dense(X, Q, ti, 10, O.IP)
    gi, gd = K.kann_search_ex(idx, dev(Q), 10, 100, rerank=100)
    torch.cuda.synchronize()
    gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
    assert id_set_match_fraction(gi, oi) >= 0.999
    ref = O.dist_dense(X, Q, gi, O.IP)
    mag = np.einsum("qd,qkd->qk", np.abs(Q.astype(np.float64)), np.abs(X.astype(np.float64)[gi]))
    assert np.all(np.abs(gd - ref) <= 1e-5 * np.maximum(np.abs(ref), mag))


def test_pq_m32_and_exact_special_case():
    # m = 32 subspaces of 2 dims with <= 256 distinct sub-vectors: PQ is exact,
    # so the PQ search equals the plain FP32 search
    rng = np.random.default_rng(5)
    m, dsub = 32, 2
    protos = rng.integers(-5, 6, size=(m, 200, dsub)).astype(np.float32)
    pick = rng.integers(0, 200, size=(3000, m))
    X = np.concatenate([protos[j][pick[:, j]] for j in range(m)], axis=1)
    Q = rng.standard_normal((300, m * dsub)).astype(np.float32) * 3
    g = O.build_dense(X, O.L2, 12, 80, 6)
    cb = np.zeros((m, 256, dsub), np.float32)
    cb[:, :200] = protos
    cb[:, 200:] = 1000.0
    codes = O.pq_encode(X, cb)
    assert np.array_equal(O.pq_reconstruct(codes, cb), X)
    idx = K.kann_index_upload(K.graph_to_device(g.arrays()), pq=dict(codes=dev(codes), codebooks=dev(cb),
                                                                     metric=K.KANN_L2))
    gi, gd = K.kann_search(idx, dev(Q), 10, 64)
    torch.cuda.synchronize()
    oi, od, _ = O.search_dense(g, X, Q, 10, 64, O.L2)
    assert id_set_match_fraction(gi.cpu().numpy(), oi) >= 0.99


@pytest.fixture(scope="module")
def sparse_setup():
    base, qs = G.sparse_zipf(4000, 1000, vocab=3000, lam_doc=40, lam_query=12, seed=51)
    g = O.build_sparse(*base, M=16, efC=100, seed=51)
    return base, qs, g


def sparse_index(g, base, vocab):
    sp = dict(indptr=dev(base[0]), terms=dev(base[1].view(np.int16)), weights=dev(base[2]), vocab=vocab)
    return K.kann_index_upload(K.graph_to_device(g.arrays()), sparse=sp)


def test_sparse_parity(sparse_setup):
    base, qs, g = sparse_setup
    idx = sparse_index(g, base, 3000)
    for ef in (32, 128):
        oi, od, _ = O.search_sparse(g, base, qs, 10, ef)
        gi, gd = K.kann_search_sparse(idx, dev(qs[0]), dev(qs[1].view(np.int16)), dev(qs[2]), 10, ef)
        torch.cuda.synchronize()
        gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
        assert id_set_match_fraction(gi, oi) >= 0.999
        Xd = G.densify(base, 3000).astype(np.float64)
        Qd = G.densify(qs, 3000).astype(np.float64)
        ref = -np.einsum("qd,qkd->qk", Qd, Xd[gi])
        mag = np.einsum("qd,qkd->qk", np.abs(Qd), np.abs(Xd[gi]))
        assert np.all(np.abs(gd - ref) <= 1e-5 * np.maximum(np.abs(ref), mag) + 1e-30)


def test_sparse_long_query_is_flagged(sparse_setup):
    base, _, g = sparse_setup
    idx = sparse_index(g, base, 3000)
    terms = np.arange(0, 3000, 5, dtype=np.uint16)[:600]
    qi = np.array([0, len(terms)], np.int64)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    gi, gd = K.kann_search_sparse(idx, dev(qi), dev(terms.view(np.int16)), dev(np.ones(len(terms), np.float32)),
                                  10, 32, status=st)
    torch.cuda.synchronize()
    assert (st.cpu().numpy()[0] & K.KANN_QSTAT_QUERY_TRUNCATED) != 0
    assert np.all(gi.cpu().numpy() >= 0)


def test_device_pq_encode_matches_oracle_on_integer_data():
    # integer data and codebooks: every FP32 distance is exact, so the nearest
    # centroid (ties to the lowest index) is the same decision on both sides
    rng = np.random.default_rng(9)
    X = rng.integers(0, 16, (3000, 64)).astype(np.float32)
    cb = rng.integers(0, 16, (16, 256, 4)).astype(np.float32)
    codes = K.kann_pq_encode(dev(X), dev(cb))
    torch.cuda.synchronize()
    assert np.array_equal(codes.cpu().numpy(), O.pq_encode(X, cb))


@pytest.mark.parametrize("iters", [0, 1, 6])
def test_device_pq_training_equals_oracle_on_integer_data(iters):
    # integer data: every distance, running sum and mean decision is exact on
    # both sides, so k-means++ seeding and the Lloyd iterations give the
    # oracle's codebooks bit for bit (empty clusters included: 256 centroids
    # over a few thousand points with many repeats)
    rng = np.random.default_rng(13 + iters)
    X = rng.integers(0, 16, (3000, 32)).astype(np.float32)
    X[:400] = X[400:800]  # repeated rows make clusters empty
    cb = K.kann_pq_train(dev(X), 8, iters=iters, seed=7)
    torch.cuda.synchronize()
    ocb, obj = O.pq_train(X, m=8, ksub=256, iters=iters, seed=7)
    assert np.array_equal(cb.cpu().numpy(), ocb)


def test_device_pq_training_real_data_close_to_oracle():
    # real-valued data: the same steps; parallel FP64 sums may round apart, so
    # the quantisation error is compared, within 2%
    X, _ = G.vmf_mixture(20000, 1, d=64, clusters=16, kappa=50.0, seed=61)
    cb = K.kann_pq_train(dev(X), 16, iters=10, seed=3)
    torch.cuda.synchronize()
    ocb, obj = O.pq_train(X, m=16, ksub=256, iters=10, seed=3)
    err = lambda c: float(np.mean((O.pq_reconstruct(O.pq_encode(X, c), c) - X) ** 2))
    assert abs(err(cb.cpu().numpy()) - err(ocb)) <= 0.02 * err(ocb)


def test_sparse_exact_knn_matches_oracle():
    base, qs = G.sparse_zipf(5000, 200, vocab=3000, lam_doc=40, lam_query=12, seed=71)
    td = lambda c: (dev(c[0]), dev(c[1].view(np.int16)), dev(c[2]))
    gi, gd = K.kann_exact_knn_sparse(td(base), td(qs), 3000, 20)
    torch.cuda.synchronize()
    gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
    oi, od = O.exact_sparse(base, qs, 20)
    assert id_set_match_fraction(gi, oi) >= 0.99
    Xd = G.densify(base, 3000).astype(np.float64)
    Qd = G.densify(qs, 3000).astype(np.float64)
    ref = -np.einsum("qd,qkd->qk", Qd, Xd[gi])
    mag = np.einsum("qd,qkd->qk", np.abs(Qd), np.abs(Xd[gi]))
    assert np.all(np.abs(gd - ref) <= 1e-5 * np.maximum(np.abs(ref), mag) + 1e-30)
    assert np.all(np.diff(gd, axis=1) >= 0)


@pytest.mark.parametrize("metric", [K.KANN_IP, K.KANN_L2])
def test_pq_u8_table_bit_exact(pq_setup, metric):
    # the uint8 table: both sides build it with the same FP32 operations and
    # order rows by exact integer sums, so ids, work and the reported
    # distances (summin + scale * sum, two FP32 roundings) are identical
    X, Q, g, cb, codes = pq_setup
    idx = K.kann_index_upload(K.graph_to_device(g.arrays()),
                              pq=dict(codes=dev(codes), codebooks=dev(cb), metric=metric))
    for ef in (16, 64, 200):
        oi, od, oc = O.search_pq(g, codes, cb, Q, 10, ef, metric, lut=O.LUT_U8)
        cnt = torch.zeros((len(Q), 4), dtype=torch.int32, device="cuda")
        gi, gd = K.kann_search_ex(idx, dev(Q), 10, ef, pq_lut=K.KANN_PQ_LUT_U8, counters=cnt, hash_bits=15)
        torch.cuda.synchronize()
        gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
        assert np.array_equal(gi, oi), ef
        assert np.array_equal(cnt.cpu().numpy().astype(np.int64), oc), ef
        want = np.empty(gd.shape, np.float32)
        for qi in range(len(Q)):
            _, sc, sm = O.pq_lut_u8(cb, Q[qi], metric)
            want[qi] = np.float32(sm) + np.float32(sc) * od[qi].astype(np.float32)
        assert np.array_equal(gd, want), ef
