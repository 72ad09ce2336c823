"""Parity with the FP64 oracle on the code paths the full-size workloads take.

The 1M x 768 inner-product workload (the MS MARCO Star/Dragon stand-in of the
paper's Sec. 3, Table 1: HNSW built on the original vectors, searched with PQ
codes, Sec. 2 and 3.1) runs the PQ back-end at m = 192 subspaces of 4 dims:
12 chunks of 16 code bytes per row, 8 lanes per row and 2 chunks per lane with
a bounds check on the second, a 192 KB FP32 table (96 KB in FP16) at the
opt-in shared-memory limit, and a re-rank of 100 candidates on 3 KB FP32 rows
(32 lanes per row, 6 chunks each).  Its plain FP32 arm runs the general dense
kernel with 8 chunks per lane.  At ef up to 1,024 the beam holds up to 1,024
keys, and a PQ search at m = 192 then gives up visited-table bits to fit its
table.  Each of these paths is checked here at small n, with the same contract
as the other parity tests: >= 99.9% identical ID sets and distances within
1e-5 * max(|d|, sum |terms|) of the oracle's FP64 value (FP32 arithmetic on
both table formats' entries as the oracle rounds them)."""
import numpy as np
import pytest
import torch

import oracle as O
from helpers import id_set_match_fraction
from paper_2501_06121_b300 import datagen as G
from paper_2501_06121_b300 import kann as K

pytestmark = pytest.mark.gpu

M192, DSUB = 192, 4


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def set768():
    """6,000 x 768 unit vectors (16 directions, normalize(mu + 0.04 g)), 400
    queries, IP, HNSW M = 16 built by the oracle on the FP32 vectors; PQ
    m = 192 x 256 with codebooks of 256 distinct training sub-vectors per
    subspace drawn by a seeded generator (the search's parity does not depend
    on how the codebooks were chosen) and codes from the oracle's encoder."""
    X, Q = G.vmf_mixture(6000, 400, d=768, clusters=16, kappa=50.0, seed=81, concentration=0.04)
    g = O.build_dense(X, O.IP, 16, 64, 81)
    rng = np.random.default_rng(81)
    cb = np.empty((M192, 256, DSUB), np.float32)
    for j in range(M192):
        cb[j] = X[rng.permutation(len(X))[:256], j * DSUB:(j + 1) * DSUB]
    codes = O.pq_encode(X, cb)
    return X, Q, g, cb, codes


def pq_index(g, cb, codes, metric, rerank=None):
    return K.kann_index_upload(K.graph_to_device(g.arrays()), pq=dict(codes=dev(codes), codebooks=dev(cb),
                                                                      metric=metric), rerank=rerank)


def check_adc(cb, codes, Q, gi, gd, metric, lut_f16=False):
    """Each returned ADC distance against the oracle's table sum for that id."""
    ref = np.zeros(gi.shape)
    mag = np.zeros(gi.shape)
    for qi in range(len(Q)):
        lut = O.pq_lut(cb, Q[qi], metric, lut_f16=lut_f16)
        terms = lut[np.arange(M192)[None, :], codes[np.maximum(gi[qi], 0)].astype(int)]
        ref[qi] = terms.sum(1)
        mag[qi] = np.abs(terms).sum(1)
    tol = 1e-5 * np.maximum(np.abs(ref), mag) + 1e-30
    if lut_f16:
        # the GPU rounds its FP32 entry and the oracle its FP64 entry: an entry
        # on an FP16 rounding boundary may land one step (2^-10, or 2^-9 with
        # the scale) apart
        assert np.mean(np.abs(gd - ref) <= tol) >= 0.99
        tol = tol + 2.0 ** -9 * mag
    assert np.all(np.abs(gd - ref) <= tol)


def check_ip(X, Q, gi, gd):
    ref = O.dist_dense(X, Q, np.maximum(gi, 0), O.IP)
    mag = np.einsum("qd,qkd->qk", np.abs(Q.astype(np.float64)), np.abs(X.astype(np.float64)[np.maximum(gi, 0)]))
    ok = gi >= 0
    assert np.all(np.abs(gd - ref)[ok] <= 1e-5 * np.maximum(np.abs(ref), mag)[ok])


@pytest.mark.parametrize("ef", [128, 1000])
@pytest.mark.parametrize("lut_f16", [False, True])
def test_pq_m192_parity(set768, ef, lut_f16):
    X, Q, g, cb, codes = set768
    idx = pq_index(g, cb, codes, K.KANN_IP)
    oi, od, oc = O.search_pq(g, codes, cb, Q, 10, ef, O.IP, lut_f16=lut_f16)
    gi, gd = K.kann_search_ex(idx, dev(Q), 10, ef, pq_lut_f16=int(lut_f16))
    torch.cuda.synchronize()
    gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
    assert id_set_match_fraction(gi, oi) >= 0.999
    check_adc(cb, codes, Q, gi, gd, O.IP, lut_f16)


@pytest.mark.parametrize("ef", [128, 1000])
def test_pq_m192_u8_table_bit_exact(set768, ef):
    # the uint8 table at m = 192 (48 KB, four teams per SM): identical
    # integer decisions on both sides
    X, Q, g, cb, codes = set768
    idx = pq_index(g, cb, codes, K.KANN_IP)
    oi, od, oc = O.search_pq(g, codes, cb, Q, 10, ef, O.IP, lut=O.LUT_U8)
    cnt = torch.zeros((len(Q), 4), dtype=torch.int32, device="cuda")
    gi, gd = K.kann_search_ex(idx, dev(Q), 10, ef, pq_lut=K.KANN_PQ_LUT_U8, counters=cnt, hash_bits=14)
    torch.cuda.synchronize()
    assert np.array_equal(gi.cpu().numpy(), oi)
    assert np.array_equal(cnt.cpu().numpy().astype(np.int64), oc)


@pytest.mark.parametrize("k", [10, 100])
def test_pq_m192_u8_table_rerank100(set768, k):
    X, Q, g, cb, codes = set768
    idx = pq_index(g, cb, codes, K.KANN_IP, rerank=dev(X))
    ti, _, _ = O.search_pq(g, codes, cb, Q, 128, 128, O.IP, lut=O.LUT_U8)
    oi, od = O.rerank_dense(X, Q, ti[:, :100], k, O.IP)
    gi, gd = K.kann_search_ex(idx, dev(Q), k, 128, rerank=100, pq_lut=K.KANN_PQ_LUT_U8)
    torch.cuda.synchronize()
    gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
    assert id_set_match_fraction(gi, oi) >= 0.999
    check_ip(X, Q, gi, gd)


def test_pq_m192_l2_parity(set768):
    X, Q, g, cb, codes = set768
    idx = pq_index(g, cb, codes, K.KANN_L2)
    oi, od, _ = O.search_pq(g, codes, cb, Q, 10, 96, O.L2)
    gi, gd = K.kann_search(idx, dev(Q), 10, 96)
    torch.cuda.synchronize()
    gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
    assert id_set_match_fraction(gi, oi) >= 0.999
    check_adc(cb, codes, Q, gi, gd, O.L2)


@pytest.mark.parametrize("k", [10, 100])
@pytest.mark.parametrize("lut_f16", [False, True])
def test_pq_m192_rerank100_on_fp32_rows(set768, k, lut_f16):
    # ADC traversal at ef = 128, then the best 100 of W re-ranked exactly on
    # the 768-d FP32 copy (32 lanes per row, 6 chunks per lane)
    X, Q, g, cb, codes = set768
    idx = pq_index(g, cb, codes, K.KANN_IP, rerank=dev(X))
    ti, _, _ = O.search_pq(g, codes, cb, Q, 128, 128, O.IP, lut_f16=lut_f16)
    oi, od = O.rerank_dense(X, Q, ti[:, :100], k, O.IP)
    gi, gd = K.kann_search_ex(idx, dev(Q), k, 128, rerank=100, pq_lut_f16=int(lut_f16))
    torch.cuda.synchronize()
    gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
    assert id_set_match_fraction(gi, oi) >= 0.999
    check_ip(X, Q, gi, gd)


@pytest.mark.parametrize("fmt,hb", [(K.KANN_VISITED_WIDE, 0), (K.KANN_VISITED_COMPACT, 16)])
def test_pq_m192_ef1024_shrinks_the_visited_table_and_keeps_parity(set768, fmt, hb):
    # FP32 table 192 KB + beam 8 KB + candidates + a visited table of 2^13
    # wide (32 KB) or 2^16 compact (128 KB) slots exceed one CTA: the search
    # runs with fewer table bits, which only makes it forget visited ids
    # (parity-safe)
    X, Q, g, cb, codes = set768
    idx = pq_index(g, cb, codes, K.KANN_IP)
    assert K.kann_search_workspace_bytes(idx, len(Q), 10, 1024, visited_format=fmt, hash_bits=hb) > 0
    st = torch.zeros(len(Q), dtype=torch.int32, device="cuda")
    oi, od, _ = O.search_pq(g, codes, cb, Q, 10, 1024, O.IP)
    gi, gd = K.kann_search_ex(idx, dev(Q), 10, 1024, status=st, visited_format=fmt, hash_bits=hb)
    torch.cuda.synchronize()
    gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
    assert id_set_match_fraction(gi, oi) >= 0.999
    check_adc(cb, codes, Q, gi, gd, O.IP)


@pytest.mark.parametrize("ef", [64, 1024])
def test_dense_768_fp32_ip_general_kernel(set768, ef):
    # 192 chunks per row: 32 lanes per row, 6 chunks per lane -> the general
    # kernel with 8 chunks per lane and its chunk-bounds checks
    X, Q, g, _, _ = set768
    idx = K.kann_index_upload(K.graph_to_device(g.arrays()), vectors=dev(X), dtype=K.KANN_F32, metric=K.KANN_IP)
    oi, od, _ = O.search_dense(g, X, Q, 10, ef, O.IP)
    gi, gd = K.kann_search(idx, dev(Q), 10, ef)
    torch.cuda.synchronize()
    gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
    assert id_set_match_fraction(gi, oi) >= 0.999
    check_ip(X, Q, gi, gd)


@pytest.mark.parametrize("dtype", [K.KANN_F32, K.KANN_F16])
@pytest.mark.parametrize("ef", [768, 1024])
def test_dense_large_ef_integer_bit_exact(int_small, dtype, ef):
    # a 20,000-node graph, beam of up to 1,024 keys and a 2^13-slot table; on
    # integer data the results equal the oracle's bit for bit
    X, Q, g = int_small
    Xd = dev(X)
    data = Xd if dtype == K.KANN_F32 else K.kann_quantize(Xd, dtype)[0]
    idx = K.kann_index_upload(K.graph_to_device(g.arrays()), vectors=data, dtype=dtype)
    Qs = Q[:120]
    oi, od, _ = O.search_dense(g, X, Qs, 10, ef, O.L2)
    gi, gd = K.kann_search(idx, dev(Qs), 10, ef)
    torch.cuda.synchronize()
    assert np.array_equal(gi.cpu().numpy(), oi)
    assert np.array_equal(gd.cpu().numpy().astype(np.float64), od)


def test_dense_large_ef_with_rerank_all(int_small):
    # FP16 traversal at ef = 1,000 and a re-rank of all 1,000 candidates
    X, Q, g = int_small
    Xd = dev(X)
    idx = K.kann_index_upload(K.graph_to_device(g.arrays()), vectors=K.kann_quantize(Xd, K.KANN_F16)[0],
                              dtype=K.KANN_F16, rerank=Xd)
    Qs = Q[:60]
    ti, _, _ = O.search_dense(g, X, Qs, 1000, 1000, O.L2)
    oi, od = O.rerank_dense(X, Qs, ti, 10, O.L2)
    gi, gd = K.kann_search_ex(idx, dev(Qs), 10, 1000, rerank=-1)
    torch.cuda.synchronize()
    assert np.array_equal(gi.cpu().numpy(), oi)
    assert np.array_equal(gd.cpu().numpy().astype(np.float64), od)


# ------------------------------------------------------------------ admission agrees with the search
def _runs(fn):
    try:
        fn()
        torch.cuda.synchronize()
        return True
    except K.KannError:
        return False


def test_workspace_bytes_is_positive_exactly_when_the_search_runs():
    # PQ at m = 384 (d = 384, dsub = 1): the FP32 table (384 KB) never fits a
    # CTA, the FP16 table (192 KB) does at small ef and stops fitting as the
    # beam grows; m = 192 fits in both formats at every ef
    rng = np.random.default_rng(3)
    n = 2000
    X = rng.standard_normal((n, 384)).astype(np.float32)
    g = O.build_dense(X[:, :16], O.L2, 8, 40, 3)
    Q = dev(rng.standard_normal((8, 384)).astype(np.float32))
    for m, dsub in ((384, 1), (192, 2)):
        cb = np.ascontiguousarray(rng.standard_normal((m, 256, dsub)).astype(np.float32))
        codes = rng.integers(0, 256, (n, m)).astype(np.uint8)
        idx = pq_index(g, cb, codes, K.KANN_L2)
        seen = set()
        for lut in (K.KANN_PQ_LUT_F32, K.KANN_PQ_LUT_F16, K.KANN_PQ_LUT_U8):
            for efmax in (16, 64, 256, 512, 1024, 1025):
                ws = K.kann_search_workspace_bytes(idx, 8, 10, efmax, pq_lut=lut)
                ran = _runs(lambda: K.kann_search_ex(idx, Q, 10, efmax, pq_lut=lut))
                assert (ws > 0) == ran, (m, lut, efmax, ws)
                seen.add(ran)
        if m == 384:
            assert seen == {True, False}
    # dense: refused exactly when ef_eff exceeds the build's maximum
    Xd = dev(X[:, :128].copy())
    idx = K.kann_index_upload(K.graph_to_device(g.arrays()), vectors=Xd)
    for efmax in (16, 1024, 1025):
        ws = K.kann_search_workspace_bytes(idx, 8, 10, efmax)
        assert (ws > 0) == _runs(lambda: K.kann_search(idx, dev(np.zeros((8, 128), np.float32)), 10, efmax))
