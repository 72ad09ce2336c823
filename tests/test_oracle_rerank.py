"""Pin of the oracle's re-rank (the exact re-ordering of a traversal's best
candidates on a full-precision copy, the precision mode's last step) against
an independent top-k: numpy FP64 distances of every candidate, ordered by
numpy's lexsort on (distance, id), -1 candidates skipped, the result padded
with -1 / +inf.  Integer-valued rows make every distance exact in FP64 in any
summation order, so ties between duplicate rows are real and must fall to the
lower id; a continuous case checks the order without ties."""
import numpy as np
import pytest

import oracle as O


def numpy_rerank(X, Q, cand, k, metric):
    X = X.astype(np.float64)
    Q = Q.astype(np.float64)
    ids = np.full((len(Q), k), -1, np.int64)
    dists = np.full((len(Q), k), np.inf)
    for qi in range(len(Q)):
        c = cand[qi][cand[qi] >= 0].astype(np.int64)
        if metric == O.L2:
            d = ((X[c] - Q[qi]) ** 2).sum(1)
        else:
            d = -(X[c] * Q[qi]).sum(1)
        order = np.lexsort((c, d))[:k]
        ids[qi, :len(order)] = c[order]
        dists[qi, :len(order)] = d[order]
    return ids, dists


def candidates(rng, n, nq, R, holes):
    cand = np.stack([rng.permutation(n)[:R] for _ in range(nq)]).astype(np.int32)
    if holes:
        cand[rng.random(cand.shape) < 0.2] = -1
        cand[0, :] = -1          # a query with no candidate at all
        cand[1, 3:] = -1         # fewer candidates than k
    return cand


@pytest.mark.parametrize("metric", [O.L2, O.IP])
@pytest.mark.parametrize("holes", [False, True])
def test_rerank_equals_numpy_lexsort_on_tied_integer_rows(metric, holes):
    rng = np.random.default_rng(7 + metric + 2 * holes)
    base = rng.integers(0, 4, (300, 16)).astype(np.float32)
    X = np.concatenate([base, base[::-1], base[:50]])   # many exact duplicates
    Q = rng.integers(0, 4, (40, 16)).astype(np.float32)
    cand = candidates(rng, len(X), len(Q), 120, holes)
    for k in (1, 10, 100):
        oi, od = O.rerank_dense(X, Q, cand, k, metric)
        ni, nd = numpy_rerank(X, Q, cand, k, metric)
        assert np.array_equal(oi, ni), k
        assert np.array_equal(od, nd), k


def test_rerank_continuous_rows_and_padding():
    rng = np.random.default_rng(11)
    X = rng.standard_normal((2000, 48)).astype(np.float32)
    Q = rng.standard_normal((30, 48)).astype(np.float32)
    cand = candidates(rng, len(X), len(Q), 64, True)
    oi, od = O.rerank_dense(X, Q, cand, 10, O.L2)
    ni, nd = numpy_rerank(X, Q, cand, 10, O.L2)
    assert np.array_equal(oi, ni)
    assert np.allclose(od[np.isfinite(nd)], nd[np.isfinite(nd)], rtol=1e-12, atol=0)
    assert np.all(oi[0] == -1) and np.all(np.isinf(od[0]))
    assert np.all(oi[1, 3:] == -1)


def test_rerank_of_stored_formats_decodes_them():
    # a BF16 copy: the oracle decodes the stored bits, numpy decodes them by
    # the format's definition (the high 16 bits of a binary32)
    rng = np.random.default_rng(13)
    X = (rng.standard_normal((500, 32)) * 3).astype(np.float32)
    Q = rng.standard_normal((20, 32)).astype(np.float32)
    xb = O.encode_bf16(X)
    Xdec = (xb.astype(np.uint32) << 16).view(np.float32)
    cand = candidates(rng, len(X), len(Q), 50, False)
    oi, od = O.rerank_dense(xb, Q, cand, 10, O.L2, dtype=O.DT_BF16)
    ni, nd = numpy_rerank(Xdec, Q, cand, 10, O.L2)
    assert np.array_equal(oi, ni)
    assert np.allclose(od, nd, rtol=1e-12, atol=0)


def test_distances_on_stored_fp16_and_e4m3_rows_decode_them():
    # the oracle's distances on FP16 and per-vector-scaled E4M3 rows against
    # numpy on rows decoded by the formats' definitions (numpy's float16,
    # torch's float8_e4m3fn, times the row's scale)
    import torch
    rng = np.random.default_rng(14)
    X = (rng.standard_normal((300, 32)) * 3).astype(np.float32)
    Q = rng.standard_normal((10, 32)).astype(np.float32)
    ids = np.tile(np.arange(300, dtype=np.int32), (len(Q), 1))
    h = X.astype(np.float16)
    got = O.dist_dense(h.view(np.uint16), Q, ids, O.L2, dtype=O.DT_F16)
    ref = ((Q.astype(np.float64)[:, None] - h.astype(np.float64)[None]) ** 2).sum(-1)
    assert np.allclose(got, ref, rtol=1e-12, atol=0)
    codes, sc = O.encode_e4m3_rows(X)
    dec = torch.from_numpy(codes).view(torch.float8_e4m3fn).double().numpy() * sc.astype(np.float64)[:, None]
    got = O.dist_dense(codes, Q, ids, O.IP, dtype=O.DT_E4M3, scale=sc)
    ref = -(Q.astype(np.float64) @ dec.T)
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-12)
