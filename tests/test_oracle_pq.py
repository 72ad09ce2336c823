"""Pins for the oracle's Product Quantization (Jegou et al., the quantizer of
kANNolo Sec. 2): ADC identities, the exact special case, k-means descent,
nearest-centroid encoding."""
import numpy as np
import pytest

import oracle as O


def _data(n=3000, d=16, seed=0):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, d)).astype(np.float32), rng.standard_normal((20, d)).astype(np.float32)


def test_kmeans_objective_never_increases():
    X, _ = _data()
    cb, obj = O.pq_train(X, m=4, ksub=16, iters=10, seed=1)
    assert cb.shape == (4, 16, 4)
    assert np.all(np.diff(obj, axis=1) <= 1e-12 * np.abs(obj[:, :-1]))


def test_adc_equals_exact_distance_to_reconstruction():
    X, Q = _data()
    for metric in (O.L2, O.IP):
        cb, _ = O.pq_train(X, m=4, ksub=16, iters=5, seed=2)
        codes = O.pq_encode(X, cb)
        R = O.pq_reconstruct(codes, cb)
        ids = np.tile(np.arange(50, dtype=np.int32), (len(Q), 1))
        exact = O.dist_dense(R, Q, ids, metric)
        # ADC: per-query table, then a sum of lookups
        adc = np.zeros_like(exact)
        for qi, q in enumerate(Q):
            lut = O.pq_lut(cb, q, metric)
            adc[qi] = lut[np.arange(4)[None, :], codes[:50].astype(int)].sum(1)
        # same value up to the order of the FP64 sums
        assert np.allclose(adc, exact, rtol=1e-12, atol=1e-12)
        # and against numpy on the reconstructed vectors
        R64, Q64 = R.astype(np.float64)[:50], Q.astype(np.float64)
        ref = ((Q64[:, None] - R64[None]) ** 2).sum(-1) if metric == O.L2 else -(Q64 @ R64.T)
        assert np.allclose(adc, ref, rtol=1e-12, atol=1e-12)


def test_pq_is_exact_when_every_subvector_is_a_centroid():
    # 8 distinct sub-vectors per subspace and 16 centroids: k-means places a
    # centroid on each, codes reconstruct exactly, ADC equals the true distance
    rng = np.random.default_rng(3)
    m, dsub = 4, 2
    protos = rng.integers(-5, 6, size=(m, 8, dsub)).astype(np.float32)
    pick = rng.integers(0, 8, size=(600, m))
    X = np.concatenate([protos[j][pick[:, j]] for j in range(m)], axis=1)
    cb, obj = O.pq_train(X, m=m, ksub=16, iters=10, seed=4)
    assert np.all(obj[:, -1] == 0.0)
    codes = O.pq_encode(X, cb)
    assert np.array_equal(O.pq_reconstruct(codes, cb), X)
    Q = rng.standard_normal((30, m * dsub)).astype(np.float32)
    g = O.build_dense(X, O.L2, 8, 60, 5)
    a = O.search_pq(g, codes, cb, Q, 10, 50, O.L2)
    b = O.search_dense(g, X, Q, 10, 50, O.L2)
    assert np.array_equal(a[0], b[0]) and np.allclose(a[1], b[1], rtol=1e-12, atol=1e-12)
    e = O.exact_pq(codes, cb, Q, 10, O.L2)
    f = O.exact_dense(X, Q, 10, O.L2)
    assert np.array_equal(e[0], f[0])


def test_encode_picks_nearest_and_lowest_on_ties():
    cb = np.zeros((1, 4, 2), np.float32)
    cb[0, 0] = [1, 0]
    cb[0, 1] = [0, 1]
    cb[0, 2] = [1, 0]   # duplicate of centroid 0
    cb[0, 3] = [5, 5]
    X = np.array([[1, 0], [0, 1], [0.9, 0.1], [4, 4], [0.5, 0.5]], np.float32)
    codes = O.pq_encode(X, cb)
    # [0.5, 0.5] is equidistant from centroids 0, 1 and 2 -> lowest index
    assert codes[:, 0].tolist() == [0, 1, 0, 3, 0]


def test_fp16_table_is_the_scaled_half_rounding_of_the_fp64_table():
    # independent restatement with numpy: scale by the power of two that puts
    # the largest |entry| in [2^14, 2^15), round to float16 (nearest, ties to
    # even), scale back
    X, Q = _data(d=32, seed=7)
    for metric in (O.L2, O.IP):
        cb, _ = O.pq_train(X, m=8, ksub=64, iters=4, seed=8)
        for q in Q[:6]:
            t64 = O.pq_lut(cb, q, metric)
            t16 = O.pq_lut(cb, q, metric, lut_f16=True)
            mx = np.abs(t64).max()
            e = int(np.floor(np.log2(mx))) + 1 - 15
            ref = np.ldexp(np.ldexp(t64, -e).astype(np.float16).astype(np.float64), e)
            assert np.array_equal(t16, ref)
            assert 2.0 ** 14 <= np.abs(np.ldexp(t16, -e)).max() <= 2.0 ** 15
            # half-ulp bound of the rounding
            assert np.all(np.abs(t16 - t64) <= np.maximum(2.0 ** -11 * np.abs(t64), 2.0 ** (e - 25)))


def test_fp16_table_is_exact_on_small_integer_tables():
    # entries are small integers (after the exact power-of-two scaling they
    # still have at most 11 significant bits): the FP16 table loses nothing,
    # so the search equals the FP64-table search
    rng = np.random.default_rng(9)
    m, dsub = 4, 2
    X = rng.integers(-6, 7, size=(800, m * dsub)).astype(np.float32)
    cb, _ = O.pq_train(X, m=m, ksub=16, iters=6, seed=9)
    cb = np.round(cb).astype(np.float32)
    codes = O.pq_encode(X, cb)
    Q = rng.integers(-6, 7, size=(25, m * dsub)).astype(np.float32)
    for metric in (O.L2, O.IP):
        for q in Q[:5]:
            assert np.array_equal(O.pq_lut(cb, q, metric, lut_f16=True), O.pq_lut(cb, q, metric))
        g = O.build_dense(X, metric, 8, 60, 10)
        a = O.search_pq(g, codes, cb, Q, 10, 40, metric, lut_f16=True)
        b = O.search_pq(g, codes, cb, Q, 10, 40, metric)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


# ------------------------------------------------------------------ the uint8 table reading
def _numpy_u8_table(cb, q, metric):
    """The uint8 reading written out with numpy float32 for dsub = 1 (each
    entry is then one correctly rounded FP32 product, as fmaf gives it)."""
    m, ksub, dsub = cb.shape
    assert dsub == 1
    c = cb[:, :, 0].astype(np.float32)
    qq = q.astype(np.float32).reshape(m, 1)
    if metric == O.L2:
        u = qq - c
        e = u * u
    else:
        e = -(qq * c)
    mn = e.min(1)
    rng = e.max(1) - mn
    rmax = np.float32(rng.max())
    scale = np.float32(rmax / np.float32(255.0)) if rmax > 0 else np.float32(1.0)
    r = np.clip((e - mn[:, None]) / scale, np.float32(0), np.float32(255))
    v = np.rint(r).astype(np.uint8)
    summin = np.float32(0)
    for x in mn:
        summin = np.float32(summin + x)
    return v, scale, summin


@pytest.mark.parametrize("metric", [O.L2, O.IP])
def test_u8_table_equals_its_definition_written_in_numpy(metric):
    rng = np.random.default_rng(17)
    cb = (rng.standard_normal((32, 256, 1)) * 3).astype(np.float32)
    for _ in range(5):
        q = rng.standard_normal(32).astype(np.float32) * 2
        v, sc, sm = O.pq_lut_u8(cb, q, metric)
        nv, nsc, nsm = _numpy_u8_table(cb, q, metric)
        assert np.array_equal(v, nv) and sc == nsc and sm == nsm
        assert v.min(1).max() == 0 and v.max() == 255  # each subspace's minimum -> 0, the widest reaches 255


def test_u8_table_is_exact_on_integer_entries_spanning_255():
    # IP with q = 1 and codebook values -255..0 (both ends present in every
    # subspace): entries are the integers 0..255, so scale = 1, the minima are
    # 0 and the uint8 search is the exact ADC search
    rng = np.random.default_rng(19)
    m = 16
    cb = -rng.integers(0, 256, (m, 256, 1)).astype(np.float32)
    cb[:, 0, 0], cb[:, 1, 0] = 0.0, -255.0
    X = rng.standard_normal((2500, m)).astype(np.float32)
    codes = rng.integers(0, 256, (2500, m)).astype(np.uint8)
    Q = np.ones((40, m), np.float32)
    v, sc, sm = O.pq_lut_u8(cb, Q[0], O.IP)
    assert sc == 1.0 and sm == 0.0
    g = O.build_dense(X, O.L2, 10, 50, 19)
    a = O.search_pq(g, codes, cb, Q, 10, 64, O.IP)
    b = O.search_pq(g, codes, cb, Q, 10, 64, O.IP, lut=O.LUT_U8)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


@pytest.mark.parametrize("metric", [O.L2, O.IP])
def test_u8_distance_within_half_a_step_per_subspace(metric):
    # summin + scale * sum differs from the exact ADC distance by at most
    # m * scale / 2 (each value rounds to the nearest step) plus the FP32
    # rounding of the entries
    rng = np.random.default_rng(23)
    m, dsub = 24, 4
    cb = rng.standard_normal((m, 256, dsub)).astype(np.float32)
    codes = rng.integers(0, 256, (500, m)).astype(np.uint8)
    for _ in range(5):
        q = rng.standard_normal(m * dsub).astype(np.float32)
        v, sc, sm = O.pq_lut_u8(cb, q, metric)
        exact = O.pq_lut(cb, q, metric)
        S = v[np.arange(m)[None, :], codes].astype(np.float64).sum(1)
        approx = np.float64(sm) + np.float64(sc) * S
        ref = exact[np.arange(m)[None, :], codes].sum(1)
        mag = np.abs(exact[np.arange(m)[None, :], codes]).sum(1)
        assert np.all(np.abs(approx - ref) <= m * sc / 2 * (1 + 1e-5) + 1e-5 * mag)
