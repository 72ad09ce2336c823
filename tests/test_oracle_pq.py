"""Pins for the oracle's Product Quantization (Jegou et al., the quantizer of
kANNolo Sec. 2): ADC identities, the exact special case, k-means descent,
nearest-centroid encoding."""
import numpy as np

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
