"""The seeded generators: determinism and the stated laws."""
import numpy as np

from paper_2501_06121_b300 import datagen as G


def test_gaussian_mixture_deterministic_and_shaped():
    a, qa = G.gaussian_mixture(2000, 50, seed=1)
    b, qb = G.gaussian_mixture(2000, 50, seed=1)
    assert a.shape == (2000, 128) and qa.shape == (50, 128) and a.dtype == np.float32
    assert np.array_equal(a, b) and np.array_equal(qa, qb)
    assert not np.array_equal(G.gaussian_mixture(2000, 50, seed=2)[0], a)


def test_integer_mixture_values():
    X, Q = G.integer_mixture(5000, 100, seed=2)
    for A in (X, Q):
        assert np.all(A == np.rint(A)) and A.min() >= 0 and A.max() <= 255


def test_vmf_unit_norm_and_concentration():
    X, Q = G.vmf_mixture(3000, 10, d=64, clusters=8, kappa=50.0, seed=3)
    assert np.allclose(np.linalg.norm(X, axis=1), 1.0, atol=1e-5)
    # Wood's sampler: mean cosine to the mean direction is A_d(kappa) ~ 0.57 at d=64, kappa=50
    Y = G.vmf_mixture(20000, 1, d=64, clusters=1, kappa=50.0, seed=4)[0].astype(np.float64)
    mu = Y.mean(0) / np.linalg.norm(Y.mean(0))
    cos = Y @ mu
    p = 64 / 2.0 - 1.0
    approx = 50.0 / (p + np.sqrt(p * p + 2500.0))  # Bessel-ratio bound-style approximation
    assert abs(cos.mean() - approx) < 0.05


def test_sparse_law():
    base, qs = G.sparse_zipf(4000, 500, vocab=30522, lam_doc=120, lam_query=40, seed=4)
    indptr, terms, w = base
    nnz = np.diff(indptr)
    assert abs(nnz.mean() - 120) < 2.0 and nnz.min() >= 1
    for i in range(0, 4000, 97):
        row = terms[indptr[i]:indptr[i + 1]]
        assert np.all(np.diff(row.astype(int)) > 0)
    # Zipf head: term 0 is the most frequent term
    cnt = np.bincount(terms.astype(int), minlength=30522)
    assert cnt.argmax() == 0
    assert np.all(w > 0)
    assert abs(np.diff(qs[0]).mean() - 40) < 2.0


def test_vmf_blocks_are_the_rows_of_the_whole_draw():
    from paper_2501_06121_b300 import datagen as G
    for conc in (None, 0.04):
        X, Q = G.vmf_mixture(70000, 50, d=16, clusters=8, seed=9, concentration=conc)
        blocks, Qb = G.vmf_mixture_blocks(70000, 50, d=16, clusters=8, seed=9, concentration=conc)
        Xb = np.concatenate([b for _, b in blocks])
        assert np.array_equal(X, Xb) and np.array_equal(Q, Qb)


def test_sparse_weights_in_blocks_are_the_stream_of_one_draw():
    # the sparse generator draws its weights in blocks of 2^22; the blocks are
    # the values one draw of all of them gives (same generator state)
    rng = np.random.default_rng(12)
    n = (1 << 22) + 12345
    one = np.exp(0.5 * rng.standard_normal(n)).astype(np.float32)
    rng = np.random.default_rng(12)
    blocks = np.concatenate([np.exp(0.5 * rng.standard_normal(m)) for m in (1 << 22, 12345)]).astype(np.float32)
    assert np.array_equal(one, blocks)
