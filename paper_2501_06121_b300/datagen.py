"""Seeded synthetic inputs (numpy only).

The paper measures on Sift1M (1M x 128, L2), MS MARCO Star/Dragon
(8.8M x 768, IP) and MS MARCO Splade (8.8M sparse, IP) (Sec. 3, Table 1).
Those datasets are not available here; these generators produce inputs with
their shapes and measures at the sizes the workloads below name, and they
stand in for them.  This module holds none of the search method's
arithmetic: it only draws numbers.  Both the CUDA library's tests/benchmark
and the CPU oracle consume what it returns.

Every generator takes a seed; base vectors and queries come from different
child streams of one ``numpy.random.SeedSequence(seed)`` (base = child 0,
queries = child 1, mixture parameters = child 2), so a query is never a base
point and each set is reproducible on its own.
"""
import numpy as np


def _streams(seed):
    ss = np.random.SeedSequence(seed)
    base, query, params = ss.spawn(3)
    return np.random.default_rng(base), np.random.default_rng(query), np.random.default_rng(params)


def _pick(rng, n, c):
    return rng.integers(0, c, size=n)


def gaussian_mixture(n, nq, d=128, clusters=32, centre_lo=0.0, centre_hi=100.0, sigma=5.0, seed=1):
    """Isotropic Gaussian mixture: centres U[lo, hi]^d, uniform component
    choice, N(0, sigma^2) noise; float32.  Returns (base[n, d], queries[nq, d])."""
    rb, rq, rp = _streams(seed)
    centres = rp.uniform(centre_lo, centre_hi, size=(clusters, d))

    def draw(rng, m):
        out = np.empty((m, d), np.float32)
        step = 1 << 16
        for s in range(0, m, step):
            e = min(m, s + step)
            c = _pick(rng, e - s, clusters)
            out[s:e] = centres[c] + sigma * rng.standard_normal((e - s, d))
        return out

    return draw(rb, n), draw(rq, nq)


def integer_mixture(n, nq, d=128, clusters=256, sigma=20.0, seed=2):
    """Integer-valued mixture: centres U[0, 255]^d, N(0, sigma^2) noise,
    rounded to nearest and clamped to [0, 255]; stored as float32 (every
    value is an integer 0..255, exactly representable in FP16 and BF16)."""
    rb, rq, rp = _streams(seed)
    centres = rp.uniform(0.0, 255.0, size=(clusters, d))

    def draw(rng, m):
        out = np.empty((m, d), np.float32)
        step = 1 << 16
        for s in range(0, m, step):
            e = min(m, s + step)
            c = _pick(rng, e - s, clusters)
            v = np.rint(centres[c] + sigma * rng.standard_normal((e - s, d)))
            out[s:e] = np.clip(v, 0.0, 255.0)
        return out

    return draw(rb, n), draw(rq, nq)


def _unit(rng, m, d):
    g = rng.standard_normal((m, d))
    return g / np.linalg.norm(g, axis=1, keepdims=True)


def _wood_w(rng, m, d, kappa):
    """Wood (1994) rejection sampler for the component w = <x, mu> of a von
    Mises-Fisher draw on S^{d-1} with concentration kappa."""
    b = (-2.0 * kappa + np.sqrt(4.0 * kappa * kappa + (d - 1.0) ** 2)) / (d - 1.0)
    x0 = (1.0 - b) / (1.0 + b)
    c = kappa * x0 + (d - 1.0) * np.log(1.0 - x0 * x0)
    out = np.empty(m)
    filled = 0
    while filled < m:
        want = int((m - filled) * 1.3) + 16
        z = rng.beta((d - 1.0) / 2.0, (d - 1.0) / 2.0, size=want)
        u = rng.uniform(size=want)
        w = (1.0 - (1.0 + b) * z) / (1.0 - (1.0 - b) * z)
        ok = kappa * w + (d - 1.0) * np.log(1.0 - x0 * w) - c >= np.log(u)
        w = w[ok][: m - filled]
        out[filled:filled + len(w)] = w
        filled += len(w)
    return out


def _vmf_blocks(rng, m, d, mus, kappa, concentration):
    """Rows of the von Mises-Fisher mixture (or the concentrated variant) in
    blocks of 32,768: yields (first row, float32 block)."""
    step = 1 << 15
    clusters = len(mus)
    for s in range(0, m, step):
        e = min(m, s + step)
        mu = mus[_pick(rng, e - s, clusters)]
        if concentration is not None:
            v = mu + concentration * rng.standard_normal((e - s, d))
            yield s, (v / np.linalg.norm(v, axis=1, keepdims=True)).astype(np.float32)
            continue
        w = _wood_w(rng, e - s, d, kappa)
        g = rng.standard_normal((e - s, d))
        g -= np.sum(g * mu, axis=1, keepdims=True) * mu
        g /= np.linalg.norm(g, axis=1, keepdims=True)
        yield s, (w[:, None] * mu + np.sqrt(np.maximum(0.0, 1.0 - w * w))[:, None] * g).astype(np.float32)


def vmf_mixture(n, nq, d=768, clusters=1024, kappa=50.0, seed=3, concentration=None):
    """Unit-norm mixture of von Mises-Fisher components (Wood's sampler),
    uniform component choice, mean directions uniform on the sphere.  With
    ``concentration=sigma`` it instead draws normalize(mu + sigma * g)."""
    rb, rq, rp = _streams(seed)
    mus = _unit(rp, clusters, d)

    def draw(rng, m):
        out = np.empty((m, d), np.float32)
        for s, blk in _vmf_blocks(rng, m, d, mus, kappa, concentration):
            out[s:s + len(blk)] = blk
        return out

    return draw(rb, n), draw(rq, nq)


def vmf_mixture_blocks(n, nq, d=768, clusters=1024, kappa=50.0, seed=3, concentration=None):
    """The rows of vmf_mixture(n, nq, ...) without holding the base set:
    (a generator of (first row, block) over the n base rows, the queries)."""
    rb, rq, rp = _streams(seed)
    mus = _unit(rp, clusters, d)
    queries = np.empty((nq, d), np.float32)
    for s, blk in _vmf_blocks(rq, nq, d, mus, kappa, concentration):
        queries[s:s + len(blk)] = blk
    return _vmf_blocks(rb, n, d, mus, kappa, concentration), queries


def _zipf_cdf(vocab, s):
    p = 1.0 / np.arange(1, vocab + 1, dtype=np.float64) ** s
    c = np.cumsum(p)
    return c / c[-1]


def _sparse_rows(rng, m, vocab, lam, cdf, wsigma):
    nnz = np.maximum(1, rng.poisson(lam, size=m)).astype(np.int64)
    nnz = np.minimum(nnz, vocab)
    indptr = np.zeros(m + 1, np.int64)
    np.cumsum(nnz, out=indptr[1:])
    terms = np.empty(indptr[-1], np.uint16)
    # Terms are drawn one at a time from the truncated Zipf law and a draw
    # that repeats a term already in the row is redrawn; taking the first
    # nnz distinct values of an i.i.d. stream is the same law.
    step = 4096
    for s in range(0, m, step):
        e = min(m, s + step)
        need = nnz[s:e]
        width = int(need.max() * 2 + 32)
        rows = [None] * (e - s)
        todo = np.arange(e - s)
        while len(todo):
            draws = np.searchsorted(cdf, rng.uniform(size=(len(todo), width)), side="right")
            draws = np.minimum(draws, vocab - 1)
            still = []
            for r, row in zip(todo, draws):
                prev = rows[r]
                seq = row if prev is None else np.concatenate([prev, row])
                _, first = np.unique(seq, return_index=True)
                first.sort()
                if len(first) >= need[r]:
                    rows[r] = np.sort(seq[first[: need[r]]])
                else:
                    rows[r] = seq
                    still.append(r)
            todo = np.array(still, dtype=np.int64)
        for r in range(e - s):
            terms[indptr[s + r]:indptr[s + r + 1]] = rows[r]
    # weights in blocks of 2^22 draws (the same stream as one draw of all of
    # them, with bounded temporaries at 8.8M documents)
    weights = np.empty(indptr[-1], np.float32)
    wstep = 1 << 22
    for s in range(0, len(weights), wstep):
        e = min(len(weights), s + wstep)
        weights[s:e] = np.exp(wsigma * rng.standard_normal(e - s))
    return indptr, terms, weights


def sparse_zipf(n, nq, vocab=30522, lam_doc=120.0, lam_query=40.0, zipf_s=1.1, wsigma=0.5, seed=4):
    """Sparse vectors: nnz = max(1, Poisson(lam)), distinct term ids from a
    truncated Zipf(s) over ranks 1..vocab (term = rank - 1), weights
    exp(N(0, wsigma^2)) float32.  Returns two CSR triples
    (indptr int64, terms uint16 sorted per row, weights float32)."""
    rb, rq, _ = _streams(seed)
    cdf = _zipf_cdf(vocab, zipf_s)
    return (_sparse_rows(rb, n, vocab, lam_doc, cdf, wsigma),
            _sparse_rows(rq, nq, vocab, lam_query, cdf, wsigma))


def densify(csr, vocab):
    indptr, terms, weights = csr
    m = len(indptr) - 1
    out = np.zeros((m, vocab), np.float32)
    rows = np.repeat(np.arange(m), np.diff(indptr))
    out[rows, terms.astype(np.int64)] = weights
    return out
