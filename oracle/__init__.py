"""FP64 CPU oracle for batched HNSW search (TEST INFRASTRUCTURE).

This package is the slow, plain reference that the CUDA search path is
checked against.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it; the library itself never
does, and it shares no code with the library.

The arithmetic lives in ``kann_oracle.cpp`` (HNSW per Malkov & Yashunin,
PQ per Jegou et al., the paper's three measures from its Table 1); this
module only marshals numpy arrays through ctypes.

Parity unpinned (no independent value exists to match): the exact edge set
chosen by the construction heuristic, and the PQ training choices
(k-means++ seeding, iteration count, empty-cluster reseeding).
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

DT_F32, DT_F16, DT_BF16, DT_E4M3 = 0, 1, 2, 3
L2, IP = 0, 1

_p = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int
_u64 = ctypes.c_uint64


def lib():
    global _lib
    if _lib is None:
        _lib = load(_build.build())
    return _lib


def load(path):
    """The oracle library at `path` with its argument types set (lib() loads
    the built oracle; the tests also load copies with planted mistakes)."""
    L = ctypes.CDLL(path)
    sig = {
        "orc_encode_f16": [_p, _i64, _p],
        "orc_encode_bf16": [_p, _i64, _p],
        "orc_decode_f16": [_p, _i64, _p],
        "orc_decode_bf16": [_p, _i64, _p],
        "orc_decode_e4m3": [_p, _i64, _p],
        "orc_encode_e4m3_rows": [_p, _i64, _i32, _p, _p],
        "orc_splitmix64_seq": [_u64, _i64, _p],
        "orc_levels": [_i64, _i32, _u64, _p],
        "orc_graph_build_dense": [_i32, _p, _p, _i64, _i32, _i32, _i32, _i32, _u64, _i32],
        "orc_graph_build_sparse": [_p, _p, _p, _i64, _i32, _i32, _u64, _i32],
        "orc_graph_free": [_p],
        "orc_graph_info": [_p, _p],
        "orc_graph_export": [_p, _p, _p, _p, _p],
        "orc_graph_import": [_i64, _i32, _i32, _i32, _i64, _p, _p, _p, _p],
        "orc_search_dense": [_p, _i32, _p, _p, _i32, _i32, _p, _i64, _i32, _i32, _i32, _i64, _i32,
                             _p, _p, _p],
        "orc_search_dense_multi": [_p, _i32, _p, _p, _i32, _i32, _p, _i64, _i32, _i32, _i32, _i32, _p, _p, _p],
        "orc_search_pq": [_p, _p, _p, _i32, _i32, _i32, _i32, _i32, _p, _i64, _i32, _i32, _i32, _i32, _p, _p,
                          _p],
        "orc_search_sparse": [_p, _p, _p, _p, _p, _p, _p, _i64, _i32, _i32, _i32, _i32, _p, _p, _p],
        "orc_rerank_dense": [_i32, _p, _p, _i32, _i32, _p, _i64, _p, _i32, _i32, _p, _p],
        "orc_dist_dense": [_i32, _p, _p, _i32, _i32, _p, _i64, _p, _i32, _p],
        "orc_exact_dense": [_i32, _p, _p, _i64, _i32, _i32, _p, _i64, _i32, _i32, _p, _p],
        "orc_exact_sparse": [_p, _p, _p, _i64, _p, _p, _p, _i64, _i32, _i32, _p, _p],
        "orc_exact_pq": [_p, _p, _i64, _i32, _i32, _i32, _i32, _p, _i64, _i32, _p, _p],
        "orc_pq_lut": [_p, _i32, _i32, _i32, _i32, _i32, _p, _p],
        "orc_pq_lut_u8": [_p, _i32, _i32, _i32, _i32, _p, _p, _p, _p],
        "orc_pq_encode": [_p, _i64, _i32, _i32, _i32, _p, _p],
        "orc_pq_reconstruct": [_p, _i64, _i32, _i32, _i32, _p, _p],
        "orc_pq_train": [_p, _i64, _i32, _i32, _i32, _i32, _u64, _p, _p],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = None
    L.orc_graph_build_dense.restype = _p
    L.orc_graph_build_sparse.restype = _p
    L.orc_graph_import.restype = _p
    return L


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ----------------------------------------------------------------- formats
def encode_f16(x):
    x = _c(x, np.float32)
    out = np.empty(x.shape, np.uint16)
    lib().orc_encode_f16(_ptr(x), x.size, _ptr(out))
    return out


def encode_bf16(x):
    x = _c(x, np.float32)
    out = np.empty(x.shape, np.uint16)
    lib().orc_encode_bf16(_ptr(x), x.size, _ptr(out))
    return out


def decode_f16(h):
    h = _c(h, np.uint16)
    out = np.empty(h.shape, np.float64)
    lib().orc_decode_f16(_ptr(h), h.size, _ptr(out))
    return out


def decode_bf16(h):
    h = _c(h, np.uint16)
    out = np.empty(h.shape, np.float64)
    lib().orc_decode_bf16(_ptr(h), h.size, _ptr(out))
    return out


def decode_e4m3(c):
    c = _c(c, np.uint8)
    out = np.empty(c.shape, np.float64)
    lib().orc_decode_e4m3(_ptr(c), c.size, _ptr(out))
    return out


def encode_e4m3_rows(x):
    """Per-row scaled E4M3 codes and FP32 scales (s = max|x|/448)."""
    x = _c(x, np.float32)
    n, d = x.shape
    codes = np.empty((n, d), np.uint8)
    scales = np.empty(n, np.float32)
    lib().orc_encode_e4m3_rows(_ptr(x), n, d, _ptr(codes), _ptr(scales))
    return codes, scales


# ----------------------------------------------------------------- levels
def splitmix64_seq(state, n):
    out = np.empty(n, np.uint64)
    lib().orc_splitmix64_seq(state, n, _ptr(out))
    return out


def levels(n, M, seed):
    out = np.empty(n, np.int8)
    lib().orc_levels(n, M, seed, _ptr(out))
    return out


# ----------------------------------------------------------------- graphs
class Graph:
    """An oracle-owned HNSW graph; `arrays()` gives its serialised form."""

    def __init__(self, handle, keep=()):
        self.h = handle
        self._keep = keep
        info = np.empty(6, np.int64)
        lib().orc_graph_info(self.h, _ptr(info))
        self.n, self.M, self.M0, self.max_level, self.entry, self.n_upper = (int(v) for v in info)

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.orc_graph_free(self.h)
            self.h = None

    def arrays(self):
        level = np.empty(self.n, np.int8)
        l0 = np.empty((self.n, self.M0), np.int32)
        upper_slot = np.empty(self.n, np.int32)
        upper = np.empty((max(self.n_upper, 1), max(self.max_level, 1), self.M), np.int32)
        upper.fill(-1)
        lib().orc_graph_export(self.h, _ptr(level), _ptr(l0), _ptr(upper_slot), _ptr(upper))
        return dict(n=self.n, M=self.M, M0=self.M0, max_level=self.max_level, entry=self.entry,
                    level=level, l0=l0, upper_slot=upper_slot, upper=upper)


def build_dense(data, metric, M, efC, seed, dtype=DT_F32, scale=None, simple=False):
    data = np.ascontiguousarray(data)
    n, d = data.shape
    h = lib().orc_graph_build_dense(dtype, _ptr(data), _ptr(scale), n, d, metric, M, efC, seed, int(simple))
    return Graph(h)


def build_sparse(indptr, terms, weights, M, efC, seed, simple=False):
    indptr, terms, weights = _c(indptr, np.int64), _c(terms, np.uint16), _c(weights, np.float32)
    n = len(indptr) - 1
    h = lib().orc_graph_build_sparse(_ptr(indptr), _ptr(terms), _ptr(weights), n, M, efC, seed, int(simple))
    return Graph(h)


def import_graph(g):
    """Oracle copy of a serialised graph dict (keys as in Graph.arrays())."""
    level = _c(g["level"], np.int8)
    l0 = _c(g["l0"], np.int32)
    us = _c(g["upper_slot"], np.int32)
    up = _c(g["upper"], np.int32)
    h = lib().orc_graph_import(int(g["n"]), int(g["M"]), int(g["M0"]), int(g["max_level"]), int(g["entry"]),
                               _ptr(level), _ptr(l0), _ptr(us), _ptr(up))
    return Graph(h)


# ----------------------------------------------------------------- search
FORM_TWO_HEAP, FORM_FLAGS = 0, 1


def search_dense(g, data, queries, k, ef, metric, dtype=DT_F32, scale=None, form=FORM_FLAGS,
                 visited_cap=0, nthreads=0):
    data = np.ascontiguousarray(data)
    queries = _c(queries, np.float32)
    nq, d = queries.shape
    ids = np.empty((nq, k), np.int32)
    dists = np.empty((nq, k), np.float64)
    cnt = np.empty((nq, 4), np.int64)
    lib().orc_search_dense(g.h, dtype, _ptr(data), _ptr(scale), d, metric, _ptr(queries), nq, k, ef, form,
                           visited_cap, nthreads, _ptr(ids), _ptr(dists), _ptr(cnt))
    return ids, dists, cnt


def search_dense_multi(g, data, queries, k, ef, metric, expand, dtype=DT_F32, scale=None, nthreads=0):
    """Dense search whose layer-0 step expands the `expand` best unexpanded
    entries at once (a batched variant, not HNSW's one-at-a-time step)."""
    data = np.ascontiguousarray(data)
    queries = _c(queries, np.float32)
    nq, d = queries.shape
    ids = np.empty((nq, k), np.int32)
    dists = np.empty((nq, k), np.float64)
    cnt = np.empty((nq, 4), np.int64)
    lib().orc_search_dense_multi(g.h, dtype, _ptr(data), _ptr(scale), d, metric, _ptr(queries), nq, k, ef, expand,
                                 nthreads, _ptr(ids), _ptr(dists), _ptr(cnt))
    return ids, dists, cnt


LUT_EXACT, LUT_F16, LUT_U8 = 0, 1, 2


def search_pq(g, codes, codebooks, queries, k, ef, metric, form=FORM_FLAGS, nthreads=0, lut_f16=False, lut=None):
    """ADC search.  lut: LUT_EXACT (FP64 entries), LUT_F16 (the per-query table
    held in FP16 with a power-of-two scale: each entry scaled so the largest
    |entry| is at most 2^15, rounded to nearest, scaled back) or LUT_U8 (the
    uint8 reading: FP32 entries quantised per query to 0..255 by
    (entry - min_j) / scale; distances are the integer sums of those values,
    see pq_lut_u8).  lut_f16=True is LUT_F16."""
    if lut is None:
        lut = LUT_F16 if lut_f16 else LUT_EXACT
    codes = _c(codes, np.uint8)
    codebooks = _c(codebooks, np.float32)
    queries = _c(queries, np.float32)
    m, ksub, dsub = codebooks.shape
    nq = queries.shape[0]
    ids = np.empty((nq, k), np.int32)
    dists = np.empty((nq, k), np.float64)
    cnt = np.empty((nq, 4), np.int64)
    lib().orc_search_pq(g.h, _ptr(codes), _ptr(codebooks), m, ksub, dsub, metric, int(lut), _ptr(queries),
                        nq, k, ef, form, nthreads, _ptr(ids), _ptr(dists), _ptr(cnt))
    return ids, dists, cnt


def search_sparse(g, base, queries, k, ef, form=FORM_FLAGS, nthreads=0):
    """base / queries: (indptr, terms, weights) CSR triples."""
    bi, bt, bw = _c(base[0], np.int64), _c(base[1], np.uint16), _c(base[2], np.float32)
    qi, qt, qw = _c(queries[0], np.int64), _c(queries[1], np.uint16), _c(queries[2], np.float32)
    nq = len(qi) - 1
    ids = np.empty((nq, k), np.int32)
    dists = np.empty((nq, k), np.float64)
    cnt = np.empty((nq, 4), np.int64)
    lib().orc_search_sparse(g.h, _ptr(bi), _ptr(bt), _ptr(bw), _ptr(qi), _ptr(qt), _ptr(qw), nq, k, ef, form,
                            nthreads, _ptr(ids), _ptr(dists), _ptr(cnt))
    return ids, dists, cnt


def rerank_dense(data, queries, cand, k, metric, dtype=DT_F32, scale=None):
    data = np.ascontiguousarray(data)
    queries = _c(queries, np.float32)
    cand = _c(cand, np.int32)
    nq, d = queries.shape
    R = cand.shape[1]
    ids = np.empty((nq, k), np.int32)
    dists = np.empty((nq, k), np.float64)
    lib().orc_rerank_dense(dtype, _ptr(data), _ptr(scale), d, metric, _ptr(queries), nq, _ptr(cand), R, k,
                           _ptr(ids), _ptr(dists))
    return ids, dists


def dist_dense(data, queries, ids, metric, dtype=DT_F32, scale=None):
    data = np.ascontiguousarray(data)
    queries = _c(queries, np.float32)
    ids = _c(ids, np.int32)
    nq, d = queries.shape
    out = np.empty(ids.shape, np.float64)
    lib().orc_dist_dense(dtype, _ptr(data), _ptr(scale), d, metric, _ptr(queries), nq, _ptr(ids), ids.shape[1],
                         _ptr(out))
    return out


# ----------------------------------------------------------------- exact
def exact_dense(data, queries, k, metric, dtype=DT_F32, scale=None, nthreads=0):
    data = np.ascontiguousarray(data)
    queries = _c(queries, np.float32)
    nq, d = queries.shape
    n = data.shape[0]
    ids = np.empty((nq, k), np.int32)
    dists = np.empty((nq, k), np.float64)
    lib().orc_exact_dense(dtype, _ptr(data), _ptr(scale), n, d, metric, _ptr(queries), nq, k, nthreads,
                          _ptr(ids), _ptr(dists))
    return ids, dists


def exact_sparse(base, queries, k, nthreads=0):
    bi, bt, bw = _c(base[0], np.int64), _c(base[1], np.uint16), _c(base[2], np.float32)
    qi, qt, qw = _c(queries[0], np.int64), _c(queries[1], np.uint16), _c(queries[2], np.float32)
    nq = len(qi) - 1
    ids = np.empty((nq, k), np.int32)
    dists = np.empty((nq, k), np.float64)
    lib().orc_exact_sparse(_ptr(bi), _ptr(bt), _ptr(bw), len(bi) - 1, _ptr(qi), _ptr(qt), _ptr(qw), nq, k,
                           nthreads, _ptr(ids), _ptr(dists))
    return ids, dists


def exact_pq(codes, codebooks, queries, k, metric):
    codes = _c(codes, np.uint8)
    codebooks = _c(codebooks, np.float32)
    queries = _c(queries, np.float32)
    m, ksub, dsub = codebooks.shape
    nq = queries.shape[0]
    ids = np.empty((nq, k), np.int32)
    dists = np.empty((nq, k), np.float64)
    lib().orc_exact_pq(_ptr(codes), _ptr(codebooks), codes.shape[0], m, ksub, dsub, metric, _ptr(queries), nq, k,
                       _ptr(ids), _ptr(dists))
    return ids, dists


# ----------------------------------------------------------------- PQ
def pq_train(X, m, ksub, iters, seed):
    X = _c(X, np.float32)
    n, d = X.shape
    dsub = d // m
    cb = np.empty((m, ksub, dsub), np.float32)
    obj = np.empty((m, iters + 1), np.float64)
    lib().orc_pq_train(_ptr(X), n, m, ksub, dsub, iters, seed, _ptr(cb), _ptr(obj))
    return cb, obj


def pq_encode(X, codebooks):
    X = _c(X, np.float32)
    codebooks = _c(codebooks, np.float32)
    m, ksub, dsub = codebooks.shape
    codes = np.empty((X.shape[0], m), np.uint8)
    lib().orc_pq_encode(_ptr(X), X.shape[0], m, ksub, dsub, _ptr(codebooks), _ptr(codes))
    return codes


def pq_reconstruct(codes, codebooks):
    codes = _c(codes, np.uint8)
    codebooks = _c(codebooks, np.float32)
    m, ksub, dsub = codebooks.shape
    out = np.empty((codes.shape[0], m * dsub), np.float32)
    lib().orc_pq_reconstruct(_ptr(codes), codes.shape[0], m, ksub, dsub, _ptr(codebooks), _ptr(out))
    return out


def pq_lut_u8(codebooks, q, metric):
    """The uint8 reading of one query's table: (values [m, 256] uint8, scale,
    summin) -- a row's distance is summin + scale * (sum of its values), each
    of the two operations rounded in FP32."""
    codebooks = _c(codebooks, np.float32)
    q = _c(q, np.float32)
    m, ksub, dsub = codebooks.shape
    v = np.empty((m, ksub), np.uint8)
    sc = np.empty(1, np.float32)
    sm = np.empty(1, np.float32)
    lib().orc_pq_lut_u8(_ptr(codebooks), m, ksub, dsub, metric, _ptr(q), _ptr(v), _ptr(sc), _ptr(sm))
    return v, sc[0], sm[0]


def pq_lut(codebooks, q, metric, lut_f16=False):
    codebooks = _c(codebooks, np.float32)
    q = _c(q, np.float32)
    m, ksub, dsub = codebooks.shape
    lut = np.empty((m, ksub), np.float64)
    lib().orc_pq_lut(_ptr(codebooks), m, ksub, dsub, metric, int(bool(lut_f16)), _ptr(q), _ptr(lut))
    return lut
