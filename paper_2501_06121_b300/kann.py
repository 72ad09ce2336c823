"""ctypes binding of libkann.so (argument marshalling only).

Every function here has the name of the C entry point it calls (see
include/kann.h) and does nothing but check shapes, take device pointers from
torch tensors and pass them through; every step of the search runs in the
library's CUDA kernels.  There is no CPU fallback: if the library or a GPU
is missing, the calls raise.
"""
import ctypes
import os

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libkann.so")

KANN_OK, KANN_EINVAL, KANN_ENOMEM, KANN_ECUDA, KANN_EFORMAT, KANN_ETIMEOUT = range(6)
KANN_L2, KANN_IP = 0, 1
KANN_F32, KANN_F16, KANN_BF16, KANN_E4M3 = 0, 1, 2, 3
KANN_QSTAT_HOPCAP, KANN_QSTAT_FORGOT, KANN_QSTAT_BAD_ID, KANN_QSTAT_QUERY_TRUNCATED = 1, 2, 4, 8
KANN_MAX_EF = 1024
KANN_MAX_EXPAND = 4

_TORCH_DTYPE = {KANN_F32: torch.float32, KANN_F16: torch.float16, KANN_BF16: torch.bfloat16,
                KANN_E4M3: torch.uint8}


class KannError(RuntimeError):
    def __init__(self, fn, status):
        msg = _lib().kann_status_str(status).decode()
        if status == KANN_ECUDA:
            msg += " (cudaError %d)" % _lib().kann_last_cuda_error()
        super().__init__("%s failed: %s [%d]" % (fn, msg, status))
        self.status = status


class kann_graph_desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("M", ctypes.c_int32), ("M0", ctypes.c_int32),
                ("max_level", ctypes.c_int32), ("entry", ctypes.c_int32), ("n_upper", ctypes.c_int64),
                ("d_level", ctypes.c_void_p), ("d_l0", ctypes.c_void_p), ("d_upper_slot", ctypes.c_void_p),
                ("d_upper", ctypes.c_void_p)]


class kann_vectors_desc(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int32), ("d", ctypes.c_int32), ("metric", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("d_data", ctypes.c_void_p), ("d_scale", ctypes.c_void_p),
                ("row_stride_bytes", ctypes.c_int64)]


class kann_pq_desc(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int32), ("ksub", ctypes.c_int32), ("dsub", ctypes.c_int32),
                ("metric", ctypes.c_int32), ("d_codes", ctypes.c_void_p), ("d_codebooks", ctypes.c_void_p)]


class kann_sparse_desc(ctypes.Structure):
    _fields_ = [("d_indptr", ctypes.c_void_p), ("d_terms", ctypes.c_void_p), ("d_weights", ctypes.c_void_p),
                ("vocab", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class kann_search_opts(ctypes.Structure):
    _fields_ = [("rerank", ctypes.c_int32), ("max_hops", ctypes.c_int32), ("hash_bits", ctypes.c_int32),
                ("warps_per_block", ctypes.c_int32), ("lanes_per_row", ctypes.c_int32), ("lean", ctypes.c_int32),
                ("pq_lut", ctypes.c_int32),
                ("d_status", ctypes.c_void_p), ("d_counters", ctypes.c_void_p),
                ("d_work_counter", ctypes.c_void_p), ("d_n", ctypes.c_void_p),
                ("visited_format", ctypes.c_int32), ("expand", ctypes.c_int32), ("team", ctypes.c_int32)]


_L = None


def _lib():
    global _L
    if _L is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libkann.so is not built (run paper_2501_06121_b300/build.py or "
                               "__graft_entry__.build()); there is no fallback")
        L = ctypes.CDLL(LIB_PATH)
        P, I, I64, U64, SZ = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_size_t
        sigs = {
            "kann_index_upload": (I, [P, P, P, P, P, P, I]),
            "kann_index_destroy": (I, [P]),
            "kann_search": (I, [P, P, I, I, I, P, P, P]),
            "kann_search_ex": (I, [P, P, I, I, I, P, P, P, P]),
            "kann_search_batch": (I, [P, P, I, P, P, I, I, P, P, P, P]),
            "kann_search_sparse": (I, [P, P, P, P, I, I, I, P, P, P, P]),
            "kann_search_workspace_bytes": (SZ, [P, I, I, I]),
            "kann_search_workspace_bytes_ex": (SZ, [P, I, I, I, P]),
            "kann_exact_knn": (I, [P, P, I, I64, I, I, I, I, P, P, P, SZ, P]),
            "kann_exact_knn_workspace_bytes": (SZ, [I, I64, I, I, I]),
            "kann_quantize": (I, [P, I64, I, I, P, P, P]),
            "kann_hnsw_levels": (I, [I64, I, U64, P, P, P]),
            "kann_hnsw_build_dense": (I, [P, I64, I, I, I, I, U64, I, P, P, P, P, P]),
            "kann_hnsw_build_sparse": (I, [P, P, P, I64, I, I, U64, I, P, P, P, P, P]),
            "kann_exact_knn_sparse": (I, [P, P, P, I64, P, P, P, I, I, I, P, P, P]),
            "kann_pq_train_workspace_bytes": (SZ, [I64, I, I]),
            "kann_pq_train": (I, [P, I64, I, I, I, U64, P, P, SZ, P]),
            "kann_pq_encode": (I, [P, I64, I, I, P, P, P]),
            "kann_hnsw_build_device_workspace_bytes": (SZ, [I64, I, I, I, I]),
            "kann_hnsw_build_device": (I, [P, I64, I, I, I, I, U64, I, I, P, P, P, P, P, P, SZ, P]),
            "kann_hnsw_build_device_sparse_workspace_bytes": (SZ, [I64, I64, I, I, I]),
            "kann_hnsw_build_device_sparse": (I, [P, P, P, I64, I, I, I, U64, I, I, P, P, P, P, P, P, SZ, P]),
            "kann_status_str": (ctypes.c_char_p, [I]),
            "kann_last_cuda_error": (I, []),
        }
        for name, (res, args) in sigs.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _L = L
    return _L


def _check(fn, status):
    if status != KANN_OK:
        raise KannError(fn, status)


def _dev(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _require_cuda(*ts):
    for t in ts:
        if t is not None and (not t.is_cuda or not t.is_contiguous()):
            raise ValueError("expected contiguous CUDA tensors")


# --------------------------------------------------------------------------- index
class Index:
    """A kann_index_t plus the device tensors it borrows (kept alive here)."""

    def __init__(self, handle, keep, kind, d, metric, dtype=None, n=0, M0=0):
        self.handle = handle
        self._keep = keep
        self.kind = kind
        self.d = d
        self.metric = metric
        self.dtype = dtype
        self.n = n
        self.M0 = M0

    def __del__(self):
        if getattr(self, "handle", None) is not None and _L is not None:
            _L.kann_index_destroy(self.handle)
            self.handle = None


def graph_to_device(g, device="cuda"):
    """Copy a serialised graph (dict of numpy arrays, see include/kann.h) to the device."""
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
    return dict(n=int(g["n"]), M=int(g["M"]), M0=int(g["M0"]), max_level=int(g["max_level"]),
                entry=int(g["entry"]), n_upper=int(g["upper"].shape[0]) if int(g["max_level"]) > 0 else 0,
                level=t(g["level"]), l0=t(g["l0"]), upper_slot=t(g["upper_slot"]), upper=t(g["upper"]))


def _vec_desc(data, dtype, metric, scale=None):
    _require_cuda(data, scale)
    n, d = data.shape
    esz = data.element_size()
    return kann_vectors_desc(dtype, d, metric, 0, data.data_ptr(), scale.data_ptr() if scale is not None else None,
                             d * esz)


def kann_index_upload(graph, vectors=None, dtype=KANN_F32, metric=KANN_L2, scale=None, pq=None, sparse=None,
                      rerank=None, validate_ids=True):
    """graph: dict from graph_to_device.  vectors: [n, d] device tensor in
    `dtype` (uint8 codes for KANN_E4M3 with `scale` [n] float32).
    pq: dict(codes=[n, m] uint8, codebooks=[m, 256, dsub] float32, metric).
    sparse: dict(indptr, terms (int16 view of uint16), weights, vocab).
    rerank: [n, d] float32 (exact) or bfloat16 device tensor (re-rank copy)."""
    gd = kann_graph_desc(graph["n"], graph["M"], graph["M0"], graph["max_level"], graph["entry"],
                         graph["n_upper"], graph["level"].data_ptr(), graph["l0"].data_ptr(),
                         graph["upper_slot"].data_ptr(), graph["upper"].data_ptr())
    keep = [graph]
    vd = pd = sd = rd = None
    kind, d = None, None
    if vectors is not None:
        vd = _vec_desc(vectors, dtype, metric, scale)
        keep += [vectors, scale]
        kind, d = "dense", vectors.shape[1]
    if pq is not None:
        _require_cuda(pq["codes"], pq["codebooks"])
        m, ksub, dsub = pq["codebooks"].shape
        pd = kann_pq_desc(m, ksub, dsub, pq.get("metric", metric), pq["codes"].data_ptr(),
                          pq["codebooks"].data_ptr())
        keep.append(pq)
        kind, d = "pq", m * dsub
        metric = pq.get("metric", metric)
    if sparse is not None:
        _require_cuda(sparse["indptr"], sparse["terms"], sparse["weights"])
        sd = kann_sparse_desc(sparse["indptr"].data_ptr(), sparse["terms"].data_ptr(), sparse["weights"].data_ptr(),
                              int(sparse["vocab"]), 0)
        keep.append(sparse)
        kind, d = "sparse", None
        metric = KANN_IP
    if rerank is not None:
        rd = _vec_desc(rerank, KANN_BF16 if rerank.dtype == torch.bfloat16 else KANN_F32, metric)
        keep.append(rerank)
    h = ctypes.c_void_p()
    ref = lambda s: ctypes.byref(s) if s is not None else None
    _check("kann_index_upload", _lib().kann_index_upload(ctypes.byref(h), ctypes.byref(gd), ref(vd), ref(pd), ref(sd),
                                                         ref(rd), int(bool(validate_ids))))
    return Index(h, keep, kind, d, metric, dtype=dtype if kind == "dense" else kind, n=int(graph["n"]),
                 M0=int(graph["M0"]))


KANN_VISITED_AUTO, KANN_VISITED_COMPACT, KANN_VISITED_WIDE = 0, 1, 2
KANN_PQ_LUT_F32, KANN_PQ_LUT_F16, KANN_PQ_LUT_U8 = 0, 1, 2


def _opts(rerank=0, max_hops=0, hash_bits=0, warps_per_block=0, lanes_per_row=0, status=None, counters=None,
          work_counter=None, n_device=None, lean=0, pq_lut_f16=0, visited_format=0, expand=0, pq_lut=None, team=0):
    _require_cuda(status, counters, work_counter, n_device)
    p = lambda t: t.data_ptr() if t is not None else None
    if pq_lut is None:  # pq_lut_f16=1 is the FP16 table
        pq_lut = KANN_PQ_LUT_F16 if pq_lut_f16 else KANN_PQ_LUT_F32
    return kann_search_opts(int(rerank), int(max_hops), int(hash_bits), int(warps_per_block), int(lanes_per_row),
                            int(lean), int(pq_lut),
                            p(status), p(counters), p(work_counter), p(n_device), int(visited_format),
                            int(expand), int(team))


def kann_search(index, queries, k, ef, ids=None, dists=None, stream=None):
    return kann_search_ex(index, queries, k, ef, ids=ids, dists=dists, stream=stream)


def kann_search_ex(index, queries, k, ef, ids=None, dists=None, stream=None, **opts):
    """queries [n, d] float32 on the device -> (ids [n, k] int32, dists [n, k] float32).
    opts: rerank, max_hops, hash_bits, visited_format, expand, warps_per_block, lanes_per_row, lean,
    pq_lut (PQ table format: KANN_PQ_LUT_F32 / F16 / U8; pq_lut_f16=1 is the FP16 table),
    work_counter ([1] int32
    tensor: persistent work-stealing launch), n_device ([1] int32: device-side query count,
    persistent mode), status ([n] int32
    tensor, bits KANN_QSTAT_*), counters ([n, 4] int32 tensor)."""
    _require_cuda(queries)
    n = queries.shape[0]
    if ids is None:
        ids = torch.empty((n, k), dtype=torch.int32, device=queries.device)
    if dists is None:
        dists = torch.empty((n, k), dtype=torch.float32, device=queries.device)
    o = _opts(**opts)
    _check("kann_search_ex", _lib().kann_search_ex(index.handle, _dev(queries), n, k, ef, _dev(ids), _dev(dists),
                                                   ctypes.byref(o), _stream(stream)))
    return ids, dists


def kann_search_batch(index, queries, k, ef, kmax=None, efmax=None, ids=None, dists=None, stream=None, **opts):
    """Per-query k and ef (int32 device tensors [n]); outputs [n, kmax]."""
    _require_cuda(queries, k, ef)
    n = queries.shape[0]
    kmax = int(k.max().item()) if kmax is None else kmax
    efmax = int(ef.max().item()) if efmax is None else efmax
    if ids is None:
        ids = torch.empty((n, kmax), dtype=torch.int32, device=queries.device)
    if dists is None:
        dists = torch.empty((n, kmax), dtype=torch.float32, device=queries.device)
    o = _opts(**opts)
    _check("kann_search_batch", _lib().kann_search_batch(index.handle, _dev(queries), n, _dev(k), _dev(ef), kmax, efmax,
                                                         _dev(ids), _dev(dists), ctypes.byref(o), _stream(stream)))
    return ids, dists


def kann_search_workspace_bytes(index, n, kmax, efmax, **opts):
    """Device bytes a batch of n queries (k <= kmax, ef <= efmax) needs besides
    the index (queries, k/ef words, outputs, status, counters); 0 if no search
    with these settings (and search options `opts`, as for kann_search_ex)
    can run."""
    if not opts:
        return int(_lib().kann_search_workspace_bytes(index.handle, n, kmax, efmax))
    o = _opts(**opts)
    return int(_lib().kann_search_workspace_bytes_ex(index.handle, n, kmax, efmax, ctypes.byref(o)))


def kann_search_sparse(index, q_indptr, q_terms, q_weights, k, ef, ids=None, dists=None, stream=None, **opts):
    _require_cuda(q_indptr, q_terms, q_weights)
    n = q_indptr.shape[0] - 1
    dev = q_indptr.device
    if ids is None:
        ids = torch.empty((n, k), dtype=torch.int32, device=dev)
    if dists is None:
        dists = torch.empty((n, k), dtype=torch.float32, device=dev)
    o = _opts(**opts)
    _check("kann_search_sparse", _lib().kann_search_sparse(index.handle, _dev(q_indptr), _dev(q_terms),
                                                           _dev(q_weights), n, k, ef, _dev(ids), _dev(dists),
                                                           ctypes.byref(o), _stream(stream)))
    return ids, dists


def kann_exact_knn_workspace_bytes(nq, nb, d, k, dtype=KANN_F32):
    return int(_lib().kann_exact_knn_workspace_bytes(nq, nb, d, k, dtype))


def _exact_args(fn, queries, base, k, dtype, ids, dists):
    """Shape and type checks shared by the exact k-NN calls (the library reads
    nq x d and nb x d elements of `dtype` and writes nq x k outputs, so a
    mismatch here would be an out-of-bounds access on the device)."""
    _require_cuda(queries, base, ids, dists)
    if dtype not in (KANN_F32, KANN_F16, KANN_BF16):
        raise ValueError("%s: dtype must be KANN_F32, KANN_F16 or KANN_BF16" % fn)
    want = _TORCH_DTYPE[dtype]
    if queries.dim() != 2 or base.dim() != 2 or base.shape[1] != queries.shape[1]:
        raise ValueError("%s: queries [nq, d] and base [nb, d] must share d" % fn)
    if queries.dtype != want or base.dtype != want:
        raise ValueError("%s: queries and base must be %s for this dtype, got %s / %s"
                         % (fn, want, queries.dtype, base.dtype))
    if queries.device != base.device:
        raise ValueError("%s: queries and base must be on the same device" % fn)
    nq = queries.shape[0]
    for t, tt, name in ((ids, torch.int32, "ids"), (dists, torch.float32, "dists")):
        if t is not None and (tuple(t.shape) != (nq, k) or t.dtype != tt or t.device != queries.device):
            raise ValueError("%s: %s must be a [%d, %d] %s tensor on %s" % (fn, name, nq, k, tt, queries.device))
    if ids is None:
        ids = torch.empty((nq, k), dtype=torch.int32, device=queries.device)
    if dists is None:
        dists = torch.empty((nq, k), dtype=torch.float32, device=queries.device)
    return ids, dists


def kann_exact_knn(queries, base, k, metric, dtype=KANN_F32, ws=None, ids=None, dists=None, stream=None):
    """Brute-force k-NN: queries [nq, d], base [nb, d] device tensors in `dtype`."""
    ids, dists = _exact_args("kann_exact_knn", queries, base, k, dtype, ids, dists)
    nq, d = queries.shape
    nb = base.shape[0]
    dev = queries.device
    with torch.cuda.device(dev):
        need = kann_exact_knn_workspace_bytes(nq, nb, d, k, dtype)
        if ws is None:
            ws = torch.empty(max(need, 16), dtype=torch.uint8, device=dev)
        _require_cuda(ws)
        _check("kann_exact_knn", _lib().kann_exact_knn(_dev(queries), _dev(base), nq, nb, d, metric, dtype, k,
                                                       _dev(ids), _dev(dists), _dev(ws),
                                                       ws.numel() * ws.element_size(), _stream(stream)))
    return ids, dists


def kann_exact_knn_sparse(base, queries, vocab, k, ids=None, dists=None, stream=None):
    """Sparse-IP brute force: base / queries are (indptr int64, terms int16-view
    of uint16, weights float32) device CSR triples."""
    _require_cuda(*base, *queries)
    nq = queries[0].shape[0] - 1
    dev = queries[0].device
    if ids is None:
        ids = torch.empty((nq, k), dtype=torch.int32, device=dev)
    if dists is None:
        dists = torch.empty((nq, k), dtype=torch.float32, device=dev)
    _check("kann_exact_knn_sparse", _lib().kann_exact_knn_sparse(
        _dev(base[0]), _dev(base[1]), _dev(base[2]), base[0].shape[0] - 1, _dev(queries[0]), _dev(queries[1]),
        _dev(queries[2]), nq, vocab, k, _dev(ids), _dev(dists), _stream(stream)))
    return ids, dists


def kann_quantize(x, dtype, stream=None):
    """FP32 rows [n, d] -> storage format on the device: (data, scale or None)."""
    _require_cuda(x)
    n, d = x.shape
    out = torch.empty((n, d), dtype=_TORCH_DTYPE[dtype], device=x.device)
    scale = torch.empty(n, dtype=torch.float32, device=x.device) if dtype == KANN_E4M3 else None
    _check("kann_quantize", _lib().kann_quantize(_dev(x), n, d, dtype, _dev(out), _dev(scale), _stream(stream)))
    return out, scale


def kann_pq_train(x, m, iters=25, seed=0, stream=None):
    """Device PQ codebooks [m, 256, d/m] float32 trained on FP32 rows x [n, d]."""
    _require_cuda(x)
    n, d = x.shape
    cb = torch.empty((m, 256, d // m), dtype=torch.float32, device=x.device)
    wsb = int(_lib().kann_pq_train_workspace_bytes(n, d, m))
    ws = torch.empty(max(wsb, 16), dtype=torch.uint8, device=x.device)
    _check("kann_pq_train", _lib().kann_pq_train(_dev(x), n, d, m, iters, seed, _dev(cb), _dev(ws), ws.numel(),
                                                 _stream(stream)))
    return cb


def kann_pq_encode(x, codebooks, stream=None):
    """uint8 codes [n, m] of FP32 rows x [n, d] for device codebooks [m, 256, dsub]."""
    _require_cuda(x, codebooks)
    n, d = x.shape
    m = codebooks.shape[0]
    codes = torch.empty((n, m), dtype=torch.uint8, device=x.device)
    _check("kann_pq_encode", _lib().kann_pq_encode(_dev(x), n, d, m, _dev(codebooks), _dev(codes), _stream(stream)))
    return codes


# --------------------------------------------------------------------------- host graph build
def kann_hnsw_levels(n, M, seed):
    level = np.empty(n, np.int8)
    mx = ctypes.c_int32()
    nu = ctypes.c_int64()
    _check("kann_hnsw_levels", _lib().kann_hnsw_levels(n, M, seed, level.ctypes.data_as(ctypes.c_void_p),
                                                       ctypes.byref(mx), ctypes.byref(nu)))
    return level, mx.value, nu.value


def _graph_buffers(n, M, seed):
    level, L, nu = kann_hnsw_levels(n, M, seed)
    l0 = np.empty((n, 2 * M), np.int32)
    us = np.empty(n, np.int32)
    up = np.full((max(nu, 1), max(L, 1), M), -1, np.int32)
    return level, L, nu, l0, us, up


def _vp(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def kann_hnsw_build_dense(x, metric, M, ef_construction, seed, nthreads=0):
    """Host HNSW build over FP32 rows x [n, d] (numpy); returns the serialised graph dict."""
    x = np.ascontiguousarray(x, np.float32)
    n, d = x.shape
    level, L, nu, l0, us, up = _graph_buffers(n, M, seed)
    entry = ctypes.c_int32()
    _check("kann_hnsw_build_dense", _lib().kann_hnsw_build_dense(_vp(x), n, d, metric, M, ef_construction, seed,
                                                                 nthreads, _vp(level), _vp(l0), _vp(us), _vp(up),
                                                                 ctypes.byref(entry)))
    return dict(n=n, M=M, M0=2 * M, max_level=L, entry=entry.value, level=level, l0=l0, upper_slot=us, upper=up)


def kann_hnsw_build_sparse(csr, M, ef_construction, seed, nthreads=0):
    indptr = np.ascontiguousarray(csr[0], np.int64)
    terms = np.ascontiguousarray(csr[1], np.uint16)
    w = np.ascontiguousarray(csr[2], np.float32)
    n = len(indptr) - 1
    level, L, nu, l0, us, up = _graph_buffers(n, M, seed)
    entry = ctypes.c_int32()
    _check("kann_hnsw_build_sparse", _lib().kann_hnsw_build_sparse(_vp(indptr), _vp(terms), _vp(w), n, M,
                                                                   ef_construction, seed, nthreads, _vp(level),
                                                                   _vp(l0), _vp(us), _vp(up), ctypes.byref(entry)))
    return dict(n=n, M=M, M0=2 * M, max_level=L, entry=entry.value, level=level, l0=l0, upper_slot=us, upper=up)


def kann_hnsw_build_device(x, metric, M, ef_construction, seed, batch=0, nthreads=0, stream=None):
    """HNSW over FP32 device rows x [n, d] with the layer-0 insertions on the
    GPU (the upper-layer nodes are inserted on the host first).  Returns the
    serialised graph as a dict of numpy arrays (as kann_hnsw_build_dense)."""
    _require_cuda(x)
    if x.dtype != torch.float32 or x.dim() != 2:
        raise ValueError("kann_hnsw_build_device: x must be [n, d] float32")
    n, d = x.shape
    level, L, nu, l0, us, up = _graph_buffers(n, M, seed)
    dev = x.device
    with torch.cuda.device(dev):
        d_l0 = torch.empty((n, 2 * M), dtype=torch.int32, device=dev)
        d_us = torch.empty(n, dtype=torch.int32, device=dev)
        d_up = torch.empty(up.shape, dtype=torch.int32, device=dev)
        wsb = int(_lib().kann_hnsw_build_device_workspace_bytes(n, d, M, ef_construction, batch))
        ws = torch.empty(max(wsb, 16), dtype=torch.uint8, device=dev)
        entry = ctypes.c_int32()
        _check("kann_hnsw_build_device", _lib().kann_hnsw_build_device(
            _dev(x), n, d, metric, M, ef_construction, seed, batch, nthreads, _vp(level), _dev(d_l0), _dev(d_us),
            _dev(d_up), ctypes.byref(entry), _dev(ws), ws.numel(), _stream(stream)))
        torch.cuda.synchronize()
    if L > 0:
        up = d_up.cpu().numpy()
    return dict(n=n, M=M, M0=2 * M, max_level=L, entry=entry.value, level=level, l0=d_l0.cpu().numpy(),
                upper_slot=d_us.cpu().numpy(), upper=up)


def kann_hnsw_build_device_sparse(indptr, terms, weights, vocab, M, ef_construction, seed, batch=0, nthreads=0,
                                  stream=None):
    """HNSW over a device CSR (indptr int64 [n+1], terms int16-view of uint16,
    weights float32) with the layer-0 insertions on the GPU; returns the
    serialised graph as a dict of numpy arrays."""
    _require_cuda(indptr, terms, weights)
    n = indptr.shape[0] - 1
    nnz = int(indptr[-1].item())
    level, L, nu, l0, us, up = _graph_buffers(n, M, seed)
    dev = indptr.device
    with torch.cuda.device(dev):
        d_l0 = torch.empty((n, 2 * M), dtype=torch.int32, device=dev)
        d_us = torch.empty(n, dtype=torch.int32, device=dev)
        d_up = torch.empty(up.shape, dtype=torch.int32, device=dev)
        wsb = int(_lib().kann_hnsw_build_device_sparse_workspace_bytes(n, nnz, M, ef_construction, batch))
        ws = torch.empty(max(wsb, 16), dtype=torch.uint8, device=dev)
        entry = ctypes.c_int32()
        _check("kann_hnsw_build_device_sparse", _lib().kann_hnsw_build_device_sparse(
            _dev(indptr), _dev(terms), _dev(weights), n, vocab, M, ef_construction, seed, batch, nthreads, _vp(level),
            _dev(d_l0), _dev(d_us), _dev(d_up), ctypes.byref(entry), _dev(ws), ws.numel(), _stream(stream)))
        torch.cuda.synchronize()
    if L > 0:
        up = d_up.cpu().numpy()
    return dict(n=n, M=M, M0=2 * M, max_level=L, entry=entry.value, level=level, l0=d_l0.cpu().numpy(),
                upper_slot=d_us.cpu().numpy(), upper=up)


KANN_NOALLOC_SCRATCH_BYTES = 16 << 20


def kann_exact_knn_noalloc(queries, base, k, metric, dtype=KANN_F32, ids=None, dists=None, stream=None):
    """kann_exact_knn without any device allocation inside the library: the
    scratch is the library's static per-GPU array, so the outputs are the only
    buffers involved (allocate them yourself to avoid torch allocations too).
    Raises ValueError before calling when the request needs more scratch than
    KANN_NOALLOC_SCRATCH_BYTES; calls that overlap on the GPU must not run
    concurrently (they share the array)."""
    nq, d = queries.shape
    nb = base.shape[0]
    need = kann_exact_knn_workspace_bytes(nq, nb, d, k, dtype)
    if need > KANN_NOALLOC_SCRATCH_BYTES:
        raise ValueError("kann_exact_knn_noalloc: %d queries need %d bytes of scratch, more than the %d-byte "
                         "static array; split the queries" % (nq, need, KANN_NOALLOC_SCRATCH_BYTES))
    ids, dists = _exact_args("kann_exact_knn_noalloc", queries, base, k, dtype, ids, dists)
    f = _lib().kann_exact_knn_noalloc
    P, I = ctypes.c_void_p, ctypes.c_int
    f.restype = I
    f.argtypes = [P, P, I, ctypes.c_int64, I, I, I, I, P, P, P]
    # the library looks up the static array of the current device: make it the
    # device the tensors live on
    with torch.cuda.device(queries.device):
        _check("kann_exact_knn_noalloc", f(_dev(queries), _dev(base), nq, nb, d, metric, dtype, k, _dev(ids),
                                           _dev(dists), _stream(stream)))
    return ids, dists
