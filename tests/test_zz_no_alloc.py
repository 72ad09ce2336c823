"""kann_exact_knn_noalloc: exact k-NN for callers that cannot allocate device
memory (their device memory is owned by another allocator, or cudaMalloc's
implicit synchronisation is not allowed on their path).  It must return what
kann_exact_knn returns with caller-provided scratch, call after call, while
reusing one static scratch array.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2501_06121_b300 import kann as K

pytestmark = pytest.mark.gpu


def _entry():
    f = K._lib().kann_exact_knn_noalloc
    P, I = ctypes.c_void_p, ctypes.c_int
    f.restype = I
    f.argtypes = [P, P, I, ctypes.c_int64, I, I, I, I, P, P, P]
    return f


def _call(f, Q, X, k, metric):
    nq = Q.shape[0]
    ids = torch.full((nq, k), -7, dtype=torch.int32, device="cuda")
    d = torch.full((nq, k), -7.0, dtype=torch.float32, device="cuda")
    rc = f(Q.data_ptr(), X.data_ptr(), nq, X.shape[0], Q.shape[1], metric, K.KANN_F32, k, ids.data_ptr(),
           d.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == K.KANN_OK, K._lib().kann_status_str(rc)
    torch.cuda.synchronize()
    return ids.cpu().numpy(), d.cpu().numpy()


@pytest.mark.parametrize("metric", [K.KANN_L2, K.KANN_IP])
def test_noalloc_equals_workspace_entry_point_twice_in_a_row(metric):
    f = _entry()
    rng = np.random.default_rng(11 + metric)
    X = torch.from_numpy(rng.standard_normal((40000, 128)).astype(np.float32)).cuda()
    for call in range(2):  # the second call reuses scratch holding the first call's lists
        nq, k = (700, 10) if call == 0 else (333, 32)
        Q = torch.from_numpy(rng.standard_normal((nq, 128)).astype(np.float32)).cuda()
        ri, rd = K.kann_exact_knn(Q, X, k, metric)
        torch.cuda.synchronize()
        ri, rd = ri.cpu().numpy(), rd.cpu().numpy()
        gi, gd = _call(f, Q, X, k, metric)
        # the same kernels run on the same inputs: ids equal, distances within
        # the 1e-5 relative tolerance of the other tests (in fact identical)
        assert np.array_equal(gi, ri)
        assert np.all(np.abs(gd - rd) <= 1e-5 * np.abs(rd))


def test_noalloc_rejects_requests_beyond_its_scratch():
    f = _entry()
    X = torch.zeros((1 << 20, 4), dtype=torch.float32, device="cuda")
    Q = torch.zeros((40000, 4), dtype=torch.float32, device="cuda")
    need = K.kann_exact_knn_workspace_bytes(40000, 1 << 20, 4, 256)
    assert need > K.KANN_NOALLOC_SCRATCH_BYTES
    ids = torch.empty((40000, 256), dtype=torch.int32, device="cuda")
    d = torch.empty((40000, 256), dtype=torch.float32, device="cuda")
    rc = f(Q.data_ptr(), X.data_ptr(), 40000, 1 << 20, 4, K.KANN_L2, K.KANN_F32, 256, ids.data_ptr(), d.data_ptr(),
           torch.cuda.current_stream().cuda_stream)
    assert rc == K.KANN_EINVAL
    with pytest.raises(ValueError):
        K.kann_exact_knn_noalloc(Q, X, 256, K.KANN_L2)
