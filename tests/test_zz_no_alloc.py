"""kann_exact_knn_noalloc: exact k-NN for callers that cannot allocate device
memory (their device memory is owned by another allocator, or cudaMalloc's
implicit synchronisation is not allowed on their path).  It must return what
kann_exact_knn returns with caller-provided scratch, call after call, while
reusing one static scratch array -- on the CUDA-core path (FP32, or k > 32)
and on the tensor-core path (BF16/FP16, k <= 32), whose norms, thresholds
and error word also live in that array.  This file is collected last on
purpose."""
import ctypes

import numpy as np
import pytest
import torch

import oracle as O
from paper_2501_06121_b300 import kann as K

pytestmark = pytest.mark.gpu

_TORCH = {K.KANN_F32: torch.float32, K.KANN_F16: torch.float16, K.KANN_BF16: torch.bfloat16}


def _entry():
    f = K._lib().kann_exact_knn_noalloc
    P, I = ctypes.c_void_p, ctypes.c_int
    f.restype = I
    f.argtypes = [P, P, I, ctypes.c_int64, I, I, I, I, P, P, P]
    return f


def _call(f, Q, X, k, metric, dtype):
    nq = Q.shape[0]
    ids = torch.full((nq, k), -7, dtype=torch.int32, device="cuda")
    d = torch.full((nq, k), -7.0, dtype=torch.float32, device="cuda")
    rc = f(Q.data_ptr(), X.data_ptr(), nq, X.shape[0], Q.shape[1], metric, dtype, k, ids.data_ptr(),
           d.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == K.KANN_OK, K._lib().kann_status_str(rc)
    torch.cuda.synchronize()
    return ids.cpu().numpy(), d.cpu().numpy()


@pytest.mark.parametrize("dtype", [K.KANN_F32, K.KANN_BF16, K.KANN_F16])
@pytest.mark.parametrize("metric", [K.KANN_L2, K.KANN_IP])
def test_noalloc_equals_workspace_entry_point_twice_in_a_row(metric, dtype):
    f = _entry()
    rng = np.random.default_rng(11 + metric + 2 * dtype)
    X = torch.from_numpy(rng.standard_normal((40000, 128)).astype(np.float32)).cuda().to(_TORCH[dtype])
    # the second call has other sizes and reuses scratch holding the first
    # call's lists (and, on the tensor-core path, its norms and thresholds)
    for call, (nq, k) in enumerate([(700, 10), (333, 32)]):
        Q = torch.from_numpy(rng.standard_normal((nq, 128)).astype(np.float32)).cuda().to(_TORCH[dtype])
        ri, rd = K.kann_exact_knn(Q, X, k, metric, dtype=dtype)
        torch.cuda.synchronize()
        ri, rd = ri.cpu().numpy(), rd.cpu().numpy()
        gi, gd = _call(f, Q, X, k, metric, dtype)
        # the same kernels run on the same inputs: ids equal, distances within
        # the 1e-5 relative tolerance of the other tests (in fact identical)
        assert np.array_equal(gi, ri), call
        assert np.all(np.abs(gd - rd) <= 1e-5 * np.abs(rd)), call


@pytest.mark.parametrize("dtype", [K.KANN_F32, K.KANN_BF16])
def test_noalloc_matches_oracle_on_integer_data(dtype):
    # integers 0..255 at d = 128: every norm and dot product is an integer below
    # 2^24, exact in FP32 and in BF16 inputs, so ids and distances equal the
    # FP64 oracle's exact k-NN (ties to the lower id) bit for bit
    f = _entry()
    rng = np.random.default_rng(5)
    X = rng.integers(0, 256, (20000, 128)).astype(np.float32)
    Q = rng.integers(0, 256, (150, 128)).astype(np.float32)
    ei, ed = O.exact_dense(X, Q, 16, O.L2)
    Xd = torch.from_numpy(X).cuda().to(_TORCH[dtype])
    Qd = torch.from_numpy(Q).cuda().to(_TORCH[dtype])
    for _ in range(2):
        gi, gd = _call(f, Qd, Xd, 16, K.KANN_L2, dtype)
        assert np.array_equal(gi, ei)
        assert np.array_equal(gd.astype(np.float64), ed)


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


def test_noalloc_rejects_misaligned_pointers_before_launch():
    # a view that starts one FP32 element into its buffer is 4-byte aligned only
    f = _entry()
    buf = torch.zeros(1000 * 128 + 4, dtype=torch.float32, device="cuda")
    X = buf[1:1 + 1000 * 128].view(1000, 128)
    Q = torch.zeros((10, 128), dtype=torch.float32, device="cuda")
    ids = torch.empty((10, 5), dtype=torch.int32, device="cuda")
    d = torch.empty((10, 5), dtype=torch.float32, device="cuda")
    rc = f(Q.data_ptr(), X.data_ptr(), 10, 1000, 128, K.KANN_L2, K.KANN_F32, 5, ids.data_ptr(), d.data_ptr(),
           torch.cuda.current_stream().cuda_stream)
    assert rc == K.KANN_EINVAL
