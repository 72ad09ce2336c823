"""Tensor-core (tcgen05) exact k-NN against the FP64 oracle's brute force.

BF16/FP16 inputs with k <= 32 take the tensor-core path: S = Q X^T in FP32
in tensor memory, distances ||x||^2 - 2 q.x + ||q||^2 (L2) or -q.x (IP),
fused top-k.  On integer data small enough that every product and partial
sum is an exact FP32 integer, the results must equal the oracle bit for bit;
on real-valued data the oracle runs on the same BF16-rounded values and
distances must agree within 1e-5 of sum |terms|."""
import numpy as np
import pytest
import torch

import oracle as O
from helpers import id_set_match_fraction
from paper_2501_06121_b300 import kann as K

pytestmark = pytest.mark.gpu


def to16(a, dtype):
    t = torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    return t.to(torch.bfloat16 if dtype == K.KANN_BF16 else torch.float16)


@pytest.mark.parametrize("nq,nb,d,hi", [(300, 5000, 128, 256), (1, 1000, 64, 256), (129, 777, 768, 64),
                                        (1000, 20000, 128, 256), (5, 300, 16, 256), (7, 20, 32, 256),
                                        (40, 5, 64, 256), (300, 5000, 256, 64), (200, 3000, 192, 64)])
@pytest.mark.parametrize("dtype", [K.KANN_BF16, K.KANN_F16])
def test_tc_exact_integer_data_bit_exact(nq, nb, d, hi, dtype):
    rng = np.random.default_rng(nq + nb + d)
    X = rng.integers(0, hi, (nb, d)).astype(np.float32)
    Q = rng.integers(0, hi, (nq, d)).astype(np.float32)
    k = min(10, nb)
    gi, gd = K.kann_exact_knn(to16(Q, dtype), to16(X, dtype), k, K.KANN_L2, dtype=dtype)
    torch.cuda.synchronize()
    oi, od = O.exact_dense(X, Q, k, O.L2)
    assert np.array_equal(gi.cpu().numpy(), oi)
    assert np.array_equal(gd.cpu().numpy().astype(np.float64), od)


@pytest.mark.parametrize("k", [1, 10, 32])
@pytest.mark.parametrize("metric", [K.KANN_L2, K.KANN_IP])
def test_tc_exact_ties_keep_lowest_ids(k, metric):
    # a base of a few distinct rows repeated: every query's k-th distance is
    # shared by hundreds of rows, and the (distance, id) order keeps the
    # lowest ids -- the starting threshold of each scan must let them all in
    rng = np.random.default_rng(11 + k)
    proto = rng.integers(0, 64, (3, 64)).astype(np.float32)
    X = proto[rng.integers(0, 3, 6000)]
    Q = rng.integers(0, 64, (70, 64)).astype(np.float32)
    gi, gd = K.kann_exact_knn(to16(Q, K.KANN_BF16), to16(X, K.KANN_BF16), k, metric, dtype=K.KANN_BF16)
    torch.cuda.synchronize()
    oi, od = O.exact_dense(X, Q, k, metric)
    assert np.array_equal(gi.cpu().numpy(), oi)
    assert np.array_equal(gd.cpu().numpy().astype(np.float64), od)


@pytest.mark.parametrize("k", [1, 10, 32])
@pytest.mark.parametrize("metric", [K.KANN_L2, K.KANN_IP])
def test_tc_exact_real_data(k, metric):
    rng = np.random.default_rng(k + 7 * metric)
    Xb = to16(rng.standard_normal((30000, 128)), K.KANN_BF16)
    Qb = to16(rng.standard_normal((500, 128)), K.KANN_BF16)
    X = Xb.float().cpu().numpy()
    Q = Qb.float().cpu().numpy()
    gi, gd = K.kann_exact_knn(Qb, Xb, k, metric, dtype=K.KANN_BF16)
    torch.cuda.synchronize()
    gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
    oi, od = O.exact_dense(X, Q, k, metric)
    assert id_set_match_fraction(gi, oi) >= 0.99
    ref = O.dist_dense(X, Q, gi, metric)
    if metric == K.KANN_L2:
        mag = np.einsum("qd,qkd->qk", Q.astype(np.float64) ** 2, np.ones_like(X[gi], np.float64)) + \
            np.einsum("qkd->qk", X.astype(np.float64)[gi] ** 2) + \
            2 * np.einsum("qd,qkd->qk", np.abs(Q.astype(np.float64)), np.abs(X.astype(np.float64)[gi]))
    else:
        mag = np.einsum("qd,qkd->qk", np.abs(Q.astype(np.float64)), np.abs(X.astype(np.float64)[gi]))
    assert np.all(np.abs(gd - ref) <= 1e-5 * np.maximum(np.abs(ref), mag))


def test_large_k_falls_back_to_cuda_cores():
    rng = np.random.default_rng(3)
    X = rng.integers(0, 256, (4000, 64)).astype(np.float32)
    Q = rng.integers(0, 256, (50, 64)).astype(np.float32)
    gi, gd = K.kann_exact_knn(to16(Q, K.KANN_BF16), to16(X, K.KANN_BF16), 40, K.KANN_L2, dtype=K.KANN_BF16)
    torch.cuda.synchronize()
    oi, od = O.exact_dense(X, Q, 40, O.L2)
    assert np.array_equal(gi.cpu().numpy(), oi)


# ------------------------------------------------------------------ argument checks
def test_exact_knn_rejects_mismatched_arguments_before_launch():
    # each of these would make the kernel read or write past a buffer's end
    Q = torch.zeros((10, 64), dtype=torch.float32, device="cuda")
    X = torch.zeros((500, 64), dtype=torch.float32, device="cuda")
    with pytest.raises(ValueError):  # half-precision data under the FP32 default
        K.kann_exact_knn(Q.half(), X.half(), 5, K.KANN_L2)
    with pytest.raises(ValueError):  # dtype says BF16, tensors are FP16
        K.kann_exact_knn(Q.half(), X.half(), 5, K.KANN_L2, dtype=K.KANN_BF16)
    with pytest.raises(ValueError):  # base rows of another width
        K.kann_exact_knn(Q, X[:, :32].contiguous(), 5, K.KANN_L2)
    with pytest.raises(ValueError):  # ids too small for [nq, k]
        K.kann_exact_knn(Q, X, 5, K.KANN_L2, ids=torch.empty((10, 4), dtype=torch.int32, device="cuda"))
    with pytest.raises(ValueError):  # dists of the wrong type
        K.kann_exact_knn(Q, X, 5, K.KANN_L2, dists=torch.empty((10, 5), dtype=torch.float16, device="cuda"))
    with pytest.raises(ValueError):
        K.kann_exact_knn_noalloc(Q.bfloat16(), X.bfloat16(), 5, K.KANN_L2, dtype=K.KANN_F16)


@pytest.mark.parametrize("which", ["queries", "base"])
def test_exact_knn_rejects_misaligned_rows(which):
    # a tensor that starts one element into its buffer: the library returns
    # KANN_EINVAL instead of issuing misaligned 16-byte loads
    buf = torch.zeros(500 * 64 + 8, dtype=torch.float32, device="cuda")
    off = buf[1:1 + 500 * 64].view(500, 64)
    Q = off[:10].contiguous() if which == "base" else off[:10]
    X = off if which == "base" else torch.zeros((500, 64), dtype=torch.float32, device="cuda")
    with pytest.raises(K.KannError) as e:
        K.kann_exact_knn(Q, X, 5, K.KANN_L2)
    assert e.value.status == K.KANN_EINVAL
