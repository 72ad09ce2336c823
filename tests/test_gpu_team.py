"""Search teams: kann_search_opts.team = 2 or 4 runs one query per CTA of that
many warps.  Warp 0 runs the HNSW search (Malkov & Yashunin Alg. 2 / 5, the
index of kANNolo Sec. 2) and at every distance and re-rank batch each warp
evaluates one slice of the candidates, every row by one lane group exactly as
in the one-warp search.  So the results -- ids, distances, status words and
work counters -- equal the one-warp search's bit for bit, over storage
formats, both row-tiling forms, both metrics, the re-rank, mixed k/ef
batches, the persistent launch and the sparse back-end; and on integer data
they equal the oracle's."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2501_06121_b300 import datagen as G
from paper_2501_06121_b300 import kann as K

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run(idx, Q, k, ef, **o):
    n = len(Q)
    st = torch.zeros(n, dtype=torch.int32, device="cuda")
    cnt = torch.zeros((n, 4), dtype=torch.int32, device="cuda")
    ids, d = K.kann_search_ex(idx, dev(Q), k, ef, status=st, counters=cnt, **o)
    torch.cuda.synchronize()
    return ids.cpu().numpy(), d.cpu().numpy(), st.cpu().numpy(), cnt.cpu().numpy()


def same(a, b):
    return all(np.array_equal(x, y) for x, y in zip(a, b))


@pytest.fixture(scope="module")
def int128(int_small):
    # integer rows 0..255 (every FP32/FP16 distance exact), 20k x 128, L2,
    # the oracle's graph
    X, Q, g = int_small
    return X, Q, g


@pytest.mark.parametrize("dtype", [K.KANN_F32, K.KANN_F16, K.KANN_E4M3])
@pytest.mark.parametrize("team", [2, 4])
def test_team_equals_one_warp(int128, dtype, team):
    X, Q, g = int128
    Xd = dev(X)
    data, scale = (Xd, None) if dtype == K.KANN_F32 else K.kann_quantize(Xd, dtype)
    idx = K.kann_index_upload(K.graph_to_device(g.arrays()), vectors=data, dtype=dtype, scale=scale, rerank=Xd)
    for ef, rr in ((16, 0), (64, -1), (300, 100)):
        one = run(idx, Q, 10, ef, rerank=rr)
        assert same(run(idx, Q, 10, ef, rerank=rr, team=team), one), (ef, rr)
    # a visited table small enough to forget: the forgetting is per query,
    # so it is the same in both forms
    one = run(idx, Q, 10, 128, hash_bits=6)
    assert same(run(idx, Q, 10, 128, hash_bits=6, team=team), one)


def test_team_equals_oracle_on_integer_data(int128):
    X, Q, g = int128
    idx = K.kann_index_upload(K.graph_to_device(g.arrays()), vectors=dev(X))
    gi, gd, _, cnt = run(idx, Q, 10, 64, team=4)
    oi, od, ocnt = O.search_dense(g, X, Q, 10, 64, O.L2)
    assert np.array_equal(gi, oi)
    assert np.array_equal(gd.astype(np.float64), od)


@pytest.mark.parametrize("team", [2, 4])
def test_team_general_form_768_ip(team):
    # d = 768 FP32 inner product: the general kernel (8 chunks per lane)
    X, Q = G.vmf_mixture(4000, 120, d=768, clusters=16, kappa=50.0, seed=43, concentration=0.1)
    g = K.kann_hnsw_build_dense(X, K.KANN_IP, 16, 80, 43)
    idx = K.kann_index_upload(K.graph_to_device(g), vectors=dev(X), metric=K.KANN_IP)
    for ef in (32, 200):
        assert same(run(idx, Q, 10, ef, team=team), run(idx, Q, 10, ef))


@pytest.mark.parametrize("team", [2, 4])
def test_team_mixed_batch_and_persistent(int128, team):
    X, Q, g = int128
    Xd = dev(X)
    h, _ = K.kann_quantize(Xd, K.KANN_F16)
    idx = K.kann_index_upload(K.graph_to_device(g.arrays()), vectors=h, dtype=K.KANN_F16, rerank=Xd)
    rng = np.random.default_rng(5)
    n = len(Q)
    ks = dev(rng.choice([10, 100], n).astype(np.int32))
    efs = dev(rng.integers(64, 513, n).astype(np.int32))
    a = K.kann_search_batch(idx, dev(Q), ks, efs, kmax=100, efmax=512, rerank=-1)
    ctr = torch.zeros(1, dtype=torch.int32, device="cuda")
    b = K.kann_search_batch(idx, dev(Q), ks, efs, kmax=100, efmax=512, rerank=-1, team=team, work_counter=ctr)
    c = K.kann_search_batch(idx, dev(Q), ks, efs, kmax=100, efmax=512, rerank=-1, team=team)
    torch.cuda.synchronize()
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    assert torch.equal(a[0], c[0]) and torch.equal(a[1], c[1])
    assert int(ctr.item()) >= n


@pytest.mark.parametrize("team", [2, 4])
def test_team_sparse_equals_one_warp(team):
    base, qs = G.sparse_zipf(4000, 300, vocab=3000, lam_doc=40, lam_query=12, seed=47)
    g = O.build_sparse(*base, M=16, efC=100, seed=47)
    sp = dict(indptr=dev(base[0]), terms=dev(base[1].view(np.int16)), weights=dev(base[2]), vocab=3000)
    idx = K.kann_index_upload(K.graph_to_device(g.arrays()), sparse=sp)
    q = (dev(qs[0]), dev(qs[1].view(np.int16)), dev(qs[2]))
    for ef in (32, 128):
        out = []
        for t in (0, team):
            st = torch.zeros(len(qs[0]) - 1, dtype=torch.int32, device="cuda")
            cnt = torch.zeros((len(qs[0]) - 1, 4), dtype=torch.int32, device="cuda")
            i, d = K.kann_search_sparse(idx, *q, 10, ef, status=st, counters=cnt, team=t)
            torch.cuda.synchronize()
            out.append((i.cpu().numpy(), d.cpu().numpy(), st.cpu().numpy(), cnt.cpu().numpy()))
        assert same(out[0], out[1]), ef


def test_team_option_rejections(int128):
    X, Q, g = int128
    idx = K.kann_index_upload(K.graph_to_device(g.arrays()), vectors=dev(X))
    for bad in (dict(team=3), dict(team=8), dict(team=-1), dict(team=2, expand=2)):
        with pytest.raises(K.KannError):
            K.kann_search_ex(idx, dev(Q[:4]), 10, 64, **bad)
        assert K.kann_search_workspace_bytes(idx, 4, 10, 64, **bad) == 0
    assert K.kann_search_workspace_bytes(idx, 4, 10, 64, team=4) > 0
