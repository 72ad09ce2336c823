"""Pins for the oracle's storage-format encoders/decoders (IEEE binary16,
bfloat16, OCP FP8 E4M3 with a per-vector scale) against library casts."""
import numpy as np
import torch

import oracle as O


def test_f16_decode_all_codes():
    h = np.arange(65536, dtype=np.uint32).astype(np.uint16)
    ref = h.view(np.float16).astype(np.float64)
    got = O.decode_f16(h)
    same = (got == ref) | (np.isnan(got) & np.isnan(ref))
    assert same.all()


def test_f16_encode_matches_numpy_rne():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.integers(-8, 6, 20000),
                        [0.0, -0.0, 65504.0, 65520.0, 1e6, -1e6, 2.0 ** -25, 2.0 ** -24 * 1.5, np.inf]]).astype(np.float32)
    # exact halfway cases between two binary16 values
    a = np.arange(1, 2000, dtype=np.float32)
    x = np.concatenate([x, (a + 0.5).astype(np.float32) / 1024])
    got = O.encode_f16(x)
    ref = x.astype(np.float16).view(np.uint16)
    assert np.array_equal(got, ref)


def test_bf16_encode_matches_torch():
    rng = np.random.default_rng(1)
    x = (rng.standard_normal(50000) * 10.0 ** rng.integers(-20, 20, 50000)).astype(np.float32)
    got = O.encode_bf16(x)
    ref = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(got, ref)
    assert np.array_equal(O.decode_bf16(got), torch.from_numpy(x).to(torch.bfloat16).double().numpy())


def test_e4m3_decode_all_codes():
    c = np.arange(256, dtype=np.uint8)
    ref = torch.from_numpy(c).view(torch.float8_e4m3fn).double().numpy()
    got = O.decode_e4m3(c)
    same = (got == ref) | (np.isnan(got) & np.isnan(ref))
    assert same.all()


def test_e4m3_rows_match_torch_cast_and_error_bound():
    rng = np.random.default_rng(2)
    X = (rng.standard_normal((500, 64)) * 10.0 ** rng.integers(-3, 3, (500, 1))).astype(np.float32)
    X[0] = 0.0
    codes, s = O.encode_e4m3_rows(X)
    s_ref = (np.abs(X).max(1) / np.float32(448.0)).astype(np.float32)
    assert np.array_equal(s, s_ref)
    assert np.all(codes[0] == 0) and s[0] == 0
    t = (X[1:] / s_ref[1:, None]).astype(np.float32)  # IEEE float32 division
    ref = torch.from_numpy(t).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    assert np.array_equal(codes[1:], ref)
    # reconstruction error: |x - s * code| <= max(2^-4 |x|, s * 2^-10)
    rec = O.decode_e4m3(codes) * s.astype(np.float64)[:, None]
    err = np.abs(rec - X)
    bound = np.maximum(2.0 ** -4 * np.abs(X), s.astype(np.float64)[:, None] * 2.0 ** -10)
    assert np.all(err <= bound * (1 + 1e-12))
