"""Pins for the oracle's level assignment (HNSW layer law, Malkov & Yashunin
Sec. 4: level = floor(-ln U * mL), mL = 1/ln M) and its generator."""
import numpy as np
import pytest

import oracle as O
from helpers import GOLDEN


def test_splitmix64_matches_published_vector():
    with open(GOLDEN + "/splitmix64_seed0.txt") as f:
        want = [int(l, 16) for l in f if l.strip() and not l.startswith("#")]
    got = O.splitmix64_seq(0, len(want))
    assert [int(v) for v in got] == want


@pytest.mark.parametrize("M", [16, 32])
def test_level_law_chi_square(M):
    # P(level >= t) = M^-t: a chi-square test over the bins 0, 1, 2, >= 3.
    n = 400_000
    lv = O.levels(n, M, 12345).astype(int)
    p = [1 - 1 / M, 1 / M - 1 / M ** 2, 1 / M ** 2 - 1 / M ** 3, 1 / M ** 3]
    obs = [np.sum(lv == 0), np.sum(lv == 1), np.sum(lv == 2), np.sum(lv >= 3)]
    exp = [n * q for q in p]
    # merge the last bin into the previous one if its expectation is tiny
    if exp[3] < 5:
        obs[2] += obs[3]
        exp[2] += exp[3]
        obs, exp = obs[:3], exp[:3]
    chi2 = sum((o - e) ** 2 / e for o, e in zip(obs, exp))
    # 99.9% quantile of chi-square with <= 3 dof is 16.27
    assert chi2 < 16.27, (obs, exp)


def test_levels_are_a_function_of_seed_and_id():
    a = O.levels(5000, 16, 7)
    b = O.levels(5000, 16, 7)
    c = O.levels(5000, 16, 8)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, c)
    # the prefix does not depend on n (counter-based, not a stream)
    assert np.array_equal(O.levels(100, 16, 7), a[:100])
