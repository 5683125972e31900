"""Pins for the oracle's counter-based sample (Sec. 3.1: a uniform 1 % key sample)."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_published_vector(orc):
    want = [int(l) for l in open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt")) if l.strip() and l[0] != "#"]
    assert [orc.splitmix64_at(1234567, k) for k in range(5)] == want


def test_default_sample_size(orc):
    # 1 % of the input, at least 1000 keys, capped at 10M for inputs above 1B (Sec. 6)
    assert orc.default_sample_size(0) == 0
    assert orc.default_sample_size(10) == 1000
    assert orc.default_sample_size(1_000_000) == 10_000
    assert orc.default_sample_size(100_000_001) == 1_000_001
    assert orc.default_sample_size(1_000_000_000) == 10_000_000
    assert orc.default_sample_size(5_000_000_000) == 10_000_000


def _index_keyed_records(n):
    """Record i's key spells i in base 95, so enc9 recovers the sampled position."""
    recs = np.full((n, 100), ord(" "), dtype=np.uint8)
    v = np.arange(n, dtype=np.int64)
    for pos in range(8, -1, -1):
        recs[:, pos] = 32 + (v % 95)
        v //= 95
    return recs.reshape(-1)


def test_sample_positions_uniform_and_in_range(orc):
    n = 1000
    recs = _index_keyed_records(n)
    S = 200_000
    pos = orc.sample(recs, S, seed=101).astype(np.int64)
    assert pos.min() >= 0 and pos.max() < n
    counts = np.bincount(pos, minlength=n)
    # chi-square against uniform: 999 dof, mean 999, sd ~ 44.7
    chi2 = ((counts - S / n) ** 2 / (S / n)).sum()
    assert 800 < chi2 < 1200
    # with replacement, drawn from the whole input, deterministic per seed
    assert np.array_equal(pos, orc.sample(recs, S, seed=101).astype(np.int64))
    assert not np.array_equal(pos, orc.sample(recs, S, seed=102).astype(np.int64))


def test_sample_position_formula(orc, gen):
    # position k = mulhi64(SplitMix64_k(seed), n); recgen implements the same published generator independently
    n = 977
    recs = _index_keyed_records(n)
    pos = orc.sample(recs, 50, seed=5).astype(np.int64)
    for k in range(50):
        x = gen.splitmix64((5 + k * 0x9E3779B97F4A7C15) & ((1 << 64) - 1))
        assert pos[k] == (x * n) >> 64
