"""Pins for the oracle's radix classifier: equal-width ranges of the printable
key domain, the radix-based partitioning the paper compares its model-based
partitions with (Sec. 3, Sec. 3.3)."""
import numpy as np
import pytest

TOP = 95**9


def test_bins_are_equal_slices_of_the_domain(orc):
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.integers(0, TOP, 5000, dtype=np.uint64), np.array([0, 1, TOP - 1], dtype=np.uint64)])
    for log2B in (1, 6, 10, 17, 22):
        q = orc.radix_bins(x, log2B)
        want = [(int(v) << log2B) // TOP for v in x]  # Python integers: exact
        assert q.tolist() == want


def test_bins_follow_the_leading_characters(orc):
    """A key's slice is set by its first characters, whatever follows: every key
    starting with character c falls in the slices of [(c-32)/95, (c-31)/95)."""
    rng = np.random.default_rng(2)
    log2B = 12
    B = 1 << log2B
    for c in (32, 33, 80, 126):
        keys = [bytes([c]) + bytes(rng.integers(32, 127, 8).tolist()) + b"A" for _ in range(300)]
        keys += [bytes([c]) + b" " * 9, bytes([c]) + b"~" * 9]
        x = np.array([orc.encode9(k) for k in keys], dtype=np.uint64)
        q = orc.radix_bins(x, log2B).astype(np.int64)
        assert q.min() >= (c - 32) * B // 95 and q.max() <= (c - 31) * B // 95


def test_splitters_are_the_first_key_of_each_slice(orc):
    for log2B in (3, 10, 16):
        t = orc.radix_splitters(log2B)
        q = np.arange(1 << log2B)
        assert t[0] == 0 and np.all(np.diff(t.astype(np.float64)) > 0)
        assert np.array_equal(orc.radix_bins(t, log2B).astype(np.int64), q)
        assert np.all(orc.radix_bins(t[1:] - np.uint64(1), log2B).astype(np.int64) == q[1:] - 1)


def test_radix_method_sorts_and_balances_uniform_keys(orc, gen):
    n, P = 200_000, 64
    recs = gen.generate_cpu(n, gen.KeySpec("uniform", seed=3))
    log2B = orc.default_fine_log2(n, P)
    t = orc.radix_splitters(log2B)
    out, det = orc.sort_by_splitters(recs, t, log2B, P, balance=0)
    assert np.array_equal(out, orc.stable_sort(recs))
    assert np.array_equal(det["q"], orc.radix_bins(orc.encode9_records(recs), log2B))
    sizes = np.diff(det["part_off"].astype(np.int64))
    assert sizes.max() / (n / P) < 1.1  # uniform keys: equal slices hold equal counts


def test_radix_partitions_are_skew_sensitive(orc, gen):
    """On skewed keys equal-width slices are far from equal in size, while the
    RMI's partitions (paper rule) stay close to the mean -- the contrast the
    paper draws between radix and model-based partitioning."""
    n, P = 200_000, 64
    recs = gen.generate_cpu(n, gen.KeySpec("zipf", s=1.1, dup=0.05, seed=3))
    log2B = orc.default_fine_log2(n, P)
    _, det = orc.sort_by_splitters(recs, orc.radix_splitters(log2B), log2B, P, balance=0, want_out=False)
    radix = np.diff(det["part_off"].astype(np.int64))
    _, dm = orc.sort(recs, P, log2B, S=2000, seed=1, balance=0, want_detail=True)
    model = np.diff(dm["part_off"].astype(np.int64))
    assert radix.std() > 5 * model.std()
