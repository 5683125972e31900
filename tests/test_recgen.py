"""The synthetic record generator: format, distributions, determinism."""
import numpy as np


def test_record_format(gen):
    n = 5000
    r = gen.generate_cpu(n, gen.KeySpec("uniform", seed=1)).reshape(n, 100)
    assert r[:, :10].min() >= 0x20 and r[:, :10].max() <= 0x7E
    for i in (0, 1, 4999):
        assert bytes(r[i, 10:42]) == f"{i:032X}".encode()
        assert bytes(r[i, 42:98]) == bytes(65 + (i + j) % 26 for j in range(56))
        assert bytes(r[i, 98:100]) == b"\r\n"


def test_chunks_and_threads_agree(gen):
    spec = gen.KeySpec("zipf", s=1.1, dup=0.05, seed=3)
    full = gen.generate_cpu(200000, spec, threads=4)
    part = gen.generate_cpu(200000, spec, i0=123456, count=1000, threads=1)
    assert np.array_equal(full[123456 * 100:124456 * 100], part)


def test_uniform_histogram_spread(gen):
    """1000 equal-width bins of the leading key bytes: std/mean ~ sqrt(1000/N) for uniform keys
    (the paper's uniform data shows 0.14 % at its size; Sec. 7.3)."""
    n = 2_000_000
    r = gen.generate_cpu(n, gen.KeySpec("uniform", seed=2)).reshape(n, 100)
    v = np.zeros(n, dtype=np.int64)
    for c in range(4):
        v = v * 95 + (r[:, c].astype(np.int64) - 32)
    bins = np.bincount(v * 1000 // 95**4, minlength=1000)
    rel = bins.std() / bins.mean()
    assert abs(rel / np.sqrt(1000 / n) - 1) < 0.15


def test_zipf_rank_frequencies(gen):
    n = 400_000
    spec = gen.KeySpec("zipf", s=1.3, dup=0.0, seed=5)
    r = gen.generate_cpu(n, spec).reshape(n, 100)
    _, perm, _ = spec.tables()
    perm = perm.reshape(10, 95)
    w = np.arange(1, 96, dtype=np.float64) ** -1.3
    w /= w.sum()
    for pos in (0, 9):
        counts = np.bincount(r[:, pos].astype(np.int64) - 32, minlength=95)
        by_rank = counts[perm[pos]] / n
        assert np.allclose(by_rank[:5], w[:5], rtol=0.03)


def test_duplicate_fraction(gen):
    n = 300_000
    r = gen.generate_cpu(n, gen.KeySpec("uniform", dup=0.10, seed=6)).reshape(n, 100)
    keys = r[:, :10].copy().view("S10").ravel()
    _, counts = np.unique(keys, return_counts=True)
    dup_records = n - counts.size  # records whose key already appeared
    # a copy of a record that is itself a copy brings a new key, so about d(1-d) of records repeat one
    assert abs(dup_records / n - 0.10 * 0.90) < 0.005


def test_prefix_skew_follows_the_table_rule(gen):
    """The paper's skewed data (Sec. 7.1): the leading key bytes of record i are
    entry log2(i) mod 128 of a table of 128 six-byte entries.  Records sharing
    floor(log2 i) share their 6-byte prefix, so the prefixes of an n-record set
    take floor(log2(n-1)) + 1 values, group k holding 2^k records; the last 4
    key bytes stay uniform and the payload is unchanged."""
    n = 1 << 16
    r = gen.generate_cpu(n, gen.KeySpec("prefix", seed=8)).reshape(n, 100)
    assert r[:, :10].min() >= 0x20 and r[:, :10].max() <= 0x7E
    pre = r[:, :6].copy().view("S6").ravel()
    assert pre[0] == pre[1]
    for k in range(16):
        grp = pre[1 << k:1 << (k + 1)]
        assert np.all(grp == grp[0])  # one entry per group
        if k:
            assert grp[0] != pre[(1 << (k - 1))]  # a new entry per group (128 random entries differ)
    assert np.unique(pre).size == 16
    # bytes 6-9: uniform over the printable characters
    c = np.bincount(r[:, 6:10].ravel().astype(np.int64) - 32, minlength=95)
    assert c.min() > 0.8 * c.mean() and c.max() < 1.2 * c.mean()
    assert bytes(r[12345, 10:42]) == f"{12345:032X}".encode()


def test_prefix_skew_histogram_is_spiky(gen):
    """1000 equal-width bins of the leading key characters: the table rule puts
    whole groups of 2^k records into single bins, far from the uniform data's
    sqrt(1000/N) spread (the paper's Fig. 3 contrasts 0.14 % with 65.65 %)."""
    n = 1_000_000
    r = gen.generate_cpu(n, gen.KeySpec("prefix", seed=8)).reshape(n, 100)
    v = np.zeros(n, dtype=np.int64)
    for c in range(4):
        v = v * 95 + (r[:, c].astype(np.int64) - 32)
    bins = np.bincount(v * 1000 // 95**4, minlength=1000)
    assert bins.max() >= n // 4 and bins.std() / bins.mean() > 5
