"""Pins for the oracle's partition-and-concatenate sort.

The result has a plain definition: every record, stably sorted by memcmp on
the 10-byte key (Sec. 7.1 methodology).  Any monotone partition (Eq. 1) that
keeps equal keys together, each part sorted and the parts concatenated
(Sec. 3.5), reaches exactly that result, whatever the model.  The pins: brute
force against Python's stable sort on tiny inputs, P = 1, invariants of the
partition step, the paper's partition rule and the refined cut rule.
"""
import itertools

import numpy as np
import pytest

R = 100


def _records(keys):
    """Records with the given 10-byte keys and their index in the payload."""
    n = len(keys)
    recs = np.zeros((n, R), dtype=np.uint8)
    for i, k in enumerate(keys):
        recs[i, :10] = np.frombuffer(k, dtype=np.uint8)
        recs[i, 10:42] = np.frombuffer(f"{i:032X}".encode(), dtype=np.uint8)
        recs[i, 42:98] = [65 + (i + j) % 26 for j in range(56)]
        recs[i, 98:100] = [13, 10]
    return recs.reshape(-1)


def _python_stable(recs):
    rows = recs.reshape(-1, R)
    order = sorted(range(len(rows)), key=lambda i: bytes(rows[i, :10]))  # list.sort is stable
    return rows[order].reshape(-1)


def test_brute_force_tiny(orc):
    alphabet = [b" " + b"M" * 8 + b" ", b" " + b"M" * 8 + b"~", b"~" + b" " * 9, b"A" * 10]
    cases = 0
    for n in range(0, 5):
        for keys in itertools.product(alphabet, repeat=n):
            recs = _records(list(keys))
            want = _python_stable(recs)
            for P, log2B, bal in ((1, 6, 1), (2, 6, 0), (4, 6, 1), (64, 6, 0)):
                got = orc.sort(recs, P, log2B, S=8, seed=3, balance=bal, T=1)
                assert np.array_equal(got, want), (keys, P, bal)
                cases += 1
    assert cases > 1000


@pytest.mark.parametrize("seed", range(20))
def test_random_small_sets(orc, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 300))
    alpha = rng.integers(32, 127, size=int(rng.integers(1, 6)), dtype=np.uint8)
    keys = [bytes(rng.choice(alpha, size=10)) for _ in range(n)]
    recs = _records(keys)
    want = _python_stable(recs)
    P = int(2 ** rng.integers(0, 6))
    got = orc.sort(recs, P, 8, S=int(rng.integers(1, 100)), seed=seed, balance=int(seed % 2),
                   T=int(rng.integers(1, 20)))
    assert np.array_equal(got, want)
    assert orc.validate(recs, got) == 0


def test_p1_equals_plain_stable_sort(orc, gen):
    recs = gen.generate_cpu(20000, gen.KeySpec("zipf", s=1.3, dup=0.2, seed=9))
    want = _python_stable(recs)
    assert np.array_equal(orc.stable_sort(recs), want)
    assert np.array_equal(orc.sort(recs, 1, 6, S=1000, seed=1), want)


@pytest.mark.parametrize("spec", [("uniform", 1.1, 0.0), ("zipf", 1.1, 0.05), ("zipf", 1.3, 0.10)])
@pytest.mark.parametrize("balance", [0, 1])
def test_partition_invariants(orc, gen, spec, balance):
    kind, s, d = spec
    n, P, log2B = 60000, 64, 12
    recs = gen.generate_cpu(n, gen.KeySpec(kind, s=s, dup=d, seed=21))
    out, det = orc.sort(recs, P, log2B, S=1000, seed=7, balance=balance, want_detail=True)
    assert np.array_equal(out, _python_stable(recs))
    off = det["part_off"].astype(np.int64)
    pid = det["pid"].astype(np.int64)
    q = det["q"].astype(np.int64)
    assert off[0] == 0 and off[-1] == n and np.all(np.diff(off) >= 0)
    assert np.array_equal(np.diff(off), np.bincount(pid, minlength=P))  # offsets = exclusive sum of sizes
    assert np.array_equal(det["bin_counts"].astype(np.int64), np.bincount(q, minlength=1 << log2B))
    keys = recs.reshape(-1, R)[:, :10]
    kb = [bytes(k) for k in keys]
    # Eq. 1: every key of partition j <= every key of partition j+1; equal keys share a partition
    lo = {}
    hi = {}
    for i in range(n):
        p = pid[i]
        lo[p] = min(lo.get(p, kb[i]), kb[i])
        hi[p] = max(hi.get(p, kb[i]), kb[i])
    ps = sorted(lo)
    for a, b in zip(ps, ps[1:]):
        assert hi[a] < lo[b]
    first = {}
    for i in range(n):
        assert first.setdefault(kb[i], pid[i]) == pid[i]
    # the output holds partition p's records at [off_p, off_{p+1})
    out_rows = out.reshape(-1, R)
    idx = np.array([int(bytes(r[26:42]), 16) for r in out_rows])
    assert np.array_equal(pid[idx], np.repeat(np.arange(P), np.diff(off)))


def test_paper_rule_is_floor_P_F(orc, gen):
    n, P, log2B, S, seed = 30000, 16, 10, 500, 4
    recs = gen.generate_cpu(n, gen.KeySpec("zipf", s=1.1, dup=0.05, seed=2))
    _, det = orc.sort(recs, P, log2B, S=S, seed=seed, balance=0, want_detail=True)
    smp = np.sort(orc.sample(recs, S, seed))
    F, _ = orc.Rmi(smp).eval(orc.encode9_records(recs))
    assert np.array_equal(det["q"], np.minimum((1 << log2B) - 1, np.floor(F * (1 << log2B))).astype(np.uint32))
    assert np.array_equal(det["pid"], np.minimum(P - 1, np.floor(F * P)).astype(np.uint32))


def test_refined_cuts_are_closest_boundaries(orc, gen):
    n, P, log2B = 50000, 32, 11
    recs = gen.generate_cpu(n, gen.KeySpec("zipf", s=1.3, dup=0.1, seed=8))
    _, det = orc.sort(recs, P, log2B, S=800, seed=2, balance=1, want_detail=True)
    C = np.concatenate([[0], np.cumsum(det["bin_counts"].astype(np.int64))])
    cuts = det["cuts"].astype(np.int64)
    assert cuts[0] == 0 and cuts[-1] == 1 << log2B and np.all(np.diff(cuts) >= 0)
    for p in range(1, P):
        dist = np.abs(P * C - p * n)
        assert cuts[p] == int(np.argmin(dist))  # argmin returns the first (smallest) minimiser
    sizes = np.diff(det["part_off"].astype(np.int64))
    # each cut is within half of the largest fine bin of its ideal position
    assert sizes.max() <= n / P + det["bin_counts"].max()


def test_refined_rule_balances_better_than_paper_rule(orc, gen):
    n, P, log2B = 200000, 64, 14
    recs = gen.generate_cpu(n, gen.KeySpec("zipf", s=1.1, dup=0.05, seed=3))
    _, d0 = orc.sort(recs, P, log2B, S=2000, seed=1, balance=0, want_detail=True)
    _, d1 = orc.sort(recs, P, log2B, S=2000, seed=1, balance=1, want_detail=True)
    r0 = np.diff(d0["part_off"].astype(np.int64)).max() / (n / P)
    r1 = np.diff(d1["part_off"].astype(np.int64)).max() / (n / P)
    assert r1 < r0 and r1 < 1.15


def test_validator_catches_planted_faults(orc, gen):
    recs = gen.generate_cpu(3000, gen.KeySpec("zipf", s=1.3, dup=0.3, seed=4))
    good = orc.stable_sort(recs)
    assert orc.validate(recs, good) == 0
    rows = good.reshape(-1, R).copy()
    bad = rows.copy()
    bad[[10, 2000]] = bad[[2000, 10]]
    assert orc.validate(recs, bad.reshape(-1)) & 1
    bad = rows.copy()
    bad[5, 50] ^= 1
    assert orc.validate(recs, bad.reshape(-1)) & 2
    bad = rows.copy()
    bad[7] = bad[8]
    assert orc.validate(recs, bad.reshape(-1)) & 2
    keys = [bytes(r[:10]) for r in rows]
    i = next(i for i in range(len(keys) - 1) if keys[i] == keys[i + 1])
    bad = rows.copy()
    bad[[i, i + 1]] = bad[[i + 1, i]]
    assert orc.validate(recs, bad.reshape(-1)) == 4


def test_empty_input(orc):
    out = orc.sort(np.zeros(0, dtype=np.uint8), 4, 6, S=0, seed=1)
    assert out.size == 0
