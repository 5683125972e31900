"""Pins for the oracle's RMI CDF model (Sec. 3.1 of the paper).

Every node's least-squares fit is checked against numpy.polyfit (an
independent library least-squares routine) on the same points.  The tree's
structure is checked against its split rule; the monotonicity Eq. 1 needs,
the [0, 1] range, the equi-depth leaves the paper describes, and degenerate
samples are checked directly.
"""
import numpy as np
import pytest

T = 16


def _sample(kind, S, seed=3):
    rng = np.random.default_rng(seed)
    top = 95**9
    if kind == "uniform":
        x = rng.integers(0, top, size=S, dtype=np.uint64)
    elif kind == "skew":
        # product-Zipf digits in base 95, like the skewed workloads
        ranks = np.minimum(rng.zipf(1.2, size=(S, 9)) - 1, 94).astype(np.uint64)
        x = np.zeros(S, dtype=np.uint64)
        for c in range(9):
            x = x * np.uint64(95) + ranks[:, c]
    elif kind == "dups":
        x = rng.integers(0, 50, size=S).astype(np.uint64) * np.uint64(95**6)
    return np.sort(x)


KINDS = ["uniform", "skew", "dups"]


@pytest.mark.parametrize("kind", KINDS)
def test_every_node_matches_library_least_squares(orc, kind):
    x = _sample(kind, 20000)
    m = orc.Rmi(x, T)
    checked = 0
    for i in range(len(m)):
        s, e = int(m.s_[i]), int(m.e_[i])
        if e - s == 0:
            continue
        base, sh = int(m.base[i]), int(m.shift[i])
        assert base == int(x[s])
        span = int(x[e - 1]) - base
        assert (span >> sh) < 2**32 and (sh == 0 or (span >> (sh - 1)) >= 2**32)
        u = np.array([(int(v) - base) >> sh for v in x[s:e]], dtype=np.float64)
        r = np.arange(e - s, dtype=np.float64)
        if e - s >= 3 and np.ptp(u) > 0:
            ls, li = np.polyfit(u, r, 1)
            if ls > 1e-12:
                assert m.gamma[i] == pytest.approx(ls, rel=1e-6)
                assert m.delta[i] == pytest.approx(li, rel=1e-6, abs=1e-6 * (e - s))
                checked += 1
                continue
        if np.ptp(u) == 0:
            assert m.gamma[i] == 0 and m.delta[i] == pytest.approx((e - s - 1) / 2)
    assert checked > 100 or kind == "dups"


@pytest.mark.parametrize("kind", KINDS)
def test_tree_structure_follows_split_rule(orc, kind):
    x = _sample(kind, 20000)
    S = x.size
    m = orc.Rmi(x, T)
    assert m.s_[0] == 0 and m.e_[0] == S and m.depth[0] == 0
    seen_children = 1
    for i in range(len(m)):
        s, e, f = int(m.s_[i]), int(m.e_[i]), int(m.fanout[i])
        n = e - s
        if f:
            assert n > 2 * T and x[s] < x[e - 1] and f == -(-n // T)
            c0 = int(m.child0[i])
            assert c0 == seen_children  # breadth-first numbering
            seen_children += f
            kids = range(c0, c0 + f)
            assert int(m.s_[c0]) == s and int(m.e_[c0 + f - 1]) == e
            for a, b in zip(kids, list(kids)[1:]):
                assert m.e_[a] == m.s_[b]
            assert all(m.depth[k] == m.depth[i] + 1 for k in kids)
            assert m.scale[i] == f / n
        else:
            assert m.lo[i] == s / S and m.hi[i] == e / S
    assert seen_children == len(m)
    # every sample point is routed to the leaf whose rank range holds it
    _, leaf = m.eval(x)
    k = np.arange(S)
    assert np.all((m.s_[leaf] <= k) & (k < m.e_[leaf]))


@pytest.mark.parametrize("kind", KINDS)
def test_monotone_and_in_unit_interval(orc, kind):
    x = _sample(kind, 20000)
    m = orc.Rmi(x, T)
    rng = np.random.default_rng(11)
    probe = np.sort(np.concatenate([x, rng.integers(0, 95**9, size=200000, dtype=np.uint64),
                                    x + np.uint64(1), x - np.minimum(x, np.uint64(1)),
                                    np.array([0, 95**9 - 1], dtype=np.uint64)]))
    F, leaf = m.eval(probe)
    assert np.all(np.diff(F) >= 0)
    assert F.min() >= 0 and F.max() <= 1
    # leaves are visited in rank order along the key axis
    assert np.all(np.diff(m.s_[leaf].astype(np.int64)) >= 0)


def test_skewed_leaves_are_equi_depth(orc):
    """Dense regions get more nodes: leaves hold at most 2T sample keys unless all their keys are equal."""
    x = _sample("skew", 50000, seed=5)
    m = orc.Rmi(x, T)
    leaves = np.nonzero(m.fanout == 0)[0]
    n = (m.e_[leaves] - m.s_[leaves]).astype(np.int64)
    big = leaves[n > 2 * T]
    for i in big:
        s, e = int(m.s_[i]), int(m.e_[i])
        assert x[s] == x[e - 1] or m.depth[i] == 32
    F, _ = m.eval(x)
    k = np.arange(x.size) / x.size
    small = np.isin(np.arange(x.size), np.concatenate([np.arange(m.s_[i], m.e_[i]) for i in big])) if len(big) else \
        np.zeros(x.size, bool)
    assert np.abs(F - k)[~small].max() <= 2 * T / x.size
    assert m.depth.max() > 2  # the skew needed deeper nodes


def test_uniform_fit_tracks_empirical_cdf(orc):
    x = _sample("uniform", 100000)
    F, _ = orc.Rmi(x, T).eval(x)
    k = np.arange(x.size) / x.size
    assert np.abs(F - k).max() < 2 * T / x.size


def test_all_equal_sample_gives_constant_cdf(orc):
    S = 1000
    x = np.full(S, 12345678901234, dtype=np.uint64)
    m = orc.Rmi(x, T)
    assert len(m) == 1 and m.fanout[0] == 0
    F, _ = m.eval(np.array([0, 12345678901234, 95**9 - 1], dtype=np.uint64))
    assert np.all(F == (S - 1) / 2 / S)


def test_single_key_sample(orc):
    m = orc.Rmi(np.array([777], dtype=np.uint64), T)
    F, leaf = m.eval(np.array([0, 777, 95**9 - 1], dtype=np.uint64))
    assert np.all(F == 0) and np.all(leaf == 0)


def test_unsorted_sample_rejected(orc):
    with pytest.raises(ValueError):
        orc.Rmi(np.array([5, 3], dtype=np.uint64), T)


def _budget_sample(S=20000, frac=0.8, A=1000):
    """A block of equal keys with a geometric tail of larger keys: every level's
    linear router sends the block (and the tail's smallest keys) to one child,
    which splits again, so each level adds about S/T nodes until the node
    budget stops the tree."""
    nb = int(S * frac)
    k = np.arange(S - nb)
    off = np.floor(2.0 ** (58.0 * k / (S - nb - 1))).astype(np.uint64)
    return np.sort(np.concatenate([np.full(nb, A, dtype=np.uint64), np.uint64(A) + off]))


def _route_exact(gamma, delta, scale, fanout, base, shift, x):
    """The router clamp(floor(fma(gamma, u, delta) * scale), 0, f-1), with the
    fused multiply-add done in exact rationals and rounded once to double."""
    from fractions import Fraction

    u = (int(x) - int(base)) >> int(shift) if int(x) > int(base) else 0
    t = float(Fraction(float(gamma)) * u + Fraction(float(delta))) * float(scale)
    if not t > 0.0:
        return 0
    return fanout - 1 if t >= fanout else int(t)


def test_node_budget_caps_a_whole_level(orc):
    """The budget rule of the RMI reading (Sec. 3.1 defers the architecture to
    the RMI papers): the children of a level are created only if the tree then
    holds at most 4*ceil(S/T) + 1024 nodes; otherwise every node of that level
    becomes a leaf.  Checked on a sample that reaches the budget: every level
    that split stayed within it, the level that did not split would have gone
    past it, and that level is all leaves."""
    x = _budget_sample()
    S = x.size
    budget = 4 * (-(-S // T)) + 1024
    m = orc.Rmi(x, T)
    assert len(m) <= budget
    depth = m.depth.astype(np.int64)
    levels = int(depth.max()) + 1
    before = 0
    for d in range(levels):
        idx = np.nonzero(depth == d)[0]
        would = 0  # children this level's nodes would create under the split rule alone
        for i in idx:
            s, e = int(m.s_[i]), int(m.e_[i])
            n = e - s
            if n <= 2 * T or x[s] == x[e - 1] or d >= 32:
                continue
            f = -(-n // T)
            if _route_exact(m.gamma[i], m.delta[i], f / n, f, m.base[i], m.shift[i], x[s]) == \
                    _route_exact(m.gamma[i], m.delta[i], f / n, f, m.base[i], m.shift[i], x[e - 1]):
                continue
            would += f
        total_after_level = before + len(idx)
        if d < levels - 1:
            assert total_after_level + would <= budget
            assert int(m.fanout[idx].astype(np.int64).sum()) == would  # every node that may split did
        else:
            assert would > 0 and total_after_level + would > budget  # the cap is what stopped the tree
            assert np.all(m.fanout[idx] == 0)  # all of the level, not node by node
        before = total_after_level
    assert before == len(m)
    # the capped level's leaves still clamp to their rank ranges: F stays monotone in [0, 1]
    F, _ = m.eval(np.sort(np.concatenate([x, x + np.uint64(1)])))
    assert np.all(np.diff(F) >= 0) and F.min() >= 0 and F.max() <= 1
