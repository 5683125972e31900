"""Pins for the oracle's model choice (the network or the RMI) and for the
method with a given classifier.

The network is this project's addition; the paper's model (Sec. 3.1) is the
RMI, which stays the network's fallback and judges it.  The three checks of
the choice are pinned with hand-set networks whose outputs have closed forms:
a constant network, and a one-path network whose values at the first and last
knot are computed by hand from sigma(z) = 1/2 + z / (2 (1 + |z|)).
"""
import numpy as np
import pytest

P, S, SEED = 64, 10_000, 5


@pytest.fixture(scope="module")
def recs(gen):
    return gen.generate_cpu(200_000, gen.KeySpec("uniform", seed=8))


def _log2B(orc, n):
    return orc.default_fine_log2(n, P)


def _const_net(c):
    w = np.zeros(1517, dtype=np.float32)
    w[1504] = c  # b3: with w3 = 0 the network outputs c everywhere
    return w


def _one_path(b3):
    """h1_0 = sigma(-6 + sum(phi)), h2_0 = sigma(h1_0), F = b3 + w3 * h2_0.
    At the first knot every ramp is 0: h1 = sigma(-6) = 1/14, h2 = sigma(1/14) = 8/15.
    At the last knot every ramp is 1: h1 = sigma(6) = 13/14, h2 = sigma(13/14) = 20/27."""
    w = np.zeros(1517, dtype=np.float32)
    w[0:12] = 1.0  # W1[0][m]
    w[384] = -6.0  # b1[0]
    w[416] = 1.0  # W2[0][0]
    w3 = 0.9 / (20 / 27 - 8 / 15)
    w[1472] = w3
    w[1504] = b3
    return w, w3


def test_judge_bucket_count_closed_form(orc, recs):
    # the largest J <= B with 64 J <= S: 64 * 128 = 8192 <= 10,000 < 16,384
    _, d = orc.model_choice(recs, P, _log2B(orc, 200_000), S, SEED, 1, _const_net(0.5), skip=7)
    assert d["J"] == 128


def test_constant_network_fails_the_boundary_check(orc, recs):
    r, d = orc.model_choice(recs, P, _log2B(orc, 200_000), S, SEED, 1, _const_net(0.5))
    assert r == 1 and d["F_first_knot"] == 0.5 and d["F_last_knot"] == 0.5


def test_boundary_thresholds(orc, recs):
    log2B = _log2B(orc, 200_000)
    # F(T_0) = b3 + w3 * 8/15, F(T_12) = b3 + w3 * 20/27 = F(T_0) + 0.9
    for F0, want in ((0.05, 0), (0.07, 1), (0.03, 1)):  # 0.03 + 0.9 = 0.93 < 15/16
        w, w3 = _one_path(F0 - (0.9 / (20 / 27 - 8 / 15)) * 8 / 15)
        r, d = orc.model_choice(recs, P, log2B, S, SEED, 1, w, skip=2 | 4)
        assert d["F_first_knot"] == pytest.approx(F0, abs=1e-5)
        assert d["F_last_knot"] == pytest.approx(F0 + 0.9, abs=1e-5)
        assert r == want, F0


def test_constant_network_loses_the_judge(orc, recs):
    # every held-out key lands in fine bin B/2: one judge bucket holds all S keys
    r, d = orc.model_choice(recs, P, _log2B(orc, 200_000), S, SEED, 1, _const_net(0.5), skip=1)
    assert r == 2 and d["mlp_max_bucket"] == S and d["rmi_max_bucket"] < S / 10


@pytest.mark.parametrize("balance", [0, 1])
def test_constant_network_fails_the_full_data_check(orc, recs, balance):
    # all n records in one fine bin, hence in one partition under either cut rule
    n = recs.size // 100
    r, d = orc.model_choice(recs, P, _log2B(orc, n), S, SEED, balance, _const_net(0.5), skip=1 | 2)
    assert r == 3 and d["mlp_max_partition"] == n


def test_all_checks_skipped_keeps_the_network(orc, recs):
    r, d = orc.model_choice(recs, P, _log2B(orc, 200_000), S, SEED, 1, _const_net(0.5), skip=7)
    assert r == 0 and d["mlp_max_partition"] == 0


def test_rmi_judge_bucket_is_the_held_out_histogram_maximum(orc, recs):
    """The RMI side of the judge is the held-out sample (seed + 1) binned by the
    RMI fitted on the sample (seed), grouped into J buckets."""
    n = recs.size // 100
    log2B = _log2B(orc, n)
    _, d = orc.model_choice(recs, P, log2B, S, SEED, 1, _const_net(0.5), skip=1)
    m = orc.Rmi(np.sort(orc.sample(recs, S, SEED)))
    F, _ = m.eval(orc.sample(recs, S, SEED + 1))
    B = 1 << log2B
    q = np.minimum(B - 1, np.floor(F * B)).astype(np.int64)
    J = int(d["J"])
    assert d["rmi_max_bucket"] == np.bincount(q >> (log2B - J.bit_length() + 1), minlength=J).max()


# ---------------------------------------------------------------- the method with a given classifier
def test_sort_by_splitters_is_the_stable_sort(orc, gen):
    n = 30_000
    recs = gen.generate_cpu(n, gen.KeySpec("zipf", s=1.2, dup=0.05, seed=4))
    log2B = 8
    t = np.sort(orc.sample(recs, 255, 3))
    t = np.concatenate([[0], t]).astype(np.uint64)  # any non-decreasing splitters give a valid classifier
    for balance in (0, 1):
        out, det = orc.sort_by_splitters(recs, t, log2B, 16, balance)
        assert np.array_equal(out, orc.stable_sort(recs))
        x = orc.encode9_records(recs)
        # bin = number of splitters t[1..B) at or below the key encoding (brute force)
        want = (t[1:][None, :] <= x[:, None]).sum(axis=1)
        assert np.array_equal(det["q"].astype(np.int64), want)
        assert det["part_off"][-1] == n


def test_sort_by_splitters_rejects_decreasing_splitters(orc, gen):
    recs = gen.generate_cpu(100, gen.KeySpec("uniform", seed=1))
    t = np.array([0, 5, 3, 9], dtype=np.uint64)
    with pytest.raises(ValueError):
        orc.sort_by_splitters(recs, t, 2, 2)


@pytest.mark.parametrize("threads", [1, 2, 5])
@pytest.mark.parametrize("kind", ["uniform", "zipf"])
def test_threaded_oracle_equals_single_threaded(orc, gen, threads, kind):
    n = 120_000
    spec = gen.KeySpec(kind, s=1.1, dup=0.05, seed=6)
    recs = gen.generate_cpu(n, spec)
    log2B = orc.default_fine_log2(n, 64)
    want = orc.sort(recs, 64, log2B, S=1200, seed=9)
    assert np.array_equal(orc.sort_threads(recs, 64, log2B, S=1200, seed=9, threads=threads), want)
