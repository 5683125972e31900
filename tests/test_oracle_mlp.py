"""Pins for the oracle's monotone MLP CDF model (the learned model the GPU trains).

The network is not in the paper (whose Sec. 3.1 model is an RMI), so these pins
come from mathematics: closed forms of hand-set networks, the chain rule
checked against central finite differences, FP32 vs FP64 agreement,
monotonicity, and a trained network beating a single least-squares line.
"""
import numpy as np
import pytest

NP = 1517  # W1[32][12], b1[32], W2[32][32], b2[32], w3[32], b3, v[12]


def _w(rng, scale=1.0):
    w = rng.random(NP) * scale
    w[384:416] = rng.normal(0, 1, 32)  # b1
    w[1440:1472] = rng.normal(0, 1, 32)  # b2
    w[1472:1504] *= 2.0 / 32  # w3
    w[1504] = 0.0
    w[0:384] *= 2.0 / 12
    w[416:1440] *= 2.0 / 32
    w[1505:1517] *= 0.5 / 12  # v
    return w


def test_layout(orc):
    assert orc.MLP_PARAMS == NP == orc.lib().eo_mlp_params()
    assert sum(b - a for a, b in orc.MLP_SLICES.values()) == NP


def test_closed_form_forward(orc):
    w = np.zeros(NP)
    w[1472:1504] = 0.02
    w[1504] = 0.3
    phi = np.random.default_rng(0).random((5, 12))
    # every hidden unit sees 0 -> sigma(0) = 1/2; z = b3 + 32 * 0.02 * 1/2
    assert np.allclose(orc.mlp_forward64(w, phi), 0.3 + 0.32)
    assert np.allclose(orc.mlp_forward32(w.astype(np.float32), phi.astype(np.float32)), 0.62, atol=1e-7)
    # sigma(1) = 3/4 for one path: W1[0,0] = 1, phi_0 = 1 -> h1_0 = 3/4; W2[0,0] = 4 -> p2_0 = 3 -> h2_0 = 7/8
    w = np.zeros(NP)
    w[0] = 1.0
    w[416] = 4.0
    w[1472] = 1.0
    phi = np.zeros((1, 12))
    phi[0, 0] = 1.0
    assert orc.mlp_forward64(w, phi)[0] == pytest.approx(7 / 8)
    # output clamps to [0, 1]
    w[1504] = 5.0
    assert orc.mlp_forward64(w, phi)[0] == 1.0
    w[1504] = -5.0
    assert orc.mlp_forward64(w, phi)[0] == 0.0
    # the linear skip alone: F = sum_m v_m phi_m
    w = np.zeros(NP)
    w[1505:1517] = np.arange(1, 13) / 78.0  # sums to 1
    phi = np.random.default_rng(6).random((7, 12))
    assert np.allclose(orc.mlp_forward64(w, phi), phi @ (np.arange(1, 13) / 78.0), rtol=1e-14)


def test_start_is_the_knot_interpolation(orc):
    """The starting network is F = sum(phi) / 12: at the knots T_m it is m / 12
    (up to FP32 rounding), linear in between."""
    x = np.sort(np.random.default_rng(9).integers(0, 95**9, 20001, dtype=np.uint64))
    T = orc.mlp_knots(x)
    w = orc.mlp_init()
    F = orc.mlp_forward32(w, orc.mlp_features(T, T))
    assert np.allclose(F, np.arange(13) / 12, atol=2e-7)
    mid = T[:12] + (T[1:] - T[:12]) // np.uint64(2)
    Fm = orc.mlp_forward32(w, orc.mlp_features(T, mid))
    assert np.allclose(Fm, (np.arange(12) + 0.5) / 12, atol=1e-6)


def test_features_are_ramps_between_knots(orc):
    x = np.sort(np.random.default_rng(1).integers(0, 95**9, 100001, dtype=np.uint64))
    T = orc.mlp_knots(x)
    assert T[0] == x[0] and T[12] == x[-1] and np.all(np.diff(T.astype(np.float64)) >= 0)
    phi = orc.mlp_features(T, T)
    for m in range(12):
        assert phi[m, m] == 0.0 and phi[m + 1, m] == 1.0  # 0 at its knot, 1 at the next
        assert np.all(phi[: m + 1, m] == 0.0) and np.all(phi[m + 1:, m] == 1.0)
    mid = T[:12] + (T[1:] - T[:12]) // np.uint64(2)
    pm = orc.mlp_features(T, mid)
    assert np.allclose(np.diag(pm), 0.5, atol=1e-6)
    # monotone in the key
    f = orc.mlp_features(T, x)
    assert np.all(np.diff(f, axis=0) >= 0)


def test_backward_matches_central_differences(orc):
    rng = np.random.default_rng(2)
    w = _w(rng)
    phi = rng.random((64, 12))
    y = rng.random(64)
    F = orc.mlp_forward64(w, phi)
    assert np.all((F > 0) & (F < 1))  # away from the clamp's kinks
    g = orc.mlp_grad64(w, phi, y)
    idx = np.concatenate([rng.choice(NP, 60, replace=False), [0, 383, 384, 416, 1439, 1440, 1472, 1504, 1505, 1516]])

    def loss(v):
        return np.mean((orc.mlp_forward64(v, phi) - y) ** 2)

    for i in idx:
        h = 1e-6 * max(1.0, abs(w[i]))
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (loss(wp) - loss(wm)) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-10), i


def test_fp32_forward_within_1e5_of_fp64(orc):
    rng = np.random.default_rng(3)
    for _ in range(5):
        w = _w(rng)
        phi = rng.random((2000, 12)).astype(np.float32)
        f32 = orc.mlp_forward32(w.astype(np.float32), phi)
        f64 = orc.mlp_forward64(w.astype(np.float32).astype(np.float64), phi.astype(np.float64))
        assert np.abs(f32 - f64).max() < 1e-5


def test_nonnegative_weights_make_it_monotone(orc):
    rng = np.random.default_rng(4)
    x = np.sort(rng.integers(0, 95**9, 20001, dtype=np.uint64))
    T = orc.mlp_knots(x)
    probe = np.sort(rng.integers(0, 95**9, 50000, dtype=np.uint64))
    phi = orc.mlp_features(T, probe).astype(np.float64)
    for _ in range(3):
        F = orc.mlp_forward64(_w(rng), phi)
        assert np.all(np.diff(F) >= -1e-12)


def test_training_beats_its_start_and_a_least_squares_line(orc, gen):
    n = 200_000
    recs = gen.generate_cpu(n, gen.KeySpec("zipf", s=1.3, dup=0.1, seed=5))
    x = np.sort(orc.sample(recs, 20000, 1))
    y = np.arange(x.size) / x.size
    T = orc.mlp_knots(x)
    phi = orc.mlp_features(T, x).astype(np.float64)
    w0 = orc.mlp_init().astype(np.float64)
    init_mse = np.mean((orc.mlp_forward64(w0, phi) - y) ** 2)
    w, loss = orc.mlp_train64(w0, phi, y, batch=4096, steps=150, lr=1e-3, lr_min=1e-5)
    assert loss < init_mse
    slope, icpt = np.polyfit(x.astype(np.float64), y, 1)
    line_mse = np.mean((np.clip(slope * x.astype(np.float64) + icpt, 0, 1) - y) ** 2)
    assert loss < line_mse / 10
    # projection keeps every weight >= 0
    for k in orc.MLP_WEIGHTS:
        a, b = orc.MLP_SLICES[k]
        assert np.all(w[a:b] >= 0)


def test_learning_rate_schedule_closed_form(orc):
    """Half-cosine decay: lr at the first step, lr_min at the last, their mean
    half way, and the cosine's value in between."""
    assert orc.mlp_lr_at(1, 101, 1e-3, 1e-5) == pytest.approx(1e-3, rel=1e-15)
    assert orc.mlp_lr_at(101, 101, 1e-3, 1e-5) == pytest.approx(1e-5, rel=1e-12)
    assert orc.mlp_lr_at(51, 101, 1e-3, 1e-5) == pytest.approx((1e-3 + 1e-5) / 2, rel=1e-12)
    # a quarter of the way: cos(pi/4) = sqrt(2)/2
    assert orc.mlp_lr_at(26, 101, 1e-3, 1e-5) == pytest.approx(1e-5 + 0.99e-3 * (1 + 2**-0.5) / 2, rel=1e-12)


def test_splitters_reproduce_the_fp32_bins(orc):
    rng = np.random.default_rng(5)
    x = np.sort(rng.integers(0, 95**9, 20001, dtype=np.uint64))
    T = orc.mlp_knots(x)
    w = _w(rng).astype(np.float32)
    log2B = 8
    t = orc.mlp_splitters(w, T, log2B)
    assert t[0] == 0 and np.all(np.diff(t.astype(np.float64)) >= 0)
    probe = np.sort(rng.integers(0, 95**9, 30000, dtype=np.uint64))
    q = orc.bins_by_splitters(t, log2B, probe)
    direct = np.minimum(255, np.floor(orc.mlp_forward32(w, orc.mlp_features(T, probe)) * 256)).astype(np.uint32)
    assert np.mean(q == direct) > 0.999
    assert np.all(np.diff(q.astype(np.int64)) >= 0)


# ---------------------------------------------------------------- Adam (Kingma & Ba 2015, Algorithm 1)
W_SLICES = ("W1", "W2", "w3", "v")
B_SLICES = ("b1", "b2", "b3")
LR = 1e-3


def _mask(orc, names):
    m = np.zeros(NP, bool)
    for k in names:
        a, b = orc.MLP_SLICES[k]
        m[a:b] = True
    return m


def test_adam_first_step_moves_each_parameter_by_lr(orc):
    """From a zero moment state the bias corrections make mhat = g and
    vhat = g^2 exactly, so step 1 moves every parameter by lr * |g| / (|g| + eps)
    against its gradient -- whatever the sign or size of g."""
    rng = np.random.default_rng(10)
    w0 = rng.random(NP) + 1.0  # far from the projection
    g = rng.normal(0, 1, NP) * 10.0 ** rng.integers(-4, 3, NP)
    w, m, v = orc.mlp_adam64(w0, g, np.zeros(NP), np.zeros(NP), 1, LR)
    assert np.allclose(w - w0, -LR * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
    assert np.allclose(m, 0.1 * g, rtol=1e-15) and np.allclose(v, 0.001 * g * g, rtol=1e-15)


def test_adam_constant_gradient_keeps_step_lr(orc):
    """With the same gradient every step, mhat = g and vhat = g^2 at every t
    (the corrections 1 - beta^t undo the zero start exactly), so every step is
    lr * g / (|g| + eps): a correction taken at the wrong t changes the step."""
    rng = np.random.default_rng(11)
    g = rng.normal(0, 1, NP)
    w = rng.random(NP) + 1.0
    m = np.zeros(NP)
    v = np.zeros(NP)
    for t in range(1, 6):
        w_prev = w
        w, m, v = orc.mlp_adam64(w, g, m, v, t, LR)
        assert np.allclose(w - w_prev, -LR * g / (np.abs(g) + 1e-8), rtol=1e-10, atol=0), t


def test_adam_alternating_gradient_second_step(orc):
    """Gradient +1 then -1: m_2 = 0.9 * 0.1 - 0.1 = -0.01 and 1 - 0.9^2 = 0.19,
    so mhat_2 = -1/19; v_2 = 0.999 * 0.001 + 0.001 = 0.001999 = 1 - 0.999^2, so
    vhat_2 = 1.  The second step is therefore +lr / 19 / (1 + eps).  (With the
    two decay rates swapped it would be about +lr / 2000.)"""
    w0 = np.full(NP, 1.0)
    w1, m, v = orc.mlp_adam64(w0, np.ones(NP), np.zeros(NP), np.zeros(NP), 1, LR)
    w2, m, v = orc.mlp_adam64(w1, -np.ones(NP), m, v, 2, LR)
    assert np.allclose(m, -0.01, rtol=1e-12) and np.allclose(v, 0.001999, rtol=1e-12)
    assert np.allclose(w2 - w1, LR / 19 / (1 + 1e-8), rtol=1e-10)


def test_adam_projects_weights_not_biases(orc):
    """After the step the weights (W1, W2, w3) are projected onto >= 0, which
    keeps the network monotone; the biases are free to go negative."""
    g = np.ones(NP)  # every parameter steps down by lr
    w, _, _ = orc.mlp_adam64(np.zeros(NP), g, np.zeros(NP), np.zeros(NP), 1, LR)
    wm, bm = _mask(orc, W_SLICES), _mask(orc, B_SLICES)
    assert np.all(w[wm] == 0.0)
    assert np.allclose(w[bm], -LR / (1 + 1e-8), rtol=1e-12)
    assert wm.sum() + bm.sum() == NP


def test_training_one_full_batch_is_gradient_then_adam(orc):
    """eo_mlp_train64 with one minibatch of all samples and one epoch is one
    Adam step on the mean-squared-error gradient (whose chain rule is pinned by
    finite differences above)."""
    rng = np.random.default_rng(12)
    w0 = _w(rng)
    phi = rng.random((300, 12))
    y = rng.random(300)
    w, _ = orc.mlp_train64(w0, phi, y, batch=300, steps=1, lr=LR, lr_min=LR)
    g = orc.mlp_grad64(w0, phi, y)
    want, _, _ = orc.mlp_adam64(w0, g, np.zeros(NP), np.zeros(NP), 1, LR)
    assert np.array_equal(w, want)


def test_splitters_bracket_the_bins_exactly(orc):
    """t_q is the smallest key encoding whose FP32 fine bin is >= q: bin(t_q) >= q
    and bin(t_q - 1) < q for every q whose splitter was not raised to its
    predecessor by the running maximum; t_q = 95^9 only when no encoding
    reaches bin q."""
    rng = np.random.default_rng(13)
    x = np.sort(rng.integers(0, 95**9, 20001, dtype=np.uint64))
    T = orc.mlp_knots(x)
    log2B = 9
    B = 1 << log2B
    top = np.uint64(95**9)
    for seed in range(3):
        r = np.random.default_rng(100 + seed)
        w = orc.mlp_init().astype(np.float64)
        w += np.abs(r.normal(0, 0.05, w.size)) * (np.abs(w) + 0.05)  # non-negative perturbation keeps it monotone
        w = w.astype(np.float32)
        t = orc.mlp_splitters(w, T, log2B)
        assert t[0] == 0 and np.all(np.diff(t.astype(np.float64)) >= 0)

        def fbin(v):
            F = orc.mlp_forward32(w, orc.mlp_features(T, np.ascontiguousarray(v, dtype=np.uint64)))
            return np.minimum(B - 1, np.floor(F.astype(np.float64) * B)).astype(np.int64)

        q = np.arange(1, B)
        tq = t[1:]
        raised = np.concatenate([[False], tq[1:] == tq[:-1]])
        inside = (tq < top) & ~raised
        assert inside.sum() > B // 2
        assert np.all(fbin(tq[inside]) >= q[inside])
        pos = inside & (tq > 0)
        assert np.all(fbin(tq[pos] - np.uint64(1)) < q[pos])
        # splitters left at 95^9: even the largest encoding stays below bin q
        assert np.all(fbin(np.array([95**9 - 1], dtype=np.uint64))[0] < q[tq == top])
