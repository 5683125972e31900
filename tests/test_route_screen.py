"""The RMI routers' FP32 screen, restated on the CPU with exact rationals:
wherever the screen answers, its child equals the FP64 router's.

The FP64 router of an internal node takes t = rn(rn(fma(a, u, b)) * c) and
returns 0 if t <= 0, fanout - 1 if t >= fanout, else floor(t).  The screen
evaluates t32 = rn32(fma(A, u32, B)) with A = rn32(rn(a c)), B = rn32(rn(b c)),
u32 = rn32(u), and answers only when [t32 - err, t32 + err], err =
(|A u32| + |B|) 2^-20 + 2^-30, lies on one side of every branch.  These cases
pin that bound, including cancellation (b close to -a u), coordinates up to
2^60 and values next to a child boundary."""
from fractions import Fraction

import numpy as np


def rn64(x: Fraction) -> float:
    try:
        return float(x)  # Fraction -> float rounds to nearest, ties to even
    except OverflowError:  # beyond the double range: infinity, as the hardware rounds
        return float("inf") if x > 0 else float("-inf")


def rn32(x: float) -> np.float32:
    return np.float32(x)


def fma32(a: np.float32, b: np.float32, c: np.float32) -> np.float32:
    exact = Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c))
    with np.errstate(over="ignore"):
        return np.float32(rn64(exact))  # double rounding stays far inside the margin


def route64(a, b, c, u, fanout):
    t1 = rn64(Fraction(a) * Fraction(rn64(Fraction(u))) + Fraction(b))
    t = rn64(Fraction(t1) * Fraction(c))
    if not t > 0.0:
        return 0
    if t >= fanout:
        return fanout - 1
    return int(np.floor(t))


def screen(a, b, c, u, fanout):
    with np.errstate(over="ignore"):
        A = rn32(rn64(Fraction(a) * Fraction(c)))
        B = rn32(rn64(Fraction(b) * Fraction(c)))
    uf = np.float32(rn64(Fraction(u)))
    with np.errstate(over="ignore", invalid="ignore"):
        t = fma32(A, uf, B) if np.isfinite(A) and np.isfinite(B) else np.float32(np.nan)
        err = np.float32(np.float32(abs(np.float32(A * uf)) + abs(B)) * np.float32(2.0 ** -20) + np.float32(2.0 ** -30))
        lo, hi = np.float32(t - err), np.float32(t + err)
    F = np.float32(fanout)
    if hi <= 0.0:
        return 0
    if lo >= F:
        return fanout - 1
    if lo > 0.0 and hi < F and np.floor(lo) == np.floor(hi):
        return int(np.floor(lo))
    return None  # the FP64 router decides


def _check(a, b, c, u, fanout):
    s = screen(a, b, c, u, fanout)
    if s is not None:
        assert s == route64(a, b, c, u, fanout), (a, b, c, u, fanout)
    return s is not None


def test_screen_agrees_with_fp64_router_on_random_nodes():
    rng = np.random.default_rng(5)
    answered = 0
    for _ in range(4000):
        fanout = int(rng.integers(2, 1 << 14))
        span = int(rng.integers(1, 1 << int(rng.integers(1, 61))))
        a = float(rng.uniform(0.5, 2.0)) / span  # positions per unit of u, about one over the node's span
        b = float(rng.uniform(-0.1, 0.1))
        c = float(fanout) * float(rng.uniform(0.5, 2.0))
        u = int(rng.integers(0, span))
        answered += _check(a, b, c, u, fanout)
    assert answered > 3000  # the screen settles most points


def test_screen_hands_near_boundaries_to_fp64():
    rng = np.random.default_rng(6)
    for _ in range(3000):
        fanout = int(rng.integers(2, 4096))
        span = int(rng.integers(1 << 20, 1 << 60))
        a = 1.0 / span
        c = float(fanout)
        k = int(rng.integers(0, fanout + 1))
        # u whose exact t lies within a few ulps of the boundary k (or of 0 / fanout)
        u0 = int(Fraction(k, fanout) * span)
        for du in (-2, -1, 0, 1, 2):
            u = min(max(u0 + du, 0), span)
            _check(a, 0.0, c, u, fanout)
            _check(a, float(rng.uniform(-1e-9, 1e-9)), c, u, fanout)


def test_screen_under_cancellation_and_extremes():
    rng = np.random.default_rng(7)
    for _ in range(3000):
        fanout = int(rng.integers(2, 1 << 12))
        u = int(rng.integers(1, 1 << 60))
        a = float(rng.uniform(1e-3, 1e3))
        # b cancels most of a*u, so t is small against the terms that make it
        b = -a * u + float(rng.uniform(-5.0, fanout + 5.0))
        c = float(rng.uniform(0.25, 4.0))
        _check(a, b, c, u, fanout)
    # constants beyond the FP32 range leave the decision to FP64
    assert screen(1e300, 0.0, 1e10, 5, 100) is None
    assert screen(1e-3, 0.0, 1e42, 5, 100) is None
    assert _check(1e-3, 0.0, 1e40, 5, 100)  # 1e37 still fits: answered, and equal to FP64
    # a constant router (a = 0) away from a boundary is settled by the screen;
    # t exactly 0 lies within the margin of the first boundary and goes to FP64
    assert _check(0.0, 3.5, 1.0, 7, 10) and screen(0.0, 3.5, 1.0, 7, 10) == 3
    assert screen(0.0, 0.0, 1.0, 7, 10) is None and route64(0.0, 0.0, 1.0, 7, 10) == 0
