"""Pins of the two oracle helpers that decide which rollouts the GPU parity
tests excuse:

* the obstacle margin |p - o|^2 - r^2 of the quadrotor's indicator cost,
  checked against signed squared distances computed by hand (inside, on and
  outside the sphere), against the indicator itself, and, along a whole
  rollout, against the margin recomputed from the oracle's own trajectory;
* the bfloat16 rounding-tie flag, checked on values built at exact bfloat16
  midpoints and just inside and outside its 2^-20 band, and against the
  property the parity tests rely on: outside the band, a float32 value a few
  ulps away from the exact one rounds to the same bfloat16 value as the
  exact value itself (exact rounding computed with rational arithmetic).
"""

import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1807_06108_gb300 import workloads as W


def _quad_state(p):
    x = np.zeros(12)
    x[:3] = p
    return x


def test_obstacle_margin_signed_squared_distance():
    prob = W.quadrotor_k4096(K=1, T=1)  # obstacle at (2, 0, 1), radius 0.5
    cases = [
        ((2.0, 0.0, 1.0), -0.25),    # centre
        ((2.25, 0.0, 1.0), -0.1875),  # inside: 0.0625 - 0.25
        ((2.5, 0.0, 1.0), 0.0),      # on the sphere
        ((2.0, -0.5, 1.0), 0.0),     # on the sphere, another axis
        ((3.0, 0.0, 1.0), 0.75),     # outside: 1 - 0.25
        ((2.0, 1.0, 2.0), 1.75),     # outside: 1 + 1 - 0.25
        ((0.0, 0.0, 1.0), 3.75),     # the start point: 4 - 0.25
    ]
    for p, want in cases:
        assert oracle.obstacle_margin(prob, _quad_state(p)) == want, p
    # another obstacle: centre (1, -2, 3), radius 2 (values exact in binary)
    prob2 = W.quadrotor_k4096(K=1, T=1, params={"obs": [1.0, -2.0, 3.0], "obs_r": 2.0})
    for p, want in [((1.0, -2.0, 3.0), -4.0), ((3.0, -2.0, 3.0), 0.0), ((1.0, 0.0, 5.0), 4.0),
                    ((2.0, -1.0, 4.0), -1.0), ((-1.0, -4.0, 1.0), 8.0)]:
        assert oracle.obstacle_margin(prob2, _quad_state(p)) == want, p
    # the cart-pole has no obstacle
    cp = W.cartpole_k1000(K=1, T=1)
    assert math.isinf(oracle.obstacle_margin(cp, np.zeros(4)))


def test_obstacle_margin_sign_agrees_with_the_indicator():
    prob = W.quadrotor_k4096(K=1, T=1)
    rng = np.random.default_rng(11)
    cost = prob["params"]["obs_cost"]
    for _ in range(400):
        x = _quad_state([2.0, 0.0, 1.0] + rng.uniform(-0.8, 0.8, 3))
        x[3:] = rng.normal(0, 0.3, 9)
        mg = oracle.obstacle_margin(prob, x)
        if mg == 0.0:
            continue
        without = oracle.terminal_cost(prob, x)  # the same quadratic, no indicator
        with_ind = oracle.state_cost(prob, x)
        has = abs((with_ind - without) - cost) <= 1e-9 * cost
        assert has or abs(with_ind - without) <= 1e-9, (x[:3], mg)
        assert has == (mg < 0.0), (x[:3], mg)


def test_rollout_margin_is_smallest_distance_along_the_costed_states():
    """The per-rollout margin the oracle reports is min_j | |p_j - o|^2 - r^2 |
    over the costed states j = 0 .. T-1, recomputed here from the oracle's
    trajectory output with the hand formula."""
    prob = W.quadrotor_k4096(K=24, T=30, lam=20.0)
    x0 = W.initial_state(prob).astype(np.float64)
    x0[:3] = [1.3, 0.1, 1.0]
    x0[3] = 2.0
    U = W.initial_controls(prob)
    r = oracle.rollouts(prob, x0, U, 0, 0, 24, traj=True, margin=True)
    o = np.asarray(prob["params"]["obs"])
    r2 = prob["params"]["obs_r"] ** 2
    d = np.sum((r["traj"][:, :prob["T"], :3] - o) ** 2, axis=2) - r2
    want = np.min(np.abs(d), axis=1)
    np.testing.assert_allclose(r["margin"], want, rtol=1e-12, atol=1e-15)
    assert np.any(want < 0.05)  # some rollouts do pass close to the boundary


def _bf16(bits):
    return float(np.array([bits << 16], dtype=np.uint32).view(np.float32)[0])


def _mid(lo_bits):
    return 0.5 * (_bf16(lo_bits) + _bf16(lo_bits + 1))


@pytest.mark.parametrize("lo_bits", [0x3F80, 0x3F81, 0x3FFF, 0x4049, 0x3A12, 0x7F00, 0x0080,
                                     0xBF80, 0xC0A3])
def test_bf16_ambiguity_band_around_exact_midpoints(lo_bits):
    """Midpoints between bfloat16 neighbours lo and lo + 1 ulp (including one
    whose upper neighbour crosses into the next binade, 0x3FFF -> 2.0, and
    negative values, where the upper bit pattern is the larger magnitude)."""
    mid = _mid(lo_bits)
    assert oracle.bf16_ambiguous(mid)
    for f in (0.25, 0.5, 0.9):
        eps = f * 2.0 ** -20 * abs(mid)
        assert oracle.bf16_ambiguous(mid + eps), f
        assert oracle.bf16_ambiguous(mid - eps), f
    for f in (1.5, 4.0, 64.0):
        eps = f * 2.0 ** -20 * abs(mid)
        assert not oracle.bf16_ambiguous(mid + eps), f
        assert not oracle.bf16_ambiguous(mid - eps), f


def test_bf16_ambiguity_off_midpoints_and_special_values():
    for bits in (0x3F80, 0x4049, 0xBF80, 0x0080):
        v = _bf16(bits)  # exactly representable: never ambiguous
        assert not oracle.bf16_ambiguous(v)
        assert not oracle.bf16_ambiguous(np.nextafter(v, 0.0))
        assert not oracle.bf16_ambiguous(np.nextafter(v, np.inf))
    for v in (0.0, -0.0, math.inf, -math.inf, math.nan):
        assert not oracle.bf16_ambiguous(v)


def _exact_bf16_bits(x):
    """bfloat16 bits of the exact (rational) value x, round to nearest even."""
    q = Fraction(x)
    sign = 0x8000 if q < 0 else 0
    q = abs(q)
    e = math.floor(math.log2(q))
    while Fraction(2) ** e > q:
        e -= 1
    while Fraction(2) ** (e + 1) <= q:
        e += 1
    ulp = Fraction(2) ** (e - 7)
    n = q / ulp
    fl = math.floor(n)
    rem = n - fl
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and fl % 2 == 1):
        fl += 1
    val = fl * ulp
    return sign | int(np.array([np.float32(val)]).view(np.uint32)[0] >> 16)


def test_outside_the_band_float32_errors_do_not_change_the_bf16_value():
    """The property the parity tests depend on: for a float64 value d that is
    not flagged, a float32 approximation of d with a relative error of up to
    2^-21 rounds to the bfloat16 value of d itself."""
    rng = np.random.default_rng(5)
    checked = 0
    for _ in range(3000):
        lo = int(rng.integers(0x3000, 0x4400))
        mid = _mid(lo)
        d = mid * (1.0 + rng.uniform(-2.0 ** -17, 2.0 ** -17))
        if oracle.bf16_ambiguous(d):
            continue
        want = _exact_bf16_bits(d)
        for rel in (-2.0 ** -21, 2.0 ** -21, 0.0):
            f = np.float32(d * (1.0 + rel))
            got = int(np.array([f]).view(np.uint32)[0])
            got = ((got + 0x7FFF + ((got >> 16) & 1)) >> 16) & 0xFFFF
            assert got == want, (d, rel)
        assert int(np.array([oracle.bf16_round(d)], dtype=np.float32).view(np.uint32)[0] >> 16) == want
        checked += 1
    assert checked > 1500
