"""Pins for the oracle's estimator: the free-energy weights (Eq. 36-37), the
control update (Eq. 37, 49), the augmented cost (Eq. 34-35) and the MPC
shift (Algorithm 1).  The strongest pins are closed forms: for a one-step
horizon the cost is quadratic in the perturbation, so the exponentially
tilted mean that the update estimates is a Gaussian integral; the Monte
Carlo update must match it within its standard error, for several
exploration scales c, nominal controls u and with control-channel jumps."""

import numpy as np
import pytest
from scipy.special import logsumexp

import oracle
from paper_1807_06108_gb300 import workloads as W


# ------------------------------------------------------------------ weights

def test_softmin_normalised_shift_invariant_and_free_energy():
    rng = np.random.default_rng(0)
    S = rng.standard_normal(500) * 30 + 200
    for lam in (0.5, 1.0, 20.0):
        w, d = oracle.softmin(S, lam)
        assert w.sum() == pytest.approx(1.0, abs=1e-14)
        assert np.all(w >= 0)
        w2, d2 = oracle.softmin(S + 1234.5, lam)
        np.testing.assert_allclose(w2, w, rtol=1e-9, atol=1e-300)
        assert d2[0] == pytest.approx(d[0] + 1234.5)
        # Monte Carlo free energy of Eq. 5: -ln mean exp(-S/lambda)
        F = -(logsumexp(-S / lam) - np.log(S.size))
        assert d[2] == pytest.approx(F, rel=1e-12)
        assert d[0] == S.min()


def test_softmin_temperature_limits():
    rng = np.random.default_rng(1)
    S = rng.standard_normal(64)
    w, _ = oracle.softmin(S, 1e12)
    np.testing.assert_allclose(w, 1.0 / 64, rtol=1e-9)
    w, _ = oracle.softmin(S, 1e-9)
    assert w[np.argmin(S)] == 1.0 and np.sum(w) == 1.0


def test_softmin_non_finite_costs():
    S = np.array([np.inf, 3.0, np.nan, 1.0])
    w, d = oracle.softmin(S, 1.0)
    assert w[0] == 0.0 and w[2] == 0.0
    assert w[1] + w[3] == pytest.approx(1.0)
    with pytest.raises(oracle.OracleError):
        oracle.softmin(np.array([np.inf, np.nan]), 1.0)


# ------------------------------------------------------------------ update

def test_update_is_weighted_sum_of_perturbations():
    rng = np.random.default_rng(2)
    T, K, m = 7, 33, 4
    delta = rng.standard_normal((T, K, m))
    w = rng.random(K)
    w /= w.sum()
    U = rng.standard_normal((T, m))
    for alpha in (1.0, 0.3):
        got = oracle.update(w, delta, U, alpha)
        ref = U + alpha * np.einsum("k,tkm->tm", w, delta)
        np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("channel", ["state", "control"])
def test_single_rollout_returns_its_perturbation(channel):
    prob = W.quadrotor_k4096(K=1, T=9, nu=40.0, jump_channel=channel)
    rng = np.random.default_rng(3)
    x0, U = W.random_state(prob, rng), W.random_controls(prob, rng)
    r = oracle.iteration(prob, x0, U, 5, want_delta=True, want_counts=True)
    assert r["counts"].sum() > 0
    assert r["w"][0] == 1.0
    np.testing.assert_array_equal(r["U"], U.astype(np.float64) + r["delta"][:, 0, :])


def test_vanishing_gaussian_noise_leaves_controls_unchanged():
    """Zero-noise limit: sigma -> 0 bounds the update by max|z| sigma; state
    jumps never enter the update (Eq. 36 carries only the Gaussian term)."""
    for channel, nu in (("state", 30.0), ("control", 0.0)):
        prob = W.quadrotor_k4096(K=256, T=10, nu=nu, sigma=1e-7, jump_channel=channel)
        rng = np.random.default_rng(4)
        x0, U = W.random_state(prob, rng), W.initial_controls(prob)
        r = oracle.iteration(prob, x0, U, 0)
        assert np.max(np.abs(r["U"] - U)) < 6.0 * 1e-7


@pytest.mark.parametrize("channel", ["state", "control"])
def test_zero_rate_equals_zero_marks(channel):
    """nu = 0 (no jumps) and nu > 0 with zero-size marks give bit-identical
    costs and updates: the jump machinery adds exactly nothing."""
    base = dict(K=300, T=11, jump_channel=channel)
    p0 = W.cartpole_k1000(nu=0.0, **base)
    p1 = W.cartpole_k1000(nu=25.0, mark_scale=0.0, **base)
    rng = np.random.default_rng(5)
    x0, U = W.random_state(p0, rng), W.random_controls(p0, rng)
    r0 = oracle.iteration(p0, x0, U, 2, want_counts=True)
    r1 = oracle.iteration(p1, x0, U, 2, want_counts=True)
    assert r0["counts"].max() == 0 and r1["counts"].sum() > 0
    np.testing.assert_array_equal(r0["S"], r1["S"])
    np.testing.assert_array_equal(r0["U"], r1["U"])


# --------------------------------------------------- augmented cost structure

def test_augmented_cost_terms():
    """S~ = sum_j q(x_j) dt + phi(x_T) + lambda sum_j [1/2 u^T S^-1 u +
    u^T S^-1 d + 1/2 (1 - 1/c) d^T S^-1 d]; with u = 0 and c = 1 the
    importance-sampling terms vanish and S~ is the plain path cost S, the
    case in which the information-theoretic and stochastic-optimisation
    updates coincide (Sec. IV)."""
    for c, zero_u in ((1.0, True), (2.5, False), (0.6, False)):
        prob = W.quadrotor_k4096(K=8, T=6, c=c, lam=3.0, sigma=[0.2, 0.3, 0.25, 0.4])
        rng = np.random.default_rng(6)
        x0 = W.random_state(prob, rng)
        U = np.zeros((6, 4)) if zero_u else W.random_controls(prob, rng)
        r = oracle.rollouts(prob, x0, U, 1, 0, 8, delta=True, traj=True)
        inv = 1.0 / np.array(prob["sigma"]) ** 2
        for k in range(8):
            tr = r["traj"][k]
            plain = sum(oracle.state_cost(prob, tr[j]) for j in range(6)) * prob["dt"]
            plain += oracle.terminal_cost(prob, tr[6])
            d = r["delta"][:, k, :]
            Ud = np.asarray(U, dtype=np.float64)
            is_terms = prob["lam"] * np.sum(0.5 * Ud * inv * Ud + Ud * inv * d
                                            + 0.5 * (1 - 1 / prob["c"]) * d * inv * d)
            if zero_u and c == 1.0:
                assert is_terms == 0.0
            # q(x_j) dt is summed step by step in the oracle
            assert r["S"][k] == pytest.approx(plain + is_terms, rel=1e-12)


# ----------------------------------------------- closed-form tilted mean (T=1)

def _one_step_problem(c, u0, lam=1.0, nu=0.0, channel="state", count_law="poisson",
                      mark_scale=0.5, K=400_000, seed=11):
    params = {"Qf": [30.0, 30.0, 30.0, 30.0]}
    return W.cartpole_k1000(K=K, T=1, dt=0.05, sigma=2.0, c=c, lam=lam, nu=nu,
                            jump_channel=channel, count_law=count_law, mark_scale=mark_scale,
                            params=params, seed=seed), np.array([[u0]], dtype=np.float32)


def _quadratic_in_delta(prob, x0, u0):
    """phi(x1) = A d^2 + B d + const with x1 = a + b d (F affine in control)."""
    dt = prob["dt"]
    a = x0 + oracle.xdot(prob, x0, [u0]) * dt
    b = (oracle.xdot(prob, x0, [u0 + 1.0]) - oracle.xdot(prob, x0, [u0])) * dt
    Qf = np.array(prob["params"]["Qf"])
    g = np.array(prob["params"]["goal"])
    A = np.sum(Qf * b * b)
    B = 2.0 * np.sum(Qf * b * (a - g))
    return A, B


def _check_mc(prob, x0, U, expected):
    r = oracle.iteration(prob, x0, U, 0, want_delta=True)
    d = r["delta"][0, :, 0]
    w = r["w"]
    du = r["U"][0, 0] - U[0, 0]
    se = np.sqrt(np.sum(w * w * (d - du) ** 2))
    assert abs(du - expected) < 5 * se, (du, expected, se)
    assert se < 0.02 * max(1.0, abs(expected))  # the check is sharp
    return du, se


@pytest.mark.parametrize("c,u0", [(1.0, 0.7), (2.0, 0.7), (1.0, 0.0), (0.5, -0.4)])
def test_one_step_update_matches_tilted_gaussian_mean(c, u0):
    """With delta ~ N(0, c sigma^2) and S~(delta) = const + lambda [u delta /
    sigma^2 + (1 - 1/c) delta^2 / (2 sigma^2)] + A delta^2 + B delta, the
    weighted mean of delta is -(u/sigma^2 + B/lambda) / (1/sigma^2 + 2A/lambda),
    independent of c: the importance-sampling terms undo the change of
    sampling mean and variance (Eq. 33-36)."""
    prob, U = _one_step_problem(c, u0)
    x0 = np.array([0.3, 0.1, 2.5, 0.2], dtype=np.float32)
    A, B = _quadratic_in_delta(prob, x0.astype(np.float64), float(U[0, 0]))
    lam = prob["lam"]
    s2 = prob["sigma"][0] ** 2
    expected = -(U[0, 0] / s2 + B / lam) / (1.0 / s2 + 2.0 * A / lam)
    _check_mc(prob, x0, U, expected)


def test_one_step_update_with_control_channel_jumps_matches_mixture():
    """Control-channel Bernoulli jumps (Algorithm 1, Eq. 49): delta_eff is a
    two-component Gaussian mixture, N(0, s^2) w.p. 1 - mu and N(0, s^2 +
    sigma_J^2) w.p. mu; the tilted mean is the mixture of the tilted
    component means weighted by their tilted masses."""
    prob, U = _one_step_problem(1.0, 0.5, nu=8.0, channel="control", count_law="bernoulli",
                                mark_scale=3.0)
    x0 = np.array([0.3, 0.1, 2.5, 0.2], dtype=np.float32)
    A, B = _quadratic_in_delta(prob, x0.astype(np.float64), float(U[0, 0]))
    lam = prob["lam"]
    s2 = prob["sigma"][0] ** 2
    mu = prob["nu"] * prob["dt"]
    thr, _ = oracle.count_table(prob["nu"], prob["dt"], "bernoulli")
    pj = thr[0] / 2.0**32  # exact jump probability of the sampler
    assert abs(pj - mu) < 1e-9
    lin = U[0, 0] / s2 + B / lam
    num = den = 0.0
    for pi, var in ((1 - pj, s2), (pj, s2 + prob["mark_scale"][0] ** 2)):
        prec = 1.0 / var + 2.0 * A / lam  # c = 1: no variance-change term
        mean = -lin / prec
        mass = pi * np.sqrt(1.0 / (prec * var)) * np.exp(0.5 * lin * lin / prec)
        num += mass * mean
        den += mass
    _check_mc(prob, x0, U, num / den)


# ------------------------------------------------------------------ MPC step

def test_step_executes_first_control_and_shifts():
    prob = W.quadrotor_k4096(K=200, T=8, iters=3)
    rng = np.random.default_rng(7)
    x0, U = W.random_state(prob, rng), W.random_controls(prob, rng)
    Uo = U.astype(np.float64)
    for r in range(3):
        Uo = oracle.iteration(prob, x0, Uo, 40 + r)["U"]
    u0, Us = oracle.step(prob, x0, U, 40, 3)
    np.testing.assert_array_equal(u0, Uo[0])
    np.testing.assert_array_equal(Us[:-1], Uo[1:])
    np.testing.assert_array_equal(Us[-1], prob["u_init"])


def test_step_size_schedule_of_the_stochastic_optimisation_update():
    """Eq. 48-49 take a step size alpha^k per iteration; with alpha_decay = d
    iteration r of a step uses alpha * d^r, which is the plain iteration with
    that alpha (and d = 1 is the constant step of Eq. 36)."""
    base = W.quadrotor_k4096(K=150, T=6, iters=4, alpha=0.8)
    prob = dict(base, alpha_decay=0.5)
    rng = np.random.default_rng(9)
    x0, U = W.random_state(prob, rng), W.random_controls(prob, rng)
    Uo = U.astype(np.float64)
    for r in range(4):
        Uo = oracle.iteration(dict(prob, alpha=prob["alpha"] * 0.5 ** r), x0, Uo, 11 + r)["U"]
    u0, Us = oracle.step(prob, x0, U, 11, 4)
    np.testing.assert_allclose(u0, Uo[0], rtol=1e-15, atol=1e-15)
    np.testing.assert_allclose(Us[:-1], Uo[1:], rtol=1e-15, atol=1e-15)
    u0c, Usc = oracle.step(dict(base, alpha_decay=1.0), x0, U, 11, 4)
    u0b, Usb = oracle.step(base, x0, U, 11, 4)
    np.testing.assert_array_equal(Usc, Usb)
    # a smaller schedule moves the controls less from the first iteration on
    assert not np.allclose(Us, Usb)


def test_iterations_use_fresh_counters():
    prob = W.cartpole_k1000(K=50, T=5)
    x0, U = W.initial_state(prob), W.initial_controls(prob)
    a = oracle.iteration(prob, x0, U, 0, want_delta=True)["delta"]
    b = oracle.iteration(prob, x0, U, 1, want_delta=True)["delta"]
    c = oracle.iteration(prob, x0, U, 0, want_delta=True)["delta"]
    assert not np.array_equal(a, b)
    np.testing.assert_array_equal(a, c)
