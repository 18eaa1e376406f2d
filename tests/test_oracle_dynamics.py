"""Pins for the oracle's plants (control-affine drift, Eq. 4) and costs
(Eq. 3): closed forms at special states, conservation laws of the
frictionless mechanics, and the rigid-body kinematics checked against
scipy's rotation routines."""

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from paper_1807_06108_gb300 import workloads as W

CP = W.cartpole_k1000()
QR = W.quadrotor_k4096()


def _rk4(f, x, h, steps):
    for _ in range(steps):
        k1 = f(x)
        k2 = f(x + 0.5 * h * k1)
        k3 = f(x + 0.5 * h * k2)
        k4 = f(x + h * k3)
        x = x + h / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
    return x


# ----------------------------------------------------------------- cart-pole

def test_cartpole_pushed_at_rest_hanging():
    xd = oracle.xdot(CP, [0, 0, 0, 0], [1.0])
    p = CP["params"]
    np.testing.assert_allclose(xd, [0, 1.0 / p["mc"], 0, -1.0 / (p["l"] * p["mc"])], rtol=1e-15)


def test_cartpole_horizontal_pole_falls_at_g_over_l():
    xd = oracle.xdot(CP, [0, 0, np.pi / 2, 0], [0.0])
    p = CP["params"]
    np.testing.assert_allclose(xd[1], 0.0, atol=1e-12)
    np.testing.assert_allclose(xd[3], -p["g"] / p["l"], rtol=1e-12)


def _cp_energy_momentum(x):
    p = CP["params"]
    mc, mp, l, g = p["mc"], p["mp"], p["l"], p["g"]
    xd, th, thd = x[1], x[2], x[3]
    E = 0.5 * (mc + mp) * xd**2 + mp * l * xd * thd * np.cos(th) + 0.5 * mp * l**2 * thd**2 \
        - mp * g * l * np.cos(th)
    P = (mc + mp) * xd + mp * l * thd * np.cos(th)
    return E, P


def test_cartpole_conserves_energy_and_momentum_unforced():
    rng = np.random.default_rng(0)
    for _ in range(5):
        x = rng.standard_normal(4) * [1, 1, 2, 3]
        E0, P0 = _cp_energy_momentum(x)
        x1 = _rk4(lambda s: oracle.xdot(CP, s, [0.0]), x, 1e-3, 2000)
        E1, P1 = _cp_energy_momentum(x1)
        assert abs(E1 - E0) < 1e-7 * max(1, abs(E0))
        assert abs(P1 - P0) < 1e-9 * max(1, abs(P0))


def test_cartpole_force_power_balance():
    """With a constant force f the energy changes by f times the cart travel."""
    rng = np.random.default_rng(1)
    x = rng.standard_normal(4)
    f = 0.7
    E0, _ = _cp_energy_momentum(x)
    x1 = _rk4(lambda s: oracle.xdot(CP, s, [f]), x, 1e-3, 1500)
    E1, _ = _cp_energy_momentum(x1)
    assert abs((E1 - E0) - f * (x1[0] - x[0])) < 1e-7


def test_cartpole_costs():
    p = CP["params"]
    goal = np.array(p["goal"])
    assert oracle.state_cost(CP, goal) == 0.0
    for i in range(4):
        e = np.zeros(4)
        e[i] = 2.0
        assert oracle.state_cost(CP, goal + e) == pytest.approx(4.0 * p["Q"][i], rel=1e-14)
        assert oracle.terminal_cost(CP, goal + e) == pytest.approx(4.0 * p["Qf"][i], rel=1e-14)


# ----------------------------------------------------------------- quadrotor

def _hover(x=None):
    p = QR["params"]
    h = p["mass"] * p["g"] / 4.0
    return np.array([h, h, h, h])


def test_quadrotor_hover_is_equilibrium():
    x = np.zeros(12)
    x[:3] = [0.3, -1.0, 2.0]
    xd = oracle.xdot(QR, x, _hover())
    np.testing.assert_allclose(xd, 0.0, atol=1e-12)


def test_quadrotor_yaw_roll_pitch_torques():
    p = QR["params"]
    J, L, kap = p["J"], p["arm"], p["kappa"]
    x = np.zeros(12)
    a, b = 3.0, 2.0
    xd = oracle.xdot(QR, x, [a, b, a, b])
    np.testing.assert_allclose(xd[9:11], 0.0, atol=1e-12)
    assert xd[11] == pytest.approx(2 * kap * (a - b) / J[2], rel=1e-12)
    d = 0.5
    xd = oracle.xdot(QR, x, [2.0, 2.0, 2.0 + d, 2.0])
    assert xd[10] == pytest.approx(L * d / J[1], rel=1e-12)
    assert xd[9] == pytest.approx(0.0, abs=1e-12)
    xd = oracle.xdot(QR, x, [2.0, 2.0 + d, 2.0, 2.0])
    assert xd[9] == pytest.approx(L * d / J[0], rel=1e-12)


def test_quadrotor_thrust_direction_matches_scipy_rotation():
    p = QR["params"]
    rng = np.random.default_rng(2)
    for _ in range(50):
        eta = rng.uniform(-1.2, 1.2, size=3)
        x = np.zeros(12)
        x[6:9] = eta
        f = rng.uniform(0.5, 4.0, size=4)
        xd = oracle.xdot(QR, x, f)
        R = Rotation.from_euler("ZYX", [eta[2], eta[1], eta[0]]).as_matrix()
        acc = f.sum() / p["mass"] * R[:, 2] - np.array([0, 0, p["g"]])
        np.testing.assert_allclose(xd[3:6], acc, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(xd[0:3], x[3:6])


def test_quadrotor_euler_rates_match_body_rate_kinematics():
    """eta' = W(eta) omega equals the derivative of the ZYX angles of
    R(eta) exp([omega]x t) at t = 0 (body-frame rates)."""
    rng = np.random.default_rng(3)
    h = 1e-6
    for _ in range(30):
        eta = rng.uniform(-1.0, 1.0, size=3)
        om = rng.standard_normal(3)
        x = np.zeros(12)
        x[6:9] = eta
        x[9:12] = om
        xd = oracle.xdot(QR, x, _hover())
        R0 = Rotation.from_euler("ZYX", [eta[2], eta[1], eta[0]])

        def angles(t):
            a = (R0 * Rotation.from_rotvec(om * t)).as_euler("ZYX")
            return np.array([a[2], a[1], a[0]])

        num = (angles(h) - angles(-h)) / (2 * h)
        np.testing.assert_allclose(xd[6:9], num, rtol=1e-6, atol=1e-6)


def test_quadrotor_torque_free_rotation_conserves_energy_and_momentum():
    p = QR["params"]
    J = np.array(p["J"])
    rng = np.random.default_rng(4)
    x = np.zeros(12)
    x[9:12] = rng.standard_normal(3) * 3
    f = _hover()  # equal thrusts: zero torque

    def rot(s):
        full = x.copy()
        full[9:12] = s
        return oracle.xdot(QR, full, f)[9:12]

    w0 = x[9:12]
    w1 = _rk4(rot, w0, 1e-4, 5000)
    ke = lambda w: 0.5 * np.sum(J * w * w)
    L2 = lambda w: np.sum((J * w) ** 2)
    assert abs(ke(w1) - ke(w0)) < 1e-9 * ke(w0)
    assert abs(L2(w1) - L2(w0)) < 1e-9 * L2(w0)
    # the non-isotropic body really precesses: the test has teeth
    assert np.max(np.abs(w1 - w0)) > 1e-2


def test_quadrotor_costs_and_obstacle_indicator():
    p = QR["params"]
    x = np.zeros(12)
    x[:3] = p["goal"]
    assert oracle.state_cost(QR, x) == 0.0
    x = np.zeros(12)
    x[:3] = p["obs"]
    d2 = np.sum((np.array(p["obs"]) - np.array(p["goal"])) ** 2)
    assert oracle.state_cost(QR, x) == pytest.approx(p["wp"] * d2 + p["obs_cost"], rel=1e-14)
    assert oracle.terminal_cost(QR, x) == pytest.approx(p["wp"] * d2, rel=1e-14)
    x[0] = p["obs"][0] + p["obs_r"] + 1e-9
    assert oracle.state_cost(QR, x) < p["obs_cost"]
    x = np.zeros(12)
    x[3:6], x[6:9], x[9:12] = [1, 2, 3], [0.1, 0.2, 0.3], [1, 1, 1]
    x[:3] = p["goal"]
    ref = p["wv"] * 14 + p["weta"] * 0.14 + p["wom"] * 3
    assert oracle.state_cost(QR, x) == pytest.approx(ref, rel=1e-12)


def test_euler_step_and_state_jump_wiring():
    """x_{j+1} = x_j + F(x_j, u_j + delta_eff_j) dt + H J_j along a rollout."""
    for prob in (W.cartpole_k1000(T=12, nu=30.0), W.quadrotor_k4096(T=12, nu=30.0),
                 W.quadrotor_k4096(T=12, nu=30.0, jump_sqrt_dt=True)):
        rng = np.random.default_rng(5)
        x0 = W.random_state(prob, rng)
        U = W.random_controls(prob, rng)
        r = oracle.rollouts(prob, x0, U, 3, 10, 6, delta=True, jumps=True, traj=True, counts=True)
        assert r["counts"].sum() > 0
        s = np.sqrt(prob["dt"]) if prob["jump_sqrt_dt"] else 1.0
        for kk in range(6):
            tr = r["traj"][kk]
            for j in range(prob["T"]):
                v = U[j].astype(np.float64) + r["delta"][j, kk]
                nxt = tr[j] + oracle.xdot(prob, tr[j], v) * prob["dt"]
                for c, row in enumerate(prob["jump_rows"]):
                    nxt[row] += s * r["J"][j, kk, c]
                np.testing.assert_allclose(tr[j + 1], nxt, rtol=1e-13, atol=1e-13)
