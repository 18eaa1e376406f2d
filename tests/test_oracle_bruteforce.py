"""Brute-force pin of the oracle's whole iteration on tiny inputs (K <= 4,
T <= 3, plus one case with many jumps): a second, independent restatement in
plain Python floats of everything one iteration of Algorithm 1 computes --
the random draws from the Philox definition (normals by Box-Muller, counts
from scipy's Poisson CDF or the zero-one law, Normal or Laplace marks), the
cart-pole and quadrotor equations of motion written out from textbook
mechanics, the Euler rollout with state or control-channel jumps, the
augmented cost of Eq. 34-35, the weights of Eq. 36-37 and the update of
Eq. 37/49 -- compared element by element with the oracle.  A dropped cost
term, a wrong sign or index in the dynamics, a transposed draw or a wrong
normalisation anywhere in the oracle fails here."""

import math
import zlib

import numpy as np
import pytest
from scipy import stats

import oracle
from paper_1807_06108_gb300 import workloads as W
from tests.test_oracle_rng import _philox_py

M32 = 0xFFFFFFFF


def _uniform(w):
    return ((int(w) >> 9) + 0.5) * 2.0 ** -23


def _normals(words):
    out = []
    for a, b in ((0, 1), (2, 3)):
        r = math.sqrt(-2.0 * math.log(_uniform(words[a])))
        out += [r * math.cos(2 * math.pi * _uniform(words[b])),
                r * math.sin(2 * math.pi * _uniform(words[b]))]
    return out


def _bf16(v):
    """float64 -> float32 (RNE) -> bfloat16 (RNE), as the stored delta."""
    f = np.float32(v)
    bits = int(f.view(np.uint32))
    bits = (bits + 0x7FFF + ((bits >> 16) & 1)) & 0xFFFF0000
    return float(np.uint32(bits).view(np.float32))


def _count(prob, word):
    mu = prob["nu"] * prob["dt"]
    if prob["count_law"] == "bernoulli":
        return 1 if word < round(mu * 2.0 ** 32) else 0
    n = 0
    for i in range(1, 17):
        thr = math.ceil(stats.poisson.cdf(i - 1, mu) * 2.0 ** 32)
        if thr >= 2 ** 32:
            break
        n += word >= thr
    return n


def _draws(prob, k, j, it):
    """(delta_eff, J, N) of rollout k, step j, iteration it."""
    m = 1 if prob["system"] == "cartpole" else 4
    key = (prob["seed"] & M32, (prob["seed"] >> 32) & M32)
    delta = []
    for i in range(m):
        f = j * m + i
        z = _normals(_philox_py((k, f // 4, it, 0), key))[f % 4]
        delta.append(math.sqrt(prob["c"]) * prob["sigma"][i] * z)
    N = _count(prob, _philox_py((k, j // 4, it, 1), key)[j % 4])
    q = prob["q"]
    J = [0.0] * q
    for n in range(N):
        w = _philox_py((k, j, it, 2 + n), key)
        if prob["mark_law"] == "normal":
            z = _normals(w)
            for c in range(q):
                J[c] += prob["mark_scale"][c] * z[c]
        else:
            for c in range(q):
                u = _uniform(w[c]) - 0.5
                J[c] += -prob["mark_scale"][c] * math.copysign(1.0, u) * math.log(1 - 2 * abs(u))
    if prob["jump_channel"] == "control":
        delta = [delta[i] + J[i] for i in range(m)]
    if prob["noise_dtype"] == "bf16":
        delta = [_bf16(d) for d in delta]
    return delta, J, N


def _cartpole(x, v, p):
    """Frictionless cart-pole, point-mass pole, theta = 0 hanging down."""
    _, xd, th, thd = x
    s, c = math.sin(th), math.cos(th)
    D = p["mc"] + p["mp"] * s * s
    xdd = (v[0] + p["mp"] * s * (p["l"] * thd * thd + p["g"] * c)) / D
    thdd = (-v[0] * c - p["mp"] * p["l"] * thd * thd * c * s
            - (p["mc"] + p["mp"]) * p["g"] * s) / (p["l"] * D)
    return [xd, xdd, thd, thdd]


def _quadrotor(x, f, p):
    """Rigid body with ZYX Euler angles and four rotors in a '+' layout."""
    v, (ph, th, ps), om = x[3:6], x[6:9], x[9:12]
    sph, cph, sth, cth, sps, cps = (math.sin(ph), math.cos(ph), math.sin(th), math.cos(th),
                                    math.sin(ps), math.cos(ps))
    a = sum(f) / p["mass"]
    acc = [a * (cph * sth * cps + sph * sps), a * (cph * sth * sps - sph * cps),
           a * cph * cth - p["g"]]
    tth = sth / cth
    eta_d = [om[0] + sph * tth * om[1] + cph * tth * om[2],
             cph * om[1] - sph * om[2],
             (sph * om[1] + cph * om[2]) / cth]
    Jx, Jy, Jz = p["J"]
    tau = [p["arm"] * (f[1] - f[3]), p["arm"] * (f[2] - f[0]),
           p["kappa"] * (f[0] - f[1] + f[2] - f[3])]
    Jw = [Jx * om[0], Jy * om[1], Jz * om[2]]
    cross = [om[1] * Jw[2] - om[2] * Jw[1], om[2] * Jw[0] - om[0] * Jw[2],
             om[0] * Jw[1] - om[1] * Jw[0]]
    om_d = [(tau[0] - cross[0]) / Jx, (tau[1] - cross[1]) / Jy, (tau[2] - cross[2]) / Jz]
    return list(v) + acc + eta_d + om_d


def _state_cost(prob, x, terminal):
    p = prob["params"]
    if prob["system"] == "cartpole":
        Q = p["Qf"] if terminal else p["Q"]
        return sum(Q[i] * (x[i] - p["goal"][i]) ** 2 for i in range(4))
    c = (p["wp"] * sum((x[i] - p["goal"][i]) ** 2 for i in range(3))
         + p["wv"] * sum(v * v for v in x[3:6]) + p["weta"] * sum(e * e for e in x[6:9])
         + p["wom"] * sum(w * w for w in x[9:12]))
    if not terminal and sum((x[i] - p["obs"][i]) ** 2 for i in range(3)) < p["obs_r"] ** 2:
        c += p["obs_cost"]
    return c


def _iteration(prob, x0, U, it):
    """(S, delta, U_new) of one iteration, written out in plain floats."""
    K, T, dt, lam, c = prob["K"], prob["T"], prob["dt"], prob["lam"], prob["c"]
    m = 1 if prob["system"] == "cartpole" else 4
    inv_s2 = [1.0 / (s * s) for s in prob["sigma"]]
    f = _cartpole if prob["system"] == "cartpole" else _quadrotor
    S, deltas = [], []
    for k in range(K):
        x = [float(v) for v in x0]
        s = 0.0
        dk = []
        for j in range(T):
            d, J, N = _draws(prob, k, j, it)
            dk.append(d)
            u = [float(U[j][i]) for i in range(m)]
            s += _state_cost(prob, x, False) * dt + lam * (
                0.5 * sum(u[i] * inv_s2[i] * u[i] for i in range(m))
                + sum(u[i] * inv_s2[i] * d[i] for i in range(m))
                + 0.5 * (1 - 1 / c) * sum(d[i] * inv_s2[i] * d[i] for i in range(m)))
            xd = f(x, [u[i] + d[i] for i in range(m)], prob["params"])
            x = [x[i] + xd[i] * dt for i in range(len(x))]
            if prob["jump_channel"] == "state" and N > 0:
                scale = math.sqrt(dt) if prob["jump_sqrt_dt"] else 1.0
                for cc, row in enumerate(prob["jump_rows"]):
                    x[row] += scale * J[cc]
        s += _state_cost(prob, x, True)
        S.append(s)
        deltas.append(dk)
    rho = min(S)
    e = [math.exp(-(s - rho) / lam) for s in S]
    Z = sum(e)
    U_new = [[float(U[j][i]) + prob["alpha"] * sum(e[k] * deltas[k][j][i] for k in range(K)) / Z
              for i in range(m)] for j in range(T)]
    return np.array(S), np.array(deltas), np.array(U_new)


def _cases():
    out = {
        "cartpole_state_normal": W.cartpole_k1000(K=3, T=3, nu=40.0, mark_scale=0.7, lam=2.0),
        "cartpole_control_bernoulli_c2_bf16": W.cartpole_k1000(
            K=4, T=3, nu=30.0, jump_channel="control", count_law="bernoulli", c=2.0,
            noise_dtype="bf16", alpha=0.5),
        "quadrotor_state_laplace_sqrtdt": W.quadrotor_k4096(
            K=4, T=3, nu=60.0, mark_law="laplace", jump_sqrt_dt=True, lam=5.0),
        "quadrotor_control_normal_c05": W.quadrotor_k4096(
            K=3, T=2, nu=80.0, jump_channel="control", mark_scale=0.3, c=0.5, lam=3.0),
        "quadrotor_rows_with_rates": W.quadrotor_k4096(
            K=2, T=3, nu=90.0, jump_rows=[3, 4, 5, 11], mark_scale=0.2, seed=5 | (3 << 32)),
        "cartpole_many_jumps": W.cartpole_k1000(K=4, T=6, nu=100.0, mark_scale=0.1, seed=11),
    }
    return out


CASES = _cases()


@pytest.mark.parametrize("name", list(CASES))
def test_oracle_iteration_equals_plain_restatement(name):
    prob = CASES[name]
    rng = np.random.default_rng(zlib.crc32(name.encode()))
    x0 = W.random_state(prob, rng, 0.3).astype(np.float64)
    U = W.random_controls(prob, rng, 0.5).astype(np.float64)
    it = 7
    S, delta, U_new = _iteration(prob, x0, U, it)
    got = oracle.iteration(prob, x0, U, it, want_delta=True)
    got_r = oracle.rollouts(prob, x0, U, it, counts=True)
    assert got_r["counts"].sum() > 0, "the case should draw jumps"
    np.testing.assert_allclose(got["S"], S, rtol=1e-11, atol=1e-11)
    # oracle delta is [T][K][m]
    np.testing.assert_allclose(got["delta"], delta.transpose(1, 0, 2), rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(got["U"], U_new, rtol=1e-11, atol=1e-12)
