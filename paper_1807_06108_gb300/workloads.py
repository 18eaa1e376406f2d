"""Seeded synthetic workloads for MPPI on jump-diffusion processes.

This module only *describes* problems: plant constants, noise laws, sizes,
seeds, initial states and control sequences, batched-instance draws and
request-arrival traces.  It holds none of the method's arithmetic, so both
the CUDA binding and the FP64 oracle can read the same problem description.

Every floating-point constant is rounded to the nearest float32 here, so that
the float32 device configuration and the float64 oracle see identical values.

The paper (Sec. VI) names a cart-pole swing-up and a quadrotor point-to-point
flight but prints neither equations nor constants; the constants below are the
chosen ones (cart 1.0 kg, pole 0.1 kg at 0.5 m; quadrotor 1.0 kg, inertia
diag(0.01, 0.01, 0.02), arm 0.2 m, yaw coefficient 0.02 m).
"""

from __future__ import annotations

import copy
import math

import numpy as np

SYSTEMS = ("cartpole", "quadrotor")
STATE_DIM = {"cartpole": 4, "quadrotor": 12}
CONTROL_DIM = {"cartpole": 1, "quadrotor": 4}


def f32(x):
    """Nearest float32 value, returned as a Python float (or list of them)."""
    if isinstance(x, (list, tuple, np.ndarray)):
        return [float(np.float32(v)) for v in x]
    return float(np.float32(x))


CARTPOLE_PARAMS = {
    "mc": 1.0,
    "mp": 0.1,
    "l": 0.5,
    "g": 9.81,
    # swing-up target: cart at the origin, pole upright (theta = pi, theta = 0
    # is hanging down)
    "goal": [0.0, 0.0, math.pi, 0.0],
    "Q": [1.0, 0.1, 10.0, 0.1],
    "Qf": [1.0, 0.1, 10.0, 0.1],
}

QUADROTOR_PARAMS = {
    "mass": 1.0,
    "J": [0.01, 0.01, 0.02],
    "arm": 0.2,
    "kappa": 0.02,
    "g": 9.81,
    "goal": [4.0, 0.0, 1.0],
    "wp": 10.0,
    "wv": 1.0,
    "weta": 1.0,
    "wom": 0.1,
    "obs": [2.0, 0.0, 1.0],
    "obs_r": 0.5,
    "obs_cost": 1.0e4,
}


def _canon_params(system, params):
    base = copy.deepcopy(CARTPOLE_PARAMS if system == "cartpole" else QUADROTOR_PARAMS)
    if params:
        base.update(params)
    return {k: f32(v) for k, v in base.items()}


def problem(system, K, T, dt, *, sigma, nu, mark_scale, mark_law="normal",
            count_law="poisson", jump_channel="state", jump_rows=None, lam=1.0,
            c=1.0, alpha=1.0, alpha_decay=1.0, noise_dtype="f32", seed=0, jump_sqrt_dt=False,
            params=None, u_init=None, iters=1, name=None):
    """Build one problem dictionary (all floats float32-representable)."""
    if system not in SYSTEMS:
        raise ValueError(f"unknown system {system!r}")
    m = CONTROL_DIM[system]
    prm = _canon_params(system, params)
    if np.isscalar(sigma):
        sigma = [sigma] * m
    if jump_channel == "control":
        q = m
        rows = list(range(m))
    else:
        if jump_rows is None:
            jump_rows = [1, 3] if system == "cartpole" else [3, 4, 5]
        rows = list(jump_rows)
        q = len(rows)
    if np.isscalar(mark_scale):
        mark_scale = [mark_scale] * q
    if u_init is None:
        u_init = [0.0] if system == "cartpole" else [prm["mass"] * prm["g"] / 4.0] * 4
    return {
        "name": name or (f"{system}_K{K}_T{T}_it{iters}"
                         + ("_bf16" if noise_dtype == "bf16" else "")),
        "system": system,
        "K": int(K),
        "T": int(T),
        "dt": f32(dt),
        "lam": f32(lam),
        "c": f32(c),
        "alpha": f32(alpha),
        "alpha_decay": f32(alpha_decay),
        "sigma": f32(list(sigma)),
        "nu": f32(nu),
        "count_law": count_law,
        "mark_law": mark_law,
        "mark_scale": f32(list(mark_scale)),
        "jump_channel": jump_channel,
        "jump_rows": rows,
        "q": q,
        "jump_sqrt_dt": bool(jump_sqrt_dt),
        "noise_dtype": noise_dtype,
        "u_init": f32(list(u_init)),
        "seed": int(seed) & 0xFFFFFFFFFFFFFFFF,
        "params": prm,
        "iters": int(iters),
    }


def initial_state(prob):
    """Plant state at the start of a solve: cart-pole at rest hanging down at
    the origin; quadrotor hovering level at (0, 0, 1)."""
    if prob["system"] == "cartpole":
        return np.zeros(4, dtype=np.float32)
    x = np.zeros(12, dtype=np.float32)
    x[2] = 1.0
    return x


def initial_controls(prob):
    """Control sequence U (T x m, float32) initialised to u_init."""
    m = CONTROL_DIM[prob["system"]]
    return np.tile(np.asarray(prob["u_init"], dtype=np.float32), (prob["T"], 1)).reshape(prob["T"], m)


def random_state(prob, rng, scale=0.3):
    """A seeded perturbed plant state (tests exercise non-trivial states)."""
    x = initial_state(prob).astype(np.float64)
    x = x + scale * rng.standard_normal(x.shape)
    if prob["system"] == "quadrotor":
        x[6:9] *= 0.5  # keep Euler angles well inside (-pi/2, pi/2)
    return x.astype(np.float32)


def random_controls(prob, rng, scale=0.5):
    U = initial_controls(prob).astype(np.float64)
    U = U + scale * rng.standard_normal(U.shape)
    return U.astype(np.float32)


# ---------------------------------------------------------------------------
# The five named workloads
# ---------------------------------------------------------------------------

def cartpole_k1000(K=1000, T=50, dt=0.02, **kw):
    """Cart-pole swing-up: K=1000 rollouts, T=50 steps of 0.02 s, one
    iteration, control noise N(0, 1.0^2), state jumps on (xdot, thetadot) at
    1.0/s with N(0, 0.5^2) marks, temperature 1.0, seed 0."""
    args = dict(sigma=1.0, nu=1.0, mark_scale=0.5, lam=1.0, seed=0, iters=1)
    args.update(kw)
    return problem("cartpole", K, T, dt, **args)


def quadrotor_k4096(K=4096, T=100, dt=0.01, **kw):
    """Quadrotor waypoint flight: K=4096, T=100 steps of 0.01 s, 10 iterations
    per MPC step, rotor noise N(0, 0.2^2), velocity jumps at 2.0/s with
    N(0, 1.0^2) marks per axis, obstacle penalty 1e4, seed 0."""
    args = dict(sigma=0.2, nu=2.0, mark_scale=1.0, lam=1.0, seed=0, iters=10)
    args.update(kw)
    return problem("quadrotor", K, T, dt, **args)


def quadrotor_alg1(K=4096, T=100, dt=0.01, **kw):
    """The quadrotor workload in Algorithm 1's literal form: jumps enter the
    control channels (H = G, q = m) with the zero-one jump timer, the step
    size decays over the iterations (alpha^k of Eq. 48-49, alpha_decay 0.8);
    otherwise as quadrotor_k4096."""
    args = dict(sigma=0.2, nu=2.0, mark_scale=0.5, lam=1.0, seed=0, iters=10,
                jump_channel="control", count_law="bernoulli", alpha_decay=0.8,
                name=f"quadrotor_K{K}_T{T}_alg1")
    args.update(kw)
    return problem("quadrotor", K, T, dt, **args)


def large_quadrotor(K=65536, T=200, dt=0.005, **kw):
    """Large quadrotor: K=65536, T=200 steps of 0.005 s, 5 iterations,
    Laplace(0, 1.0) velocity-jump marks at 5.0/s, bfloat16 noise storage."""
    args = dict(sigma=0.2, nu=5.0, mark_scale=1.0, mark_law="laplace", lam=1.0, seed=0,
                iters=5, noise_dtype="bf16")
    args.update(kw)
    return problem("quadrotor", K, T, dt, **args)


BATCH_K_CHOICES = (512, 1024, 2048, 4096, 8192)


def batched_instances(n=256, seed=0, noise_dtype="bf16"):
    """Independent MPC instances for the batched form: instance i is a
    cart-pole if i is even and a quadrotor otherwise, K uniform over
    {512, ..., 8192}, T uniform in [30, 150], jump rate uniform in [0.5, 3]/s,
    other parameters as in the two single-instance workloads; instance i uses
    Philox key (seed, i), i.e. seed | (i << 32)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n):
        K = int(rng.choice(BATCH_K_CHOICES))
        T = int(rng.integers(30, 151))
        nu = float(rng.uniform(0.5, 3.0))
        s = (int(seed) & 0xFFFFFFFF) | (i << 32)
        if i % 2 == 0:
            p = cartpole_k1000(K=K, T=T, nu=nu, seed=s, noise_dtype=noise_dtype,
                               name=f"batch{i}_cartpole_K{K}_T{T}")
        else:
            p = quadrotor_k4096(K=K, T=T, nu=nu, seed=s, noise_dtype=noise_dtype,
                                name=f"batch{i}_quadrotor_K{K}_T{T}")
        out.append(p)
    return out


SERVE_K_CHOICES = (1024, 2048, 4096, 8192, 16384)
SERVE_T_CHOICES = (50, 100, 150, 200)


def served_sessions(n=64, seed=0):
    """Sessions of the served form: mixed systems, K in {1024..16384},
    T in {50..200}; cart-pole sessions run 1 iteration per MPC step and
    quadrotor sessions 10."""
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    out = []
    for i in range(n):
        K = int(rng.choice(SERVE_K_CHOICES))
        T = int(rng.choice(SERVE_T_CHOICES))
        s = (int(seed) & 0xFFFFFFFF) | ((1000 + i) << 32)
        if i % 2 == 0:
            p = cartpole_k1000(K=K, T=T, seed=s, name=f"session{i}_cartpole_K{K}_T{T}")
        else:
            p = quadrotor_k4096(K=K, T=T, seed=s, name=f"session{i}_quadrotor_K{K}_T{T}")
        out.append(p)
    return out


def arrival_trace(rate_hz=2000.0, duration_s=60.0, n_sessions=64, seed=0):
    """Poisson request arrivals: exponential inter-arrival times at `rate_hz`
    for `duration_s`, each assigned to a uniformly drawn session.  Returns
    (times_s float64 array, session_ids int32 array)."""
    rng = np.random.Generator(np.random.PCG64(seed + 2))
    n_guess = int(rate_hz * duration_s * 1.2) + 16
    gaps = rng.exponential(1.0 / rate_hz, size=n_guess)
    t = np.cumsum(gaps)
    t = t[t < duration_s]
    sess = rng.integers(0, n_sessions, size=t.shape[0]).astype(np.int32)
    return t, sess


def state_drift(prob, rng, scale=0.01):
    """Small seeded drift added to a session's state between requests."""
    n = STATE_DIM[prob["system"]]
    return (scale * rng.standard_normal(n)).astype(np.float32)
