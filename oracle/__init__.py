"""FP64 CPU oracle for MPPI on jump-diffusion processes -- TEST INFRASTRUCTURE.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its binding) never imports, links or executes anything here, and nothing here
imports the product package: problems arrive as the plain dictionaries built
by ``paper_1807_06108_gb300.workloads`` (a description, not arithmetic).

The arithmetic lives in ``oracle.c`` (plain C, double precision, OpenMP over
rollouts), compiled on first use into ``oracle/_build/liboracle.so`` with
``-O2 -fno-fast-math -ffp-contract=off`` so that results are the same on x86
and Arm hosts.  This module marshals numpy arrays to it.

Parity pins that hold for every function here are in ``tests/test_oracle_*.py``.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

MAX_JUMPS = 16
STATUS = {0: "ok", 1: "invalid argument", 2: "out of memory", 5: "all costs non-finite"}


class OracleError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"oracle {what}: {STATUS.get(code, code)}")
        self.code = code


def build(force=False):
    """Compile oracle.c into _build/liboracle.so (no-op when up to date)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fno-fast-math", "-ffp-contract=off", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Problem(ctypes.Structure):
    _fields_ = [
        ("system", ctypes.c_int32), ("K", ctypes.c_int32), ("T", ctypes.c_int32),
        ("dt", ctypes.c_double), ("lam", ctypes.c_double), ("c", ctypes.c_double),
        ("alpha", ctypes.c_double),
        ("sigma", ctypes.c_double * 4), ("nu", ctypes.c_double),
        ("count_law", ctypes.c_int32), ("mark_law", ctypes.c_int32),
        ("mark_scale", ctypes.c_double * 4),
        ("jump_channel", ctypes.c_int32), ("jump_sqrt_dt", ctypes.c_int32),
        ("noise_bf16", ctypes.c_int32), ("q", ctypes.c_int32),
        ("jump_rows", ctypes.c_int32 * 4),
        ("u_init", ctypes.c_double * 4), ("seed", ctypes.c_uint64),
        ("cp_mc", ctypes.c_double), ("cp_mp", ctypes.c_double), ("cp_l", ctypes.c_double),
        ("cp_g", ctypes.c_double), ("cp_goal", ctypes.c_double * 4),
        ("cp_Q", ctypes.c_double * 4), ("cp_Qf", ctypes.c_double * 4),
        ("qr_mass", ctypes.c_double), ("qr_J", ctypes.c_double * 3),
        ("qr_arm", ctypes.c_double), ("qr_kappa", ctypes.c_double), ("qr_g", ctypes.c_double),
        ("qr_goal", ctypes.c_double * 3), ("qr_wp", ctypes.c_double), ("qr_wv", ctypes.c_double),
        ("qr_weta", ctypes.c_double), ("qr_wom", ctypes.c_double),
        ("qr_obs", ctypes.c_double * 3), ("qr_obs_r", ctypes.c_double),
        ("qr_obs_cost", ctypes.c_double),
        ("alpha_decay", ctypes.c_double),
    ]


_P = ctypes.POINTER
_d = _P(ctypes.c_double)
_u8 = _P(ctypes.c_uint8)
_u32 = _P(ctypes.c_uint32)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            pp = _P(_Problem)
            lib.orc_philox4x32_10.argtypes = [_u32, _u32, _u32]
            lib.orc_uniform.argtypes = [ctypes.c_uint32]
            lib.orc_uniform.restype = ctypes.c_double
            lib.orc_normals4.argtypes = [_u32, _d]
            lib.orc_count_table.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int32,
                                            _u32, _P(ctypes.c_int32)]
            lib.orc_count_table.restype = ctypes.c_int
            lib.orc_xdot.argtypes = [pp, _d, _d, _d]
            lib.orc_state_cost.argtypes = [pp, _d]
            lib.orc_state_cost.restype = ctypes.c_double
            lib.orc_terminal_cost.argtypes = [pp, _d]
            lib.orc_terminal_cost.restype = ctypes.c_double
            lib.orc_bf16_round.argtypes = [ctypes.c_double]
            lib.orc_bf16_round.restype = ctypes.c_double
            lib.orc_bf16_ambiguous.argtypes = [ctypes.c_double]
            lib.orc_bf16_ambiguous.restype = ctypes.c_int
            lib.orc_obstacle_margin.argtypes = [pp, _d]
            lib.orc_obstacle_margin.restype = ctypes.c_double
            lib.orc_rollouts.argtypes = [pp, _d, _d, ctypes.c_uint32, ctypes.c_int32,
                                         ctypes.c_int32, _d, _u8, _d, _d, _u8, _d, _d,
                                         ctypes.c_int32]
            lib.orc_rollouts.restype = ctypes.c_int
            lib.orc_softmin.argtypes = [ctypes.c_int32, _d, ctypes.c_double, _d, _d]
            lib.orc_softmin.restype = ctypes.c_int
            lib.orc_update.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _d, _d,
                                       ctypes.c_double, _d]
            lib.orc_iteration.argtypes = [pp, _d, _d, ctypes.c_uint32, _d, _d, _u8, _d, _d,
                                          _u8, ctypes.c_int32]
            lib.orc_iteration.restype = ctypes.c_int
            lib.orc_step.argtypes = [pp, _d, _d, ctypes.c_uint32, ctypes.c_int32, _d,
                                     ctypes.c_int32]
            lib.orc_step.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a, typ):
    if a is None:
        return ctypes.cast(None, typ)
    return a.ctypes.data_as(typ)


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def state_dim(prob):
    return 4 if prob["system"] == "cartpole" else 12


def control_dim(prob):
    return 1 if prob["system"] == "cartpole" else 4


def make_problem(prob):
    """ctypes problem struct from a workload dictionary."""
    P = _Problem()
    P.system = 0 if prob["system"] == "cartpole" else 1
    P.K, P.T = prob["K"], prob["T"]
    P.dt, P.lam, P.c, P.alpha = prob["dt"], prob["lam"], prob["c"], prob["alpha"]
    P.alpha_decay = prob.get("alpha_decay", 1.0)
    for i, s in enumerate(prob["sigma"]):
        P.sigma[i] = s
    P.nu = prob["nu"]
    P.count_law = {"poisson": 0, "bernoulli": 1}[prob["count_law"]]
    P.mark_law = {"normal": 0, "laplace": 1}[prob["mark_law"]]
    for i, s in enumerate(prob["mark_scale"]):
        P.mark_scale[i] = s
    P.jump_channel = {"state": 0, "control": 1}[prob["jump_channel"]]
    P.jump_sqrt_dt = int(prob["jump_sqrt_dt"])
    P.noise_bf16 = int(prob["noise_dtype"] == "bf16")
    P.q = prob["q"]
    for i, r in enumerate(prob["jump_rows"]):
        P.jump_rows[i] = r
    for i, u in enumerate(prob["u_init"]):
        P.u_init[i] = u
    P.seed = prob["seed"]
    p = prob["params"]
    if prob["system"] == "cartpole":
        P.cp_mc, P.cp_mp, P.cp_l, P.cp_g = p["mc"], p["mp"], p["l"], p["g"]
        for i in range(4):
            P.cp_goal[i], P.cp_Q[i], P.cp_Qf[i] = p["goal"][i], p["Q"][i], p["Qf"][i]
    else:
        P.qr_mass = p["mass"]
        for i in range(3):
            P.qr_J[i], P.qr_goal[i], P.qr_obs[i] = p["J"][i], p["goal"][i], p["obs"][i]
        P.qr_arm, P.qr_kappa, P.qr_g = p["arm"], p["kappa"], p["g"]
        P.qr_wp, P.qr_wv, P.qr_weta, P.qr_wom = p["wp"], p["wv"], p["weta"], p["wom"]
        P.qr_obs_r, P.qr_obs_cost = p["obs_r"], p["obs_cost"]
    return P


# --------------------------------------------------------------------------
# Random stream
# --------------------------------------------------------------------------

def philox(ctr, key):
    """Philox4x32-10 block for counter (4 words) and key (2 words)."""
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.orc_philox4x32_10(_ptr(c, _u32), _ptr(k, _u32), _ptr(out, _u32))
    return out


def uniform(word):
    return _load().orc_uniform(int(word))


def normals4(words):
    w = np.ascontiguousarray(words, dtype=np.uint32)
    z = np.zeros(4)
    _load().orc_normals4(_ptr(w, _u32), _ptr(z, _d))
    return z


def count_table(nu, dt, law="poisson"):
    """(thresholds uint32[16], nmax) for jump rate nu and step dt."""
    thr = np.zeros(MAX_JUMPS, dtype=np.uint32)
    nmax = ctypes.c_int32(0)
    st = _load().orc_count_table(float(nu), float(dt), {"poisson": 0, "bernoulli": 1}[law],
                                 _ptr(thr, _u32), ctypes.byref(nmax))
    if st:
        raise OracleError(st, "count_table")
    return thr, nmax.value


def bf16_round(x):
    return _load().orc_bf16_round(float(x))


def bf16_ambiguous(x):
    """True when the float64 value x lies within 2^-20 |x| of the midpoint
    between the two bfloat16 neighbours of float32(x) (the rollouts whose
    stored bfloat16 perturbation may legitimately differ between a float32
    and a float64 computation)."""
    return bool(_load().orc_bf16_ambiguous(float(x)))


# --------------------------------------------------------------------------
# Plants and costs
# --------------------------------------------------------------------------

def xdot(prob, x, v):
    """F(x, v) = f(x) + G(x) v for the problem's plant."""
    P = make_problem(prob)
    x = _f64(x)
    v = _f64(v)
    out = np.zeros(state_dim(prob))
    _load().orc_xdot(ctypes.byref(P), _ptr(x, _d), _ptr(v, _d), _ptr(out, _d))
    return out


def state_cost(prob, x):
    P = make_problem(prob)
    x = _f64(x)
    return _load().orc_state_cost(ctypes.byref(P), _ptr(x, _d))


def obstacle_margin(prob, x):
    """|p - obs|^2 - obs_r^2 of the quadrotor state x (inf for the cart-pole)."""
    P = make_problem(prob)
    x = _f64(x)
    return _load().orc_obstacle_margin(ctypes.byref(P), _ptr(x, _d))


def terminal_cost(prob, x):
    P = make_problem(prob)
    x = _f64(x)
    return _load().orc_terminal_cost(ctypes.byref(P), _ptr(x, _d))


# --------------------------------------------------------------------------
# Rollouts, weights, update, iteration, MPC step
# --------------------------------------------------------------------------

def rollouts(prob, x0, U, it, k_begin=0, k_count=None, *, counts=False, delta=False,
             jumps=False, ambig=False, traj=False, margin=False, nthreads=0):
    """Rollouts k_begin..k_begin+k_count-1 of iteration `it`.

    Returns a dict with "S" (k_count,) and, when requested, "counts"
    (T, k_count) uint8, "delta" (T, k_count, m), "J" (T, k_count, q),
    "ambig" (T, k_count, m) bool, "traj" (k_count, T+1, n), "margin" (k_count,).
    """
    P = make_problem(prob)
    T, m, q, n = prob["T"], control_dim(prob), prob["q"], state_dim(prob)
    kc = prob["K"] - k_begin if k_count is None else int(k_count)
    x0 = _f64(x0)
    U = _f64(U).reshape(T, m)
    out = {"S": np.zeros(kc)}
    if counts:
        out["counts"] = np.zeros((T, kc), dtype=np.uint8)
    if delta:
        out["delta"] = np.zeros((T, kc, m))
    if jumps:
        out["J"] = np.zeros((T, kc, max(q, 1)))
    if ambig:
        out["ambig"] = np.zeros((T, kc, m), dtype=np.uint8)
    if traj:
        out["traj"] = np.zeros((kc, T + 1, n))
    if margin:
        out["margin"] = np.zeros(kc)
    st = _load().orc_rollouts(
        ctypes.byref(P), _ptr(x0, _d), _ptr(U, _d), int(it) & 0xFFFFFFFF, int(k_begin), kc,
        _ptr(out["S"], _d), _ptr(out.get("counts"), _u8), _ptr(out.get("delta"), _d),
        _ptr(out.get("J"), _d), _ptr(out.get("ambig"), _u8), _ptr(out.get("traj"), _d),
        _ptr(out.get("margin"), _d), int(nthreads))
    if st:
        raise OracleError(st, "rollouts")
    if ambig:
        out["ambig"] = out["ambig"].astype(bool)
    return out


def softmin(S, lam):
    """(w, (rho, Z, F)) -- free-energy weights of Eq. 36-37."""
    S = _f64(S)
    w = np.zeros_like(S)
    diag = np.zeros(3)
    st = _load().orc_softmin(S.shape[0], _ptr(S, _d), float(lam), _ptr(w, _d), _ptr(diag, _d))
    if st:
        raise OracleError(st, "softmin")
    return w, diag


def update(w, delta, U, alpha=1.0):
    """U + alpha * sum_k w_k delta[:, k, :]  (delta laid out [T][K][m])."""
    w = _f64(w)
    delta = _f64(delta)
    T, K, m = delta.shape
    Uo = _f64(U).reshape(T, m).copy()
    _load().orc_update(K, T, m, _ptr(w, _d), _ptr(delta, _d), float(alpha), _ptr(Uo, _d))
    return Uo


def iteration(prob, x0, U, it, *, want_delta=False, want_counts=False, want_ambig=False,
              nthreads=0):
    """One iteration from (x0, U) at counter `it`: dict with U (updated), S, w,
    diag = (rho, Z, F) and, when requested, counts / delta / ambig."""
    P = make_problem(prob)
    T, K, m = prob["T"], prob["K"], control_dim(prob)
    x0 = _f64(x0)
    Uo = _f64(U).reshape(T, m).copy()
    out = {"S": np.zeros(K), "w": np.zeros(K), "diag": np.zeros(3)}
    if want_counts:
        out["counts"] = np.zeros((T, K), dtype=np.uint8)
    if want_delta:
        out["delta"] = np.zeros((T, K, m))
    if want_ambig:
        out["ambig"] = np.zeros((T, K, m), dtype=np.uint8)
    st = _load().orc_iteration(
        ctypes.byref(P), _ptr(x0, _d), _ptr(Uo, _d), int(it) & 0xFFFFFFFF, _ptr(out["S"], _d),
        _ptr(out["w"], _d), _ptr(out.get("counts"), _u8), _ptr(out.get("delta"), _d),
        _ptr(out["diag"], _d), _ptr(out.get("ambig"), _u8), int(nthreads))
    if st:
        raise OracleError(st, "iteration")
    out["U"] = Uo
    if want_ambig:
        out["ambig"] = out["ambig"].astype(bool)
    return out


def step(prob, x0, U, it0, iters=None, nthreads=0):
    """One MPC step (Algorithm 1): returns (u0, U_shifted)."""
    P = make_problem(prob)
    T, m = prob["T"], control_dim(prob)
    iters = prob["iters"] if iters is None else int(iters)
    x0 = _f64(x0)
    Uo = _f64(U).reshape(T, m).copy()
    u0 = np.zeros(m)
    st = _load().orc_step(ctypes.byref(P), _ptr(x0, _d), _ptr(Uo, _d), int(it0) & 0xFFFFFFFF,
                          iters, _ptr(u0, _d), int(nthreads))
    if st:
        raise OracleError(st, "step")
    return u0, Uo
