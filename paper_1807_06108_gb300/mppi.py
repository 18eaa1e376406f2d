"""ctypes binding of libmppi_jump.so (argument marshalling only).

Every function named ``mppi_jump_*`` here is the C entry point of the same
name from ``include/mppi_jump.h``: device buffers are passed as integer
device pointers (``tensor.data_ptr()``), streams as ``cudaStream_t`` integers
(``torch.cuda.Stream().cuda_stream``).  Nonzero status codes raise
:class:`MppiError`.  All compute runs in the library's CUDA kernels; there is
no CPU or PyTorch fallback: importing this module raises if the library has
not been built.

:class:`Solver` is a small convenience wrapper that owns a context and the
PyTorch tensors used to exchange data with it.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build
from . import workloads as _wl

# MPPI_JUMP_LIB selects another build of the library, e.g. the checked debug
# variant (_build.LIB_CHECKED).
LIB_PATH = os.environ.get("MPPI_JUMP_LIB") or _build.LIB

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build the CUDA library first "
        "(python -c 'import __graft_entry__ as g; g.build()')")

_lib = ctypes.CDLL(LIB_PATH)

MAX_JUMPS = 16
STATUS = {0: "MPPI_OK", 1: "MPPI_EINVAL", 2: "MPPI_ENOMEM", 3: "MPPI_ECUDA",
          4: "MPPI_ETIMEOUT", 5: "MPPI_ENONFINITE", 6: "MPPI_EBUSY", 7: "MPPI_EBOUNDS"}
OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ENONFINITE, EBUSY, EBOUNDS = range(8)


class MppiError(RuntimeError):
    def __init__(self, code, what, detail=""):
        msg = f"{what}: {STATUS.get(code, code)}"
        if detail:
            msg += f" ({detail})"
        super().__init__(msg)
        self.code = code


class CartpoleParams(ctypes.Structure):
    _fields_ = [("mc", ctypes.c_float), ("mp", ctypes.c_float), ("l", ctypes.c_float),
                ("g", ctypes.c_float), ("goal", ctypes.c_float * 4), ("Q", ctypes.c_float * 4),
                ("Qf", ctypes.c_float * 4)]


class QuadrotorParams(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_float), ("J", ctypes.c_float * 3), ("arm", ctypes.c_float),
                ("kappa", ctypes.c_float), ("g", ctypes.c_float), ("goal", ctypes.c_float * 3),
                ("wp", ctypes.c_float), ("wv", ctypes.c_float), ("weta", ctypes.c_float),
                ("wom", ctypes.c_float), ("obs", ctypes.c_float * 3), ("obs_r", ctypes.c_float),
                ("obs_cost", ctypes.c_float)]


class Config(ctypes.Structure):
    """mppi_jump_config."""
    _fields_ = [
        ("system", ctypes.c_int32), ("K", ctypes.c_int32), ("T", ctypes.c_int32),
        ("dt", ctypes.c_float), ("lam", ctypes.c_float), ("c", ctypes.c_float),
        ("alpha", ctypes.c_float), ("sigma", ctypes.c_float * 4),
        ("jump_rate", ctypes.c_float), ("count_law", ctypes.c_int32),
        ("mark_law", ctypes.c_int32), ("mark_scale", ctypes.c_float * 4),
        ("jump_channel", ctypes.c_int32), ("q", ctypes.c_int32),
        ("jump_rows", ctypes.c_int32 * 4), ("jump_sqrt_dt", ctypes.c_int32),
        ("noise_dtype", ctypes.c_int32), ("u_init", ctypes.c_float * 4),
        ("seed", ctypes.c_uint64), ("cartpole", CartpoleParams),
        ("quadrotor", QuadrotorParams), ("alpha_decay", ctypes.c_float),
    ]


class Tuning(ctypes.Structure):
    """mppi_jump_tuning: rollout variant (1 fused, 2 split, 3 staged, 4 staged
    with block records), threads per block and steps per chunk or stage."""
    _fields_ = [("rollout_variant", ctypes.c_int32), ("rollout_block", ctypes.c_int32),
                ("rollout_chunk", ctypes.c_int32)]


_P = ctypes.POINTER
_vp = ctypes.c_void_p
_st = ctypes.c_int


def _sig(name, restype, *argtypes):
    f = getattr(_lib, name)
    f.restype = restype
    f.argtypes = list(argtypes)
    return f


_CTX = _vp
_sig("mppi_jump_config_bytes", ctypes.c_size_t)
if _lib.mppi_jump_config_bytes() != ctypes.sizeof(Config):
    raise ImportError("mppi_jump_config layout mismatch between the library and this binding")
_sig("mppi_jump_default_config", _st, ctypes.c_int32, _P(Config))
_sig("mppi_jump_validate", _st, _P(Config))
_sig("mppi_jump_count_table", _st, ctypes.c_float, ctypes.c_float, ctypes.c_int32,
     _P(ctypes.c_uint32), _P(ctypes.c_int32))
_sig("mppi_jump_workspace_bytes", _st, _P(Config), _P(ctypes.c_size_t))
_sig("mppi_jump_init", _st, _P(Config), _vp, _P(_vp))
_sig("mppi_jump_destroy", _st, _CTX)
_sig("mppi_jump_last_error", ctypes.c_char_p, _CTX)
_sig("mppi_jump_status_string", ctypes.c_char_p, ctypes.c_int)
_sig("mppi_jump_set_controls", _st, _CTX, _vp)
_sig("mppi_jump_get_controls", _st, _CTX, _vp)
_sig("mppi_jump_set_iteration", _st, _CTX, ctypes.c_uint32)
_sig("mppi_jump_get_iteration", _st, _CTX, _P(ctypes.c_uint32))
_sig("mppi_jump_rollout_cost", _st, _CTX, _vp, _vp)
_sig("mppi_jump_update", _st, _CTX)
_sig("mppi_jump_step", _st, _CTX, _P(ctypes.c_float), ctypes.c_int32, _P(ctypes.c_float))
_sig("mppi_jump_step_async", _st, _CTX, _vp, ctypes.c_int32, _vp)
_sig("mppi_jump_sync", _st, _CTX)
_sig("mppi_jump_set_tuning", _st, _CTX, _P(Tuning))
_sig("mppi_jump_get_tuning", _st, _CTX, _P(Tuning))
_sig("mppi_jump_autotune", _st, _CTX, _vp, ctypes.c_int32, ctypes.c_int32, _P(Tuning),
     _P(ctypes.c_float))
_sig("mppi_jump_enable_timing", _st, _CTX, ctypes.c_int32)
_sig("mppi_jump_phase_times", _st, _CTX, _P(ctypes.c_float), _P(ctypes.c_int32))
_sig("mppi_jump_set_debug", _st, _CTX, _vp, _vp)
_sig("mppi_jump_get_noise", _st, _CTX, _vp)
_sig("mppi_jump_get_weights", _st, _CTX, _vp)
_sig("mppi_jump_get_free_energy", _st, _CTX, _P(ctypes.c_float))
_sig("mppi_jump_get_state", _st, _CTX, _vp, _P(ctypes.c_size_t))
_sig("mppi_jump_set_rollout_offset", _st, _CTX, ctypes.c_uint32)
_sig("mppi_jump_rollout_partial", _st, _CTX, _vp, _vp)
_sig("mppi_jump_apply_partials", _st, _CTX, _vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _vp)
_sig("mppi_jump_set_state", _st, _CTX, _vp, ctypes.c_size_t)


def _check(st, what, ctx=None):
    if st != OK:
        detail = ""
        if ctx:
            detail = (_lib.mppi_jump_last_error(ctx) or b"").decode(errors="replace")
        raise MppiError(st, what, detail)


# --------------------------------------------------------------------------
# Thin wrappers with the C names
# --------------------------------------------------------------------------

def mppi_jump_default_config(system):
    cfg = Config()
    _check(_lib.mppi_jump_default_config(int(system), ctypes.byref(cfg)), "default_config")
    return cfg


def mppi_jump_validate(cfg):
    return _lib.mppi_jump_validate(ctypes.byref(cfg))


def mppi_jump_count_table(jump_rate, dt, count_law=0):
    thr = (ctypes.c_uint32 * MAX_JUMPS)()
    nmax = ctypes.c_int32(0)
    _check(_lib.mppi_jump_count_table(float(jump_rate), float(dt), int(count_law), thr,
                                      ctypes.byref(nmax)), "count_table")
    return np.array(list(thr), dtype=np.uint32), nmax.value


def mppi_jump_workspace_bytes(cfg):
    n = ctypes.c_size_t(0)
    _check(_lib.mppi_jump_workspace_bytes(ctypes.byref(cfg), ctypes.byref(n)), "workspace_bytes")
    return n.value


def mppi_jump_init(cfg, stream=0):
    ctx = _vp()
    st = _lib.mppi_jump_init(ctypes.byref(cfg), _vp(stream or None), ctypes.byref(ctx))
    _check(st, "init")
    return ctx


def mppi_jump_destroy(ctx):
    _check(_lib.mppi_jump_destroy(ctx), "destroy")


def mppi_jump_last_error(ctx):
    return (_lib.mppi_jump_last_error(ctx) or b"").decode(errors="replace")


def mppi_jump_set_controls(ctx, U_ptr):
    _check(_lib.mppi_jump_set_controls(ctx, _vp(U_ptr)), "set_controls", ctx)


def mppi_jump_get_controls(ctx, U_ptr):
    _check(_lib.mppi_jump_get_controls(ctx, _vp(U_ptr)), "get_controls", ctx)


def mppi_jump_set_iteration(ctx, it):
    _check(_lib.mppi_jump_set_iteration(ctx, int(it) & 0xFFFFFFFF), "set_iteration", ctx)


def mppi_jump_get_iteration(ctx):
    v = ctypes.c_uint32(0)
    _check(_lib.mppi_jump_get_iteration(ctx, ctypes.byref(v)), "get_iteration", ctx)
    return v.value


def mppi_jump_rollout_cost(ctx, x0_ptr, costs_ptr=0):
    _check(_lib.mppi_jump_rollout_cost(ctx, _vp(x0_ptr), _vp(costs_ptr or None)),
           "rollout_cost", ctx)


def mppi_jump_update(ctx):
    _check(_lib.mppi_jump_update(ctx), "update", ctx)


def mppi_jump_set_rollout_offset(ctx, k_offset):
    _check(_lib.mppi_jump_set_rollout_offset(ctx, int(k_offset)), "set_rollout_offset", ctx)


def mppi_jump_rollout_partial(ctx, x0_ptr, partial_ptr):
    _check(_lib.mppi_jump_rollout_partial(ctx, _vp(x0_ptr), _vp(partial_ptr)), "rollout_partial", ctx)


def mppi_jump_apply_partials(ctx, partials_ptr, n_parts, r=0, shift=0, u0_ptr=0):
    _check(_lib.mppi_jump_apply_partials(ctx, _vp(partials_ptr), int(n_parts), int(r), int(shift),
                                         _vp(u0_ptr or None)), "apply_partials", ctx)


def mppi_jump_step(ctx, x0_host, iters, u0_host):
    """x0_host / u0_host: contiguous float32 numpy arrays (host memory)."""
    st = _lib.mppi_jump_step(ctx, x0_host.ctypes.data_as(_P(ctypes.c_float)), int(iters),
                             u0_host.ctypes.data_as(_P(ctypes.c_float)))
    _check(st, "step", ctx)


def mppi_jump_step_async(ctx, x0_ptr, iters, u0_ptr=0):
    _check(_lib.mppi_jump_step_async(ctx, _vp(x0_ptr), int(iters), _vp(u0_ptr or None)),
           "step_async", ctx)


def mppi_jump_sync(ctx):
    _check(_lib.mppi_jump_sync(ctx), "sync", ctx)


def mppi_jump_set_tuning(ctx, variant, block, chunk=4):
    t = Tuning(int(variant), int(block), int(chunk))
    _check(_lib.mppi_jump_set_tuning(ctx, ctypes.byref(t)), "set_tuning", ctx)


def mppi_jump_get_tuning(ctx):
    t = Tuning()
    _check(_lib.mppi_jump_get_tuning(ctx, ctypes.byref(t)), "get_tuning", ctx)
    return t.rollout_variant, t.rollout_block, t.rollout_chunk


def mppi_jump_autotune(ctx, x0_ptr, iters, reps=5):
    """Returns ((variant, block, chunk), mean step ms) of the fastest tile."""
    t = Tuning()
    ms = ctypes.c_float(0.0)
    _check(_lib.mppi_jump_autotune(ctx, _vp(x0_ptr), int(iters), int(reps), ctypes.byref(t),
                                   ctypes.byref(ms)), "autotune", ctx)
    return (t.rollout_variant, t.rollout_block, t.rollout_chunk), ms.value


def mppi_jump_enable_timing(ctx, on=True):
    _check(_lib.mppi_jump_enable_timing(ctx, int(bool(on))), "enable_timing", ctx)


def mppi_jump_phase_times(ctx):
    """(rollout_ms, update_ms, iterations) summed over the last MPC step."""
    out = (ctypes.c_float * 2)()
    it = ctypes.c_int32(0)
    _check(_lib.mppi_jump_phase_times(ctx, out, ctypes.byref(it)), "phase_times", ctx)
    return float(out[0]), float(out[1]), it.value


def mppi_jump_set_debug(ctx, counts_ptr=0, jumps_ptr=0):
    _check(_lib.mppi_jump_set_debug(ctx, _vp(counts_ptr or None), _vp(jumps_ptr or None)),
           "set_debug", ctx)


def mppi_jump_get_noise(ctx, noise_ptr):
    _check(_lib.mppi_jump_get_noise(ctx, _vp(noise_ptr)), "get_noise", ctx)


def mppi_jump_get_weights(ctx, w_ptr):
    _check(_lib.mppi_jump_get_weights(ctx, _vp(w_ptr)), "get_weights", ctx)


def mppi_jump_get_free_energy(ctx):
    out = (ctypes.c_float * 3)()
    _check(_lib.mppi_jump_get_free_energy(ctx, out), "get_free_energy", ctx)
    return np.array(list(out), dtype=np.float32)


def mppi_jump_get_state(ctx):
    n = ctypes.c_size_t(0)
    _check(_lib.mppi_jump_get_state(ctx, None, ctypes.byref(n)), "get_state", ctx)
    buf = ctypes.create_string_buffer(n.value)
    _check(_lib.mppi_jump_get_state(ctx, buf, ctypes.byref(n)), "get_state", ctx)
    return bytes(buf.raw[:n.value])


def mppi_jump_set_state(ctx, blob):
    buf = ctypes.create_string_buffer(blob, len(blob))
    _check(_lib.mppi_jump_set_state(ctx, buf, len(blob)), "set_state", ctx)


# --------------------------------------------------------------------------
# Problem dictionaries -> configuration
# --------------------------------------------------------------------------

def config_from_problem(prob):
    """mppi_jump_config from a workloads.problem() dictionary."""
    cfg = Config()
    cfg.system = 0 if prob["system"] == "cartpole" else 1
    cfg.K, cfg.T = prob["K"], prob["T"]
    cfg.dt, cfg.lam, cfg.c, cfg.alpha = prob["dt"], prob["lam"], prob["c"], prob["alpha"]
    cfg.alpha_decay = prob.get("alpha_decay", 1.0)
    for i, s in enumerate(prob["sigma"]):
        cfg.sigma[i] = s
    cfg.jump_rate = prob["nu"]
    cfg.count_law = {"poisson": 0, "bernoulli": 1}[prob["count_law"]]
    cfg.mark_law = {"normal": 0, "laplace": 1}[prob["mark_law"]]
    for i, s in enumerate(prob["mark_scale"]):
        cfg.mark_scale[i] = s
    cfg.jump_channel = {"state": 0, "control": 1}[prob["jump_channel"]]
    cfg.q = prob["q"]
    for i, r in enumerate(prob["jump_rows"]):
        cfg.jump_rows[i] = r
    cfg.jump_sqrt_dt = int(prob["jump_sqrt_dt"])
    cfg.noise_dtype = {"f32": 0, "bf16": 1}[prob["noise_dtype"]]
    for i, u in enumerate(prob["u_init"]):
        cfg.u_init[i] = u
    cfg.seed = prob["seed"]
    p = prob["params"]
    if prob["system"] == "cartpole":
        c = cfg.cartpole
        c.mc, c.mp, c.l, c.g = p["mc"], p["mp"], p["l"], p["g"]
        for i in range(4):
            c.goal[i], c.Q[i], c.Qf[i] = p["goal"][i], p["Q"][i], p["Qf"][i]
    else:
        q = cfg.quadrotor
        q.mass, q.arm, q.kappa, q.g = p["mass"], p["arm"], p["kappa"], p["g"]
        for i in range(3):
            q.J[i], q.goal[i], q.obs[i] = p["J"][i], p["goal"][i], p["obs"][i]
        q.wp, q.wv, q.weta, q.wom = p["wp"], p["wv"], p["weta"], p["wom"]
        q.obs_r, q.obs_cost = p["obs_r"], p["obs_cost"]
    return cfg


class Solver:
    """One MPPI context plus the torch tensors used to talk to it.

    All device work runs on ``self.stream`` (a torch.cuda.Stream).
    """

    def __init__(self, prob, stream=None, device="cuda"):
        import torch
        self.torch = torch
        self.prob = prob
        self.n = _wl.STATE_DIM[prob["system"]]
        self.m = _wl.CONTROL_DIM[prob["system"]]
        self.K, self.T, self.q = prob["K"], prob["T"], prob["q"]
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device)
        self.cfg = config_from_problem(prob)
        self.ctx = mppi_jump_init(self.cfg, self.stream.cuda_stream)
        with torch.cuda.stream(self.stream):
            self.x0 = torch.zeros(self.n, dtype=torch.float32, device=self.device)
            self.u0 = torch.zeros(self.m, dtype=torch.float32, device=self.device)

    def close(self):
        if self.ctx:
            mppi_jump_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- data exchange -----------------------------------------------------
    # Every tensor operation runs on the solver's stream, so that it is
    # ordered with the library's work on that stream.
    def _sync(self):
        self.stream.synchronize()

    def _on(self):
        return self.torch.cuda.stream(self.stream)

    def set_x0(self, x0):
        with self._on():
            self.x0.copy_(self.torch.as_tensor(np.asarray(x0, dtype=np.float32)), non_blocking=False)

    def set_controls(self, U):
        with self._on():
            t = self.torch.as_tensor(np.ascontiguousarray(U, dtype=np.float32)).to(self.device)
            mppi_jump_set_controls(self.ctx, t.data_ptr())
        self._sync()

    def controls(self):
        with self._on():
            t = self.torch.empty((self.T, self.m), dtype=self.torch.float32, device=self.device)
            mppi_jump_get_controls(self.ctx, t.data_ptr())
        self._sync()
        return t.cpu().numpy()

    def set_iteration(self, it):
        mppi_jump_set_iteration(self.ctx, it)

    def iteration(self):
        return mppi_jump_get_iteration(self.ctx)

    # -- the method ----------------------------------------------------------
    def rollout_cost(self, x0, want_costs=True):
        self.set_x0(x0)
        costs = None
        with self._on():
            if want_costs:
                costs = self.torch.empty(self.K, dtype=self.torch.float32, device=self.device)
            mppi_jump_rollout_cost(self.ctx, self.x0.data_ptr(),
                                   costs.data_ptr() if want_costs else 0)
        return costs

    def update(self):
        mppi_jump_update(self.ctx)

    def sync(self):
        mppi_jump_sync(self.ctx)

    def step(self, x0, iters=None):
        x = np.ascontiguousarray(x0, dtype=np.float32)
        u0 = np.zeros(self.m, dtype=np.float32)
        mppi_jump_step(self.ctx, x, self.prob["iters"] if iters is None else iters, u0)
        return u0

    # -- debug copies -----------------------------------------------------
    def enable_debug(self):
        with self._on():
            self.dbg_counts = self.torch.zeros((self.T, self.K), dtype=self.torch.uint8,
                                               device=self.device)
            self.dbg_J = self.torch.zeros((self.T, self.K, max(self.q, 1)),
                                          dtype=self.torch.float32, device=self.device)
        mppi_jump_set_debug(self.ctx, self.dbg_counts.data_ptr(), self.dbg_J.data_ptr())

    def noise(self):
        """delta_eff [T][K][m] as float32 numpy (bfloat16 values widened)."""
        torch = self.torch
        dt = torch.bfloat16 if self.prob["noise_dtype"] == "bf16" else torch.float32
        with self._on():
            t = torch.empty((self.T, self.K, self.m), dtype=dt, device=self.device)
            mppi_jump_get_noise(self.ctx, t.data_ptr())
        self._sync()
        return t.float().cpu().numpy()

    def noise_bits(self):
        """Raw bfloat16 bit patterns of delta_eff (uint16 numpy), bf16 problems only."""
        torch = self.torch
        with self._on():
            t = torch.empty((self.T, self.K, self.m), dtype=torch.int16, device=self.device)
            mppi_jump_get_noise(self.ctx, t.data_ptr())
        self._sync()
        return t.cpu().numpy().view(np.uint16)

    def weights(self):
        with self._on():
            t = self.torch.empty(self.K, dtype=self.torch.float32, device=self.device)
            mppi_jump_get_weights(self.ctx, t.data_ptr())
        self._sync()
        return t.cpu().numpy()

    def free_energy(self):
        return mppi_jump_get_free_energy(self.ctx)

    # -- rollout shards ---------------------------------------------------
    def set_rollout_offset(self, k0):
        mppi_jump_set_rollout_offset(self.ctx, k0)

    def rollout_partial(self, x0):
        """This shard's partial record (rho, Z, N[T][m]) as a device tensor."""
        self.set_x0(x0)
        with self._on():
            out = self.torch.empty(2 + self.T * self.m, dtype=self.torch.float32, device=self.device)
            mppi_jump_rollout_partial(self.ctx, self.x0.data_ptr(), out.data_ptr())
        return out

    def apply_partials(self, parts, r=0, shift=False):
        """Combine partial records [G][2 + T*m] (device tensor) into U."""
        with self._on():
            p = parts.to(self.device, dtype=self.torch.float32).contiguous()
            mppi_jump_apply_partials(self.ctx, p.data_ptr(), p.shape[0], r, int(bool(shift)),
                                     self.u0.data_ptr() if shift else 0)
        self._sync()

    def get_state(self):
        return mppi_jump_get_state(self.ctx)

    def set_state(self, blob):
        mppi_jump_set_state(self.ctx, blob)


# --------------------------------------------------------------------------
# Batched form
# --------------------------------------------------------------------------

_sig("mppi_batch_create", _st, _P(Config), _P(ctypes.c_int32), ctypes.c_int32, _vp, _P(_vp))
_sig("mppi_batch_destroy", _st, _vp)
_sig("mppi_batch_last_error", ctypes.c_char_p, _vp)
_sig("mppi_batch_step_async", _st, _vp, _vp, _vp)
_sig("mppi_batch_step", _st, _vp, _P(ctypes.c_float), _P(ctypes.c_float))
_sig("mppi_batch_sync", _st, _vp)
_sig("mppi_batch_get_controls", _st, _vp, ctypes.c_int32, _vp)
_sig("mppi_batch_set_controls", _st, _vp, ctypes.c_int32, _vp)
_sig("mppi_batch_get_iteration", _st, _vp, ctypes.c_int32, _P(ctypes.c_uint32))
_sig("mppi_batch_set_tuning", _st, _vp, ctypes.c_int32)
_sig("mppi_batch_get_tuning", _st, _vp, _P(ctypes.c_int32))
_sig("mppi_batch_set_tile", _st, _vp, ctypes.c_int32, ctypes.c_int32)
_sig("mppi_batch_get_tile", _st, _vp, _P(ctypes.c_int32), _P(ctypes.c_int32))
_sig("mppi_batch_autotune", _st, _vp, _vp, ctypes.c_int32, _P(ctypes.c_int32), _P(ctypes.c_float))
_sig("mppi_batch_info", _st, _vp, _P(ctypes.c_int64), _P(ctypes.c_int32), _P(ctypes.c_int32))
_sig("mppi_batch_inject_stall", _st, _vp, ctypes.c_int32)

STATE_STRIDE = 12
CONTROL_STRIDE = 4


def _bcheck(st, what, b=None):
    if st != OK:
        detail = (_lib.mppi_batch_last_error(b) or b"").decode(errors="replace") if b else ""
        raise MppiError(st, what, detail)


class Batch:
    """n independent MPC problems advanced by one persistent launch per step."""

    def __init__(self, probs, stream=None):
        import torch
        self.torch = torch
        self.probs = list(probs)
        self.n = len(self.probs)
        cfgs = (Config * self.n)(*[config_from_problem(p) for p in self.probs])
        iters = (ctypes.c_int32 * self.n)(*[p["iters"] for p in self.probs])
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.handle = _vp()
        _bcheck(_lib.mppi_batch_create(cfgs, iters, self.n, _vp(self.stream.cuda_stream),
                                       ctypes.byref(self.handle)), "batch_create")
        with torch.cuda.stream(self.stream):
            self.x0s = torch.zeros((self.n, STATE_STRIDE), dtype=torch.float32, device="cuda")
            self.u0s = torch.zeros((self.n, CONTROL_STRIDE), dtype=torch.float32, device="cuda")
        self.stream.synchronize()

    def close(self):
        if self.handle:
            _lib.mppi_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        s, n, g = ctypes.c_int64(0), ctypes.c_int32(0), ctypes.c_int32(0)
        _bcheck(_lib.mppi_batch_info(self.handle, ctypes.byref(s), ctypes.byref(n), ctypes.byref(g)),
                "batch_info", self.handle)
        return {"steps_per_solve": s.value, "items": n.value, "grid": g.value}

    def pack_states(self, states):
        x = np.zeros((self.n, STATE_STRIDE), dtype=np.float32)
        for i, s in enumerate(states):
            s = np.asarray(s, dtype=np.float32)
            x[i, :s.shape[0]] = s
        return x

    def set_states(self, states):
        x = self.torch.from_numpy(self.pack_states(states))
        with self.torch.cuda.stream(self.stream):
            self.x0s.copy_(x)
        self.stream.synchronize()

    def step(self, states):
        """Synchronous batched step from host states; returns u0 per instance."""
        x = np.ascontiguousarray(self.pack_states(states))
        u = np.zeros((self.n, CONTROL_STRIDE), dtype=np.float32)
        _bcheck(_lib.mppi_batch_step(self.handle, x.ctypes.data_as(_P(ctypes.c_float)),
                                     u.ctypes.data_as(_P(ctypes.c_float))), "batch_step", self.handle)
        return [u[i, :_wl.CONTROL_DIM[p["system"]]] for i, p in enumerate(self.probs)]

    def step_async(self):
        _bcheck(_lib.mppi_batch_step_async(self.handle, _vp(self.x0s.data_ptr()),
                                           _vp(self.u0s.data_ptr())), "batch_step_async", self.handle)

    def sync(self):
        _bcheck(_lib.mppi_batch_sync(self.handle), "batch_sync", self.handle)

    def controls(self, i):
        p = self.probs[i]
        U = np.zeros((p["T"], _wl.CONTROL_DIM[p["system"]]), dtype=np.float32)
        _bcheck(_lib.mppi_batch_get_controls(self.handle, i, _vp(U.ctypes.data)), "batch_get_controls",
                self.handle)
        return U

    def set_controls(self, i, U):
        U = np.ascontiguousarray(U, dtype=np.float32)
        _bcheck(_lib.mppi_batch_set_controls(self.handle, i, _vp(U.ctypes.data)), "batch_set_controls",
                self.handle)

    def iteration(self, i):
        v = ctypes.c_uint32(0)
        _bcheck(_lib.mppi_batch_get_iteration(self.handle, i, ctypes.byref(v)), "batch_get_iteration",
                self.handle)
        return v.value

    def set_tuning(self, block):
        _bcheck(_lib.mppi_batch_set_tuning(self.handle, int(block)), "batch_set_tuning", self.handle)

    def tuning(self):
        v = ctypes.c_int32(0)
        _bcheck(_lib.mppi_batch_get_tuning(self.handle, ctypes.byref(v)), "batch_get_tuning", self.handle)
        return v.value

    def set_tile(self, block, chunk):
        _bcheck(_lib.mppi_batch_set_tile(self.handle, int(block), int(chunk)), "batch_set_tile", self.handle)

    def tile(self):
        b, c = ctypes.c_int32(0), ctypes.c_int32(0)
        _bcheck(_lib.mppi_batch_get_tile(self.handle, ctypes.byref(b), ctypes.byref(c)), "batch_get_tile",
                self.handle)
        return b.value, c.value

    def autotune(self, reps=3):
        """Returns ((block, chunk), mean batched-step ms) of the fastest tile."""
        blk, ms = ctypes.c_int32(0), ctypes.c_float(0.0)
        _bcheck(_lib.mppi_batch_autotune(self.handle, _vp(self.x0s.data_ptr()), int(reps),
                                         ctypes.byref(blk), ctypes.byref(ms)), "batch_autotune", self.handle)
        return self.tile(), ms.value

    def inject_stall(self, on=True):
        _bcheck(_lib.mppi_batch_inject_stall(self.handle, int(bool(on))), "batch_inject_stall",
                self.handle)


# --------------------------------------------------------------------------
# Allocation-free update (for callers that cannot allocate device memory)
# --------------------------------------------------------------------------

_sig("mppi_jump_update_noalloc", _st, _vp, _vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
     ctypes.c_float, ctypes.c_float, _vp, _vp)


def mppi_jump_update_noalloc(costs_ptr, noise_ptr, K, T, m, lam, alpha, U_ptr, stream=0):
    """Weights + weighted update from caller-owned device arrays, using the
    library's fixed device scratch instead of allocating (see the header)."""
    _check(_lib.mppi_jump_update_noalloc(_vp(costs_ptr), _vp(noise_ptr), int(K), int(T), int(m),
                                         float(lam), float(alpha), _vp(U_ptr), _vp(stream or None)),
           "update_noalloc")


# --------------------------------------------------------------------------
# Served form
# --------------------------------------------------------------------------

class ServeStats(ctypes.Structure):
    """mppi_serve_stats."""
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("inflight", ctypes.c_int64), ("evictions", ctypes.c_int64),
                ("mean_ms", ctypes.c_double), ("max_ms", ctypes.c_double),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("span_s", ctypes.c_double), ("resident_bytes", ctypes.c_size_t)]


_sig("mppi_serve_create", _st, _P(Config), _P(ctypes.c_int32), ctypes.c_int32, ctypes.c_size_t,
     ctypes.c_int32, _P(_vp))
_sig("mppi_serve_destroy", _st, _vp)
_sig("mppi_serve_last_error", ctypes.c_char_p, _vp)
_sig("mppi_serve_submit", _st, _vp, ctypes.c_int32, _P(ctypes.c_float), _P(ctypes.c_uint64))
_sig("mppi_serve_poll", _st, _vp, ctypes.c_uint64, _P(ctypes.c_float), _P(ctypes.c_int32))
_sig("mppi_serve_wait", _st, _vp, ctypes.c_uint64, _P(ctypes.c_float), ctypes.c_double)
_sig("mppi_serve_drain", _st, _vp, ctypes.c_double)
_sig("mppi_serve_get_stats", _st, _vp, _P(ServeStats))
_sig("mppi_serve_reset_stats", _st, _vp)
_sig("mppi_serve_get_controls", _st, _vp, ctypes.c_int32, _P(ctypes.c_float))


class Server:
    """Sessions served by the library's request loop (see mppi_serve_create)."""

    def __init__(self, probs, budget_bytes=20 << 30, max_inflight=16):
        self.probs = list(probs)
        self.n = len(self.probs)
        cfgs = (Config * self.n)(*[config_from_problem(p) for p in self.probs])
        iters = (ctypes.c_int32 * self.n)(*[p["iters"] for p in self.probs])
        self.handle = _vp()
        st = _lib.mppi_serve_create(cfgs, iters, self.n, int(budget_bytes), int(max_inflight),
                                    ctypes.byref(self.handle))
        if st != OK:
            raise MppiError(st, "serve_create")

    def _check(self, st, what):
        if st != OK:
            raise MppiError(st, what, (_lib.mppi_serve_last_error(self.handle) or b"").decode())

    def close(self):
        if self.handle:
            _lib.mppi_serve_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, session, x0):
        x = np.zeros(12, dtype=np.float32)
        x0 = np.asarray(x0, dtype=np.float32)
        x[:x0.shape[0]] = x0
        t = ctypes.c_uint64(0)
        self._check(_lib.mppi_serve_submit(self.handle, int(session), x.ctypes.data_as(_P(ctypes.c_float)),
                                           ctypes.byref(t)), "serve_submit")
        return t.value

    def wait(self, ticket, timeout_s=30.0):
        u = np.zeros(4, dtype=np.float32)
        self._check(_lib.mppi_serve_wait(self.handle, int(ticket), u.ctypes.data_as(_P(ctypes.c_float)),
                                         float(timeout_s)), "serve_wait")
        return u

    def poll(self, ticket):
        u = np.zeros(4, dtype=np.float32)
        d = ctypes.c_int32(0)
        st = _lib.mppi_serve_poll(self.handle, int(ticket), u.ctypes.data_as(_P(ctypes.c_float)),
                                  ctypes.byref(d))
        if d.value:
            self._check(st, "serve_poll")
            return u
        return None

    def drain(self, timeout_s=120.0):
        self._check(_lib.mppi_serve_drain(self.handle, float(timeout_s)), "serve_drain")

    def stats(self):
        s = ServeStats()
        self._check(_lib.mppi_serve_get_stats(self.handle, ctypes.byref(s)), "serve_get_stats")
        return {f: getattr(s, f) for f, _ in ServeStats._fields_}

    def reset_stats(self):
        self._check(_lib.mppi_serve_reset_stats(self.handle), "serve_reset_stats")

    def controls(self, session):
        p = self.probs[session]
        U = np.zeros((p["T"], _wl.CONTROL_DIM[p["system"]]), dtype=np.float32)
        self._check(_lib.mppi_serve_get_controls(self.handle, int(session),
                                                 U.ctypes.data_as(_P(ctypes.c_float))), "serve_get_controls")
        return U
