"""Host-side checks of the C ABI (no GPU needed): the library builds and
loads, exports every entry point that include/*.h declares, its config
struct matches the binding, its jump-count table equals the oracle's bit for
bit, and configuration validation rejects bad input."""

import ctypes
import glob
import os
import re

import numpy as np
import pytest

import oracle
from paper_1807_06108_gb300 import build as B
from paper_1807_06108_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    from paper_1807_06108_gb300 import mppi
    return mppi


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(mppi_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_entry_points():
    names = _declared_functions()
    for must in ("mppi_jump_init", "mppi_jump_rollout_cost", "mppi_jump_update", "mppi_jump_step",
                 "mppi_jump_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    so = ctypes.CDLL(B.LIB)
    missing = [n for n in _declared_functions() if not hasattr(so, n)]
    assert not missing, missing


def test_config_layout_matches_binding(lib):
    assert lib._lib.mppi_jump_config_bytes() == ctypes.sizeof(lib.Config)


@pytest.mark.parametrize("law", ["poisson", "bernoulli"])
def test_count_table_equals_oracle(lib, law):
    rng = np.random.default_rng(0)
    cases = [(1.0, 0.02), (2.0, 0.01), (5.0, 0.005), (0.0, 0.01), (3.0, 0.02), (40.0, 0.02)]
    cases += [(float(np.float32(rng.uniform(0, 30))), float(np.float32(rng.uniform(1e-3, 0.03))))
              for _ in range(200)]
    for nu, dt in cases:
        nu, dt = W.f32(nu), W.f32(dt)
        try:
            ref = oracle.count_table(nu, dt, law)
        except oracle.OracleError:
            with pytest.raises(lib.MppiError):
                lib.mppi_jump_count_table(nu, dt, {"poisson": 0, "bernoulli": 1}[law])
            continue
        got = lib.mppi_jump_count_table(nu, dt, {"poisson": 0, "bernoulli": 1}[law])
        assert got[1] == ref[1]
        np.testing.assert_array_equal(got[0], ref[0])


def test_default_config_matches_workloads(lib):
    for system, prob in ((0, W.cartpole_k1000()), (1, W.quadrotor_k4096())):
        d = lib.mppi_jump_default_config(system)
        c = lib.config_from_problem(prob)
        inactive = "quadrotor" if system == 0 else "cartpole"
        for f, _ in lib.Config._fields_:
            if f == inactive:
                continue
            a, b = getattr(d, f), getattr(c, f)
            if isinstance(a, ctypes.Structure):
                for g, _ in a._fields_:
                    assert np.allclose(np.array(getattr(a, g)), np.array(getattr(b, g)), rtol=0,
                                       atol=0), (f, g)
            elif isinstance(a, ctypes.Array):
                assert list(a) == list(b), f
            else:
                assert a == b, f


def test_validation_rejects_bad_configs(lib):
    good = lib.config_from_problem(W.quadrotor_k4096())
    assert lib.mppi_jump_validate(good) == lib.OK
    bad_edits = [
        ("K", 0), ("T", 0), ("T", 5000), ("dt", 0.0), ("dt", float("nan")), ("lam", -1.0),
        ("c", 0.0), ("jump_rate", -1.0), ("jump_rate", 1e6), ("count_law", 7), ("mark_law", 3),
        ("jump_channel", 2), ("noise_dtype", 9), ("q", 5), ("system", 4),
        ("alpha_decay", 1.5), ("alpha_decay", -0.1), ("alpha_decay", float("nan")),
    ]
    for field, val in bad_edits:
        cfg = lib.config_from_problem(W.quadrotor_k4096())
        setattr(cfg, field, val)
        assert lib.mppi_jump_validate(cfg) == lib.EINVAL, field
    cfg = lib.config_from_problem(W.quadrotor_k4096())
    cfg.sigma[2] = 0.0
    assert lib.mppi_jump_validate(cfg) == lib.EINVAL
    cfg = lib.config_from_problem(W.quadrotor_k4096())
    cfg.jump_rows[1] = 12
    assert lib.mppi_jump_validate(cfg) == lib.EINVAL
    cfg = lib.config_from_problem(W.quadrotor_k4096(jump_channel="control"))
    cfg.q = 3
    assert lib.mppi_jump_validate(cfg) == lib.EINVAL


def test_workspace_bytes_scale_with_problem(lib):
    small = lib.mppi_jump_workspace_bytes(lib.config_from_problem(W.quadrotor_k4096()))
    big = lib.mppi_jump_workspace_bytes(lib.config_from_problem(W.large_quadrotor()))
    assert small >= 4096 * 100 * 4 * 4
    assert big >= 65536 * 200 * 4 * 2
    assert big > small


def test_checked_debug_build_exports_the_same_symbols(lib):
    """The MPPI_CHECK_BOUNDS variant (launch checks that report MPPI_EBOUNDS
    through the status word) builds and exports every declared entry point."""
    path = B.build(checked=True)
    assert path == B.LIB_CHECKED and os.path.exists(path)
    so = ctypes.CDLL(path)
    missing = [n for n in _declared_functions() if not hasattr(so, n)]
    assert not missing, missing
    so.mppi_jump_status_string.restype = ctypes.c_char_p
    assert so.mppi_jump_status_string(7) == b"kernel launch check failed"
