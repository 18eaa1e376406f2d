"""GPU parity: one MPPI iteration through the C ABI against the FP64 oracle,
element by element, for the named workloads at full size and for ragged,
tiny and mode-switching variants (see tests/parity.py for the tolerances)."""

import json
import os

import numpy as np
import pytest

from paper_1807_06108_gb300 import workloads as W
from tests import parity

pytestmark = pytest.mark.gpu

REPORT = os.environ.get("MPPI_PARITY_REPORT")


def _record(name, rep):
    print(name, rep)
    if REPORT:
        with open(REPORT, "a") as f:
            f.write(json.dumps({"case": name, **rep}) + "\n")


def _obstacle_state(prob):
    x = W.initial_state(prob).astype(np.float64)
    x[0:3] = [1.45, 0.05, 1.0]
    x[3] = 1.5
    return x.astype(np.float32)


def _cases():
    rng = lambda s: np.random.default_rng(s)  # noqa: E731
    c = {}
    p = W.cartpole_k1000()
    c["cartpole_K1000_T50"] = (p, W.initial_state(p), W.initial_controls(p), 0)
    p = W.cartpole_k1000(K=777, T=23)
    r = rng(1)
    c["cartpole_K777_T23_random"] = (p, W.random_state(p, r), W.random_controls(p, r), 5)
    p = W.cartpole_k1000(K=1500, T=31, nu=10.0, jump_channel="control", count_law="bernoulli",
                         noise_dtype="bf16", c=2.0, mark_scale=1.0)
    r = rng(2)
    c["cartpole_bf16_control_bernoulli_c2"] = (p, W.random_state(p, r), W.random_controls(p, r), 9)
    p = W.quadrotor_k4096()
    c["quadrotor_K4096_T100"] = (p, W.initial_state(p), W.initial_controls(p), 0)
    p = W.quadrotor_k4096(K=1000, T=37, lam=20.0)
    r = rng(3)
    c["quadrotor_K1000_T37_obstacle"] = (p, _obstacle_state(p), W.random_controls(p, r, 0.2), 3)
    p = W.quadrotor_k4096(K=2053, T=45, nu=8.0, mark_law="laplace", noise_dtype="bf16",
                          jump_sqrt_dt=True, lam=10.0)
    r = rng(4)
    c["quadrotor_laplace_bf16_sqrtdt"] = (p, W.random_state(p, r, 0.1), W.random_controls(p, r, 0.2), 1)
    p = W.quadrotor_k4096(K=640, T=16, nu=6.0, jump_channel="control", c=2.0, lam=50.0,
                          mark_scale=0.3, alpha=0.5)
    r = rng(5)
    c["quadrotor_control_c2_alpha05"] = (p, W.random_state(p, r, 0.1), W.random_controls(p, r, 0.2), 2)
    p = W.cartpole_k1000(K=1, T=1)
    c["cartpole_K1_T1"] = (p, W.initial_state(p), W.initial_controls(p), 0)
    p = W.quadrotor_k4096(K=33, T=5, nu=50.0)
    r = rng(6)
    c["quadrotor_K33_T5_many_jumps"] = (p, W.random_state(p, r, 0.1), W.random_controls(p, r, 0.2), 77)
    p = W.quadrotor_k4096(K=96, T=4096, dt=0.001, lam=100.0)
    c["quadrotor_K96_T4096_max_horizon"] = (p, W.initial_state(p), W.initial_controls(p), 0)
    p = W.quadrotor_k4096(K=515, T=27, nu=12.0, jump_rows=[3, 4, 5, 9], mark_scale=0.5)
    r = rng(7)
    c["quadrotor_q4_state_rows"] = (p, W.random_state(p, r, 0.1), W.random_controls(p, r, 0.2), 6)
    # state jumps on rows other than the velocities with q <= 3 (the counted,
    # per-step jump path), float32 and bfloat16 noise
    for dt_ in ("f32", "bf16"):
        p = W.cartpole_k1000(K=700, T=33, nu=10.0, jump_rows=[0, 2], noise_dtype=dt_)
        r = rng(20)
        c[f"cartpole_rows02_{dt_}"] = (p, W.random_state(p, r), W.random_controls(p, r), 7)
        p = W.quadrotor_k4096(K=600, T=29, nu=10.0, jump_rows=[0, 1, 2], mark_scale=0.2,
                              lam=20.0, noise_dtype=dt_)
        r = rng(21)
        c[f"quadrotor_rows012_{dt_}"] = (p, W.random_state(p, r, 0.1),
                                         W.random_controls(p, r, 0.2), 8)
    p = W.quadrotor_alg1()
    r = rng(8)
    c["quadrotor_alg1_K4096_T100"] = (p, W.random_state(p, r, 0.1), W.random_controls(p, r, 0.2), 12)
    p = W.cartpole_k1000(K=5000, T=50, nu=0.0)
    c["cartpole_no_jumps"] = (p, W.initial_state(p), W.initial_controls(p), 4)
    return c


CASES = _cases()


@pytest.mark.parametrize("name", list(CASES))
def test_iteration_matches_oracle(cuda, name):
    prob, x0, U, it = CASES[name]
    rep = parity.run_and_compare(prob, x0, U, it)
    _record(name, rep)


@pytest.mark.parametrize("tile", [(1, 64, 4), (2, 96, 8), (3, 32, 4), (4, 128, 8), (4, 32, 16)],
                         ids=["fused", "split", "staged_small_blocks", "block_records",
                              "block_records_small_blocks"])
def test_other_rollout_tiles_match_oracle(cuda, tile):
    """Non-default launch shapes against the oracle directly (they are also
    compared bit for bit with one another in test_gpu_api)."""
    prob, x0, U, it = CASES["quadrotor_laplace_bf16_sqrtdt"]
    rep = parity.run_and_compare(prob, x0, U, it, tile=tile)
    _record(f"quadrotor_laplace_bf16_sqrtdt_tile{tile}", rep)


@pytest.mark.parametrize("tile", [(1, 64, 4), (2, 96, 8), (3, 32, 4), (3, 128, 16), (4, 96, 8)],
                         ids=["fused", "split", "staged_small_blocks", "staged_long_stages",
                              "block_records"])
@pytest.mark.parametrize("name", ["cartpole_rows02_f32", "cartpole_rows02_bf16",
                                  "quadrotor_rows012_f32", "quadrotor_rows012_bf16"])
def test_non_default_jump_rows_every_tile_matches_oracle(cuda, name, tile):
    prob, x0, U, it = CASES[name]
    rep = parity.run_and_compare(prob, x0, U, it, tile=tile)
    assert rep["jumps"] > 100
    _record(f"{name}_tile{tile}", rep)


def _sparse_cases():
    """State-jump problems with more rollout blocks of 128 than a GB300 has
    SMs (152), where the jump records are sparse (jump masks, marks drawn by
    the lanes of a warp on jumps, records gathered by the rollout): a ragged K
    and a horizon that ends inside a stage, default and other jump rows."""
    c = {}
    p = W.quadrotor_k4096(K=24577, T=40, nu=10.0, lam=20.0, name="quadrotor_K24577_T40_sparse")
    r = np.random.default_rng(30)
    c["quadrotor_K24577_T40"] = (p, W.random_state(p, r, 0.1), W.random_controls(p, r, 0.2), 3)
    p = W.cartpole_k1000(K=20001, T=33, nu=10.0, jump_rows=[0, 2], noise_dtype="bf16",
                         name="cartpole_rows02_K20001_T33_sparse")
    r = np.random.default_rng(31)
    c["cartpole_rows02_K20001_T33_bf16"] = (p, W.random_state(p, r), W.random_controls(p, r), 11)
    return c


SPARSE_CASES = _sparse_cases()


@pytest.mark.parametrize("tile", [None, (2, 128, 4), (2, 64, 8), (3, 128, 16), (3, 64, 4), (3, 96, 8),
                                  (4, 128, 8), (4, 96, 16)],
                         ids=["default", "split", "split_64", "staged_long", "staged_64_short",
                              "staged_96", "block_records", "block_records_96"])
@pytest.mark.parametrize("name", list(SPARSE_CASES))
def test_sparse_jump_records_every_tile_match_oracle(cuda, name, tile):
    prob, x0, U, it = SPARSE_CASES[name]
    rep = parity.run_and_compare(prob, x0, U, it, tile=tile)
    assert rep["jumps"] > 10000
    _record(f"{name}_tile{tile}", rep)


@pytest.mark.parametrize("tile", [None, (4, 128, 8)], ids=["default", "block_records"])
def test_large_quadrotor_sampled_and_full_update(cuda, tile):
    """K=65536, T=200, dt=0.005, Laplace marks at 5/s, bfloat16 noise: every
    rollout's counts, marks, noise and cost, and the full update, against the
    oracle over all K."""
    prob = W.large_quadrotor()
    x0, U = W.initial_state(prob), W.initial_controls(prob)
    g = parity.gpu_iteration(prob, x0, U, 0, tile=tile)
    r = parity.oracle_iteration(prob, x0, U, 0)
    rep = parity.compare_iteration(prob, U, g, r)
    _record(f"quadrotor_K65536_T200_bf16_laplace_tile{tile}", rep)


def test_maximum_rollout_count(cuda):
    """K = 2^24, the largest rollout count the library accepts (T = 2, a jump
    rate high enough for many jumps): every rollout's counts, marks and noise,
    all K costs and the full update against the oracle."""
    prob = W.cartpole_k1000(K=1 << 24, T=2, nu=20.0, name="cartpole_K16777216_T2")
    x0 = W.random_state(prob, np.random.default_rng(24), 0.2)
    U = W.random_controls(prob, np.random.default_rng(25), 0.5)
    g = parity.gpu_iteration(prob, x0, U, 5)
    r = parity.oracle_iteration(prob, x0, U, 5)
    rep = parity.compare_iteration(prob, U, g, r)
    assert rep["jumps"] > 100000
    _record("cartpole_K16777216_T2", rep)


def test_all_costs_non_finite_leaves_controls(cuda):
    from paper_1807_06108_gb300 import mppi
    prob = W.cartpole_k1000(K=128, T=8)
    x0 = np.array([np.nan, 0, 0, 0], dtype=np.float32)
    U = W.random_controls(prob, np.random.default_rng(8))
    s = mppi.Solver(prob)
    try:
        s.set_controls(U)
        costs = s.rollout_cost(x0)
        s.update()
        with pytest.raises(mppi.MppiError) as e:
            s.sync()
        assert e.value.code == mppi.ENONFINITE
        assert np.all(np.isinf(costs.cpu().numpy()))
        np.testing.assert_array_equal(s.controls(), U)
        s.sync()  # the status word was cleared
    finally:
        s.close()
