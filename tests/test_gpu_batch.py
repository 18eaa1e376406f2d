"""GPU tests of the batched form: one persistent launch per batched step
solves every instance as Algorithm 1 would on its own (checked against the
oracle's MPC step, instance by instance, over two consecutive steps), any
block size gives the same answer within the update tolerance, the
autotuner leaves the state untouched, and a dependency wait that never
completes ends the step with MPPI_ETIMEOUT instead of hanging."""

import numpy as np
import pytest

import oracle
from paper_1807_06108_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _mixed(noise_dtype):
    return [
        W.cartpole_k1000(K=300, T=17, seed=11, noise_dtype=noise_dtype, iters=1),
        W.quadrotor_k4096(K=700, T=40, seed=12, noise_dtype=noise_dtype, iters=3, lam=20.0),
        W.cartpole_k1000(K=1000, T=50, seed=13, noise_dtype=noise_dtype, iters=2, nu=3.0),
        W.quadrotor_k4096(K=2048, T=23, seed=14, noise_dtype=noise_dtype, iters=1, lam=50.0,
                          mark_law="laplace", nu=4.0),
        W.quadrotor_k4096(K=96, T=64, seed=15, noise_dtype=noise_dtype, iters=2,
                          jump_channel="control", mark_scale=0.3, lam=30.0),
        W.cartpole_k1000(K=33, T=5, seed=16, noise_dtype=noise_dtype, iters=4),
        W.quadrotor_k4096(K=256, T=31, seed=17, noise_dtype=noise_dtype, iters=3, lam=20.0,
                          alpha_decay=0.6),
    ]


def _states(probs, rng):
    return [W.random_state(p, rng, 0.1) for p in probs]


def _check_against_oracle(probs, states, U_in, it0, u0s, U_out):
    for i, p in enumerate(probs):
        u0_ref, U_ref = oracle.step(p, states[i], U_in[i], it0[i], p["iters"])
        U0 = np.asarray(U_in[i], dtype=np.float64)
        den = max(np.max(np.abs(U_ref[:-1] - U0[1:])), np.max(np.abs(u0_ref - U0[0])), 1e-30)
        err = max(np.max(np.abs(U_out[i][:-1] - U_ref[:-1])), np.max(np.abs(u0s[i] - u0_ref))) / den
        np.testing.assert_array_equal(U_out[i][-1], np.asarray(p["u_init"], dtype=np.float32))
        assert err <= 1e-4 * p["iters"], (p["name"], err)


@pytest.mark.parametrize("noise_dtype", ["bf16", "f32"])
def test_batched_steps_match_oracle(cuda, noise_dtype):
    from paper_1807_06108_gb300 import mppi
    probs = _mixed(noise_dtype)
    rng = np.random.default_rng(0)
    b = mppi.Batch(probs)
    try:
        its = [0] * len(probs)
        U_in = [W.initial_controls(p) for p in probs]
        for _ in range(2):
            states = _states(probs, rng)
            u0s = b.step(states)
            U_out = [b.controls(i) for i in range(len(probs))]
            _check_against_oracle(probs, states, U_in, its, u0s, U_out)
            its = [its[i] + p["iters"] for i, p in enumerate(probs)]
            assert [b.iteration(i) for i in range(len(probs))] == its
            U_in = U_out
    finally:
        b.close()


def test_block_sizes_agree_and_autotune_restores(cuda):
    from paper_1807_06108_gb300 import mppi
    probs = _mixed("bf16")
    states = _states(probs, np.random.default_rng(1))
    results = {}
    for tile in [(64, 4), (128, 4), (256, 4), (128, 8), (64, 8)]:
        b = mppi.Batch(probs)
        try:
            b.set_tile(*tile)
            assert b.tile() == tile and b.tuning() == tile[0]
            b.step(states)
            results[tile] = [b.controls(i) for i in range(len(probs))]
        finally:
            b.close()
    for tile in [(64, 4), (256, 4), (128, 8), (64, 8)]:
        for i in range(len(probs)):
            ref = results[(128, 4)][i].astype(np.float64)
            den = max(np.max(np.abs(ref - W.initial_controls(probs[i]))), 1e-30)
            assert np.max(np.abs(results[tile][i] - ref)) / den <= 1e-4 * probs[i]["iters"]
    # the chunk only reorders when the random numbers are drawn: same block, same result
    for i in range(len(probs)):
        np.testing.assert_array_equal(results[(128, 8)][i], results[(128, 4)][i])
    b = mppi.Batch(probs)
    try:
        b.set_states(states)
        (blk, ch), ms = b.autotune(reps=1)
        assert blk in (64, 128, 256) and ch in (4, 8) and ms > 0
        assert all(b.iteration(i) == 0 for i in range(len(probs)))
        b.set_tile(128, 4)
        b.step(states)
        for i in range(len(probs)):
            np.testing.assert_array_equal(b.controls(i), results[(128, 4)][i])
    finally:
        b.close()


def test_stalled_dependency_times_out_and_recovers(cuda):
    from paper_1807_06108_gb300 import mppi
    probs = _mixed("bf16")[:2]
    states = _states(probs, np.random.default_rng(2))
    b = mppi.Batch(probs)
    try:
        b.inject_stall(True)
        with pytest.raises(mppi.MppiError) as e:
            b.step(states)
        assert e.value.code == mppi.ETIMEOUT
        b.inject_stall(False)
        for i, p in enumerate(probs):
            b.set_controls(i, W.initial_controls(p))
        b.step(states)  # the batch is usable again
    finally:
        b.close()


def test_full_batched_workload_matches_oracle_and_plain_path(cuda):
    """All 256 instances of the batched workload (bfloat16 noise, K up to
    8192, T up to 150, 35k work items on the persistent grid), two batched
    steps: a fixed subset of 38 instances -- every instance with K = 8192 and
    T >= 140 (both plants) and every eighth instance -- against the oracle's
    MPC step, and every instance against the plain one-context path."""
    from paper_1807_06108_gb300 import mppi
    probs = W.batched_instances()
    assert len(probs) == 256
    big = [i for i, p in enumerate(probs) if p["K"] == 8192 and p["T"] >= 140]
    assert {probs[i]["system"] for i in big} == {"cartpole", "quadrotor"}
    subset = sorted(set(big) | set(range(0, 256, 8)))
    assert len(subset) >= 32
    rng = np.random.default_rng(3)
    b = mppi.Batch(probs)
    solvers = [mppi.Solver(p) for p in probs]
    try:
        U_in = [W.initial_controls(p) for p in probs]
        for step in range(2):
            states = _states(probs, rng)
            u0s = b.step(states)
            U_out = [b.controls(i) for i in range(len(probs))]
            if step == 0:
                sub = [probs[i] for i in subset]
                _check_against_oracle(sub, [states[i] for i in subset], [U_in[i] for i in subset],
                                      [0] * len(subset), [u0s[i] for i in subset],
                                      [U_out[i] for i in subset])
            for i, (p, s) in enumerate(zip(probs, solvers)):
                s.set_controls(U_in[i])  # the same starting controls as the batch
                u0_p = s.step(states[i])
                U_p = s.controls()
                U0 = np.asarray(U_in[i], dtype=np.float64)
                den = max(np.max(np.abs(U_p[:-1] - U0[1:])), np.max(np.abs(u0_p - U0[0])), 1e-30)
                err = max(np.max(np.abs(U_out[i] - U_p)), np.max(np.abs(u0s[i] - u0_p))) / den
                assert err <= 1e-4 * p["iters"], (step, p["name"], err)
            assert [b.iteration(i) for i in range(len(probs))] == \
                [(step + 1) * p["iters"] for p in probs]
            U_in = U_out
    finally:
        b.close()
        for s in solvers:
            s.close()
