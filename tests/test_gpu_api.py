"""GPU tests of the C ABI beyond single-iteration parity: rollout tiles give
identical results, the graph-replayed MPC step equals the direct calls and
the oracle's Algorithm-1 step (execute u_0, shift, append u_init),
checkpoint/restore continues the random stream exactly, and phase timing
reports every iteration."""

import numpy as np
import pytest

import oracle
from paper_1807_06108_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _solver(prob, tile=None):
    from paper_1807_06108_gb300 import mppi
    s = mppi.Solver(prob)
    if tile:
        mppi.mppi_jump_set_tuning(s.ctx, *tile)
    return s


def _one_iteration(prob, x0, U, it, tile):
    s = _solver(prob, tile)
    try:
        s.set_controls(U)
        s.set_iteration(it)
        s.enable_debug()
        costs = s.rollout_cost(x0)
        s.update()
        s.sync()
        return (costs.cpu().numpy(), s.controls(), s.noise(), s.dbg_counts.cpu().numpy(),
                s.dbg_J.cpu().numpy(), s.weights())
    finally:
        s.close()


@pytest.mark.parametrize("prob", [
    W.cartpole_k1000(K=999, T=29),
    W.quadrotor_k4096(K=1100, T=41, nu=9.0),
    W.quadrotor_k4096(K=700, T=13, nu=9.0, jump_channel="control", noise_dtype="bf16",
                      mark_law="laplace"),
    W.quadrotor_k4096(K=300, T=21, nu=12.0, jump_rows=[3, 4, 5, 9], noise_dtype="bf16"),
    W.cartpole_k1000(K=500, T=19, nu=10.0, jump_rows=[0, 2], noise_dtype="bf16"),
    W.quadrotor_k4096(K=400, T=23, nu=10.0, jump_rows=[0, 1, 2], mark_scale=0.2),
], ids=["cartpole", "quadrotor_state", "quadrotor_control_bf16", "quadrotor_q4_state_bf16",
        "cartpole_rows02_bf16", "quadrotor_rows012"])
def test_rollout_tiles_are_bit_identical(cuda, prob):
    rng = np.random.default_rng(0)
    x0, U = W.random_state(prob, rng, 0.1), W.random_controls(prob, rng, 0.2)
    ref = _one_iteration(prob, x0, U, 3, (1, 128, 4))
    for tile in [(2, 128, 4), (2, 64, 2), (2, 32, 8), (1, 32, 4), (1, 64, 8), (1, 128, 16), (2, 96, 4),
                 (3, 128, 8), (3, 64, 4), (3, 32, 16), (3, 96, 8)]:
        got = _one_iteration(prob, x0, U, 3, tile)
        for a, b in zip(ref, got):
            np.testing.assert_array_equal(a, b)
    # block records (tile 4): the same costs, perturbations, counts and marks;
    # the update sums in another order
    U0 = U.astype(np.float64)
    for tile in [(4, 128, 8), (4, 64, 4), (4, 32, 16)]:
        got = _one_iteration(prob, x0, U, 3, tile)
        for i in (0, 2, 3, 4):
            np.testing.assert_array_equal(ref[i], got[i])
        dU_ref, dU = ref[1] - U0, got[1] - U0
        assert np.max(np.abs(dU - dU_ref)) <= 1e-5 * np.max(np.abs(dU_ref))
        np.testing.assert_allclose(got[5], ref[5], rtol=1e-5, atol=1e-12)


def test_invalid_tile_rejected(cuda):
    from paper_1807_06108_gb300 import mppi
    s = _solver(W.cartpole_k1000(K=64, T=4))
    try:
        for bad in [(0, 128, 4), (5, 128, 4), (4, 128, 2), (1, 128, 2), (3, 128, 2), (2, 128, 16), (2, 48, 4), (2, 256, 4),
                    (1, 16, 4), (2, 64, 3)]:
            with pytest.raises(mppi.MppiError):
                mppi.mppi_jump_set_tuning(s.ctx, *bad)
        assert mppi.mppi_jump_get_tuning(s.ctx) == (3, 96, 16)
    finally:
        s.close()


@pytest.mark.parametrize("tile", [None, (4, 128, 8)], ids=["default_tile", "block_records"])
@pytest.mark.parametrize("prob", [W.cartpole_k1000(), W.quadrotor_k4096(K=1024, T=60, iters=4),
                                  W.large_quadrotor()],
                         ids=["cartpole_K1000_T50", "quadrotor_K1024_T60_it4",
                              "quadrotor_K65536_T200_it5_bf16_streaming_update"])
def test_graph_step_equals_direct_calls_and_oracle(cuda, prob, tile):
    x0 = W.initial_state(prob)
    iters = prob["iters"]
    # graph-replayed step through the synchronous host call
    s = _solver(prob, tile)
    try:
        u0 = s.step(x0)
        U_step = s.controls()
        it_after = s.iteration()
    finally:
        s.close()
    # the same iterations through rollout_cost / update, then the shift by hand
    s = _solver(prob, tile)
    try:
        for _ in range(iters):
            s.rollout_cost(x0, want_costs=False)
            s.update()
        s.sync()
        U_direct = s.controls()
    finally:
        s.close()
    np.testing.assert_array_equal(u0, U_direct[0])
    np.testing.assert_array_equal(U_step[:-1], U_direct[1:])
    np.testing.assert_array_equal(U_step[-1], np.asarray(prob["u_init"], dtype=np.float32))
    assert it_after == iters
    # Algorithm 1 against the oracle, end to end over all iterations
    u0_ref, U_ref = oracle.step(prob, x0, W.initial_controls(prob), 0, iters)
    dU_ref = U_ref[:-1] - W.initial_controls(prob)[1:]
    den = max(np.max(np.abs(dU_ref)), np.max(np.abs(u0_ref - prob["u_init"])), 1e-30)
    err = max(np.max(np.abs(U_step[:-1] - U_ref[:-1])), np.max(np.abs(u0 - u0_ref))) / den
    print(prob["name"], "end-to-end step rel err", err)
    assert err <= 1e-4 * iters


@pytest.mark.parametrize("prob", [
    W.quadrotor_k4096(K=1024, T=60, iters=4, alpha_decay=0.6),
    W.cartpole_k1000(K=500, T=30, iters=3, alpha=0.7, alpha_decay=0.5),
], ids=["quadrotor_decay06", "cartpole_alpha07_decay05"])
def test_step_size_schedule_matches_oracle(cuda, prob):
    """alpha^r = alpha * alpha_decay^r over the iterations of one MPC step
    (Eq. 48-49): the graph-replayed step against the oracle's Algorithm-1
    step with the same schedule."""
    x0 = W.initial_state(prob)
    iters = prob["iters"]
    s = _solver(prob)
    try:
        u0 = s.step(x0)
        U_step = s.controls()
    finally:
        s.close()
    u0_ref, U_ref = oracle.step(prob, x0, W.initial_controls(prob), 0, iters)
    dU_ref = U_ref[:-1] - W.initial_controls(prob)[1:]
    den = max(np.max(np.abs(dU_ref)), np.max(np.abs(u0_ref - prob["u_init"])), 1e-30)
    err = max(np.max(np.abs(U_step[:-1] - U_ref[:-1])), np.max(np.abs(u0 - u0_ref))) / den
    assert err <= 1e-4 * iters, err


def test_checkpoint_restore_continues_stream(cuda):
    prob = W.quadrotor_k4096(K=512, T=30, iters=3)
    x0 = W.initial_state(prob)
    s = _solver(prob)
    try:
        s.step(x0)
        blob = s.get_state()
        a1 = s.step(x0)
        a2 = s.step(x0)
        Ua = s.controls()
    finally:
        s.close()
    s = _solver(prob)
    try:
        s.set_state(blob)
        assert s.iteration() == 3
        b1 = s.step(x0)
        b2 = s.step(x0)
        Ub = s.controls()
    finally:
        s.close()
    np.testing.assert_array_equal(a1, b1)
    np.testing.assert_array_equal(a2, b2)
    np.testing.assert_array_equal(Ua, Ub)


def test_checkpoint_rejects_other_configuration(cuda):
    from paper_1807_06108_gb300 import mppi
    s = _solver(W.cartpole_k1000(K=64, T=8))
    blob = s.get_state()
    s.close()
    t = _solver(W.cartpole_k1000(K=64, T=8, seed=5))
    try:
        with pytest.raises(mppi.MppiError):
            t.set_state(blob)
        with pytest.raises(mppi.MppiError):
            t.set_state(blob[:-4])
    finally:
        t.close()


def test_phase_timing_covers_every_iteration(cuda):
    from paper_1807_06108_gb300 import mppi
    prob = W.quadrotor_k4096(K=2048, T=50, iters=5)
    s = _solver(prob)
    try:
        mppi.mppi_jump_enable_timing(s.ctx, True)
        x0 = W.initial_state(prob)
        s.step(x0)
        r, u, n = mppi.mppi_jump_phase_times(s.ctx)
        assert n == 5 and r > 0 and u > 0
        mppi.mppi_jump_enable_timing(s.ctx, False)
        s.step(x0)
        assert mppi.mppi_jump_phase_times(s.ctx) == (0.0, 0.0, 0)
    finally:
        s.close()


def test_autotune_keeps_results(cuda):
    from paper_1807_06108_gb300 import mppi
    prob = W.quadrotor_k4096(K=1536, T=40, iters=3)
    x0 = W.initial_state(prob)
    s = _solver(prob)
    try:
        ref = [s.step(x0) for _ in range(2)]
        U_ref = s.controls()
    finally:
        s.close()
    s = _solver(prob)
    try:
        s.set_x0(x0)
        (variant, block, chunk), ms = mppi.mppi_jump_autotune(s.ctx, s.x0.data_ptr(), 3, reps=2)
        assert variant in (1, 2, 3) and block in (32, 64, 128) and chunk in (2, 4, 8, 16) and ms > 0
        assert s.iteration() == 0
        got = [s.step(x0) for _ in range(2)]
        np.testing.assert_array_equal(np.array(ref), np.array(got))
        np.testing.assert_array_equal(U_ref, s.controls())
    finally:
        s.close()


@pytest.mark.parametrize("tile", [None, (1, 128, 4), (2, 64, 4)], ids=["staged", "fused", "split"])
def test_step_status_word_reports_and_clears(cuda, tile):
    """A step whose every cost is non-finite (a NaN state) reports
    MPPI_ENONFINITE and leaves U unchanged; reading the status word clears
    it, so the next step from a finite state succeeds and is bit-equal to a
    fresh context's step at the same counter (the step graph re-arms the
    running minimum of its first iteration itself).  Both the synchronous
    step and the asynchronous step followed by a sync."""
    from paper_1807_06108_gb300 import mppi
    prob = W.quadrotor_k4096(K=512, T=20, iters=3)
    bad = np.full(12, np.nan, dtype=np.float32)
    good = W.initial_state(prob)
    s, ref = _solver(prob, tile), _solver(prob, tile)
    try:
        U0 = s.controls()
        with pytest.raises(mppi.MppiError) as e:
            s.step(bad)
        assert e.value.code == mppi.ENONFINITE
        np.testing.assert_array_equal(s.controls(), U0)
        assert s.iteration() == prob["iters"]
        u_s = s.step(good)
        ref.set_iteration(prob["iters"])
        u_ref = ref.step(good)
        np.testing.assert_array_equal(u_s, u_ref)
        np.testing.assert_array_equal(s.controls(), ref.controls())
        # asynchronous: the error is reported by the next sync, then cleared
        s.set_x0(bad)
        mppi.mppi_jump_step_async(s.ctx, s.x0.data_ptr(), prob["iters"])
        with pytest.raises(mppi.MppiError) as e:
            s.sync()
        assert e.value.code == mppi.ENONFINITE
        s.set_x0(good)
        mppi.mppi_jump_step_async(s.ctx, s.x0.data_ptr(), prob["iters"])
        s.sync()
        ref.set_x0(good)
        mppi.mppi_jump_step_async(ref.ctx, ref.x0.data_ptr(), prob["iters"])
        ref.sync()
        assert s.iteration() == 4 * prob["iters"] and ref.iteration() == 3 * prob["iters"]
    finally:
        s.close()
        ref.close()
