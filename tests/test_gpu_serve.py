"""GPU tests of the served form: a session's results are the same alone and
in a concurrent mix (bit for bit: the kernels' reductions have a fixed order
and sessions share no state), equal to the plain context path, and survive
eviction under a small memory budget (checkpoint and restore are exact)."""

import numpy as np
import pytest

from paper_1807_06108_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _sessions():
    return [
        W.quadrotor_k4096(K=2048, T=50, iters=3, seed=1 << 33, lam=20.0, name="s0"),
        W.cartpole_k1000(K=1000, T=50, iters=1, seed=2 << 33, name="s1"),
        W.quadrotor_k4096(K=1024, T=80, iters=2, seed=3 << 33, lam=20.0, name="s2"),
        W.cartpole_k1000(K=4096, T=64, iters=1, seed=4 << 33, noise_dtype="bf16", name="s3"),
        W.quadrotor_k4096(K=512, T=30, iters=4, seed=5 << 33, lam=20.0, mark_law="laplace", name="s4"),
    ]


def _trace(probs, n_steps, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for i, p in enumerate(probs):
        x = W.initial_state(p).astype(np.float32)
        xs = []
        for _ in range(n_steps):
            x = x + W.state_drift(p, rng)
            xs.append(x.copy())
        out.append(xs)
    return out


def test_alone_equals_in_mix_and_plain_path(cuda):
    from paper_1807_06108_gb300 import mppi
    probs = _sessions()
    xs = _trace(probs, 4)
    # session 0 alone
    srv = mppi.Server(probs[:1], max_inflight=4)
    try:
        alone = [srv.wait(srv.submit(0, x)) for x in xs[0]]
        U_alone = srv.controls(0)
    finally:
        srv.close()
    # every session, all requests submitted at once, interleaved
    srv = mppi.Server(probs, max_inflight=8)
    try:
        tickets = [[] for _ in probs]
        for step in range(4):
            for i in range(len(probs)):
                tickets[i].append(srv.submit(i, xs[i][step]))
        srv.drain()
        mix = [srv.wait(t) for t in tickets[0]]
        U_mix = srv.controls(0)
        st = srv.stats()
        assert st["completed"] == st["submitted"] == 4 * len(probs)
        assert st["p99_ms"] >= st["p50_ms"] > 0
    finally:
        srv.close()
    for a, b in zip(alone, mix):
        np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(U_alone, U_mix)
    # the plain context path
    s = mppi.Solver(probs[0])
    try:
        plain = [s.step(x) for x in xs[0]]
        U_plain = s.controls()
    finally:
        s.close()
    for a, b in zip(plain, mix):
        np.testing.assert_array_equal(a[:4], b[:4])
    np.testing.assert_array_equal(U_plain, U_mix)


def test_eviction_under_small_budget_is_exact(cuda):
    from paper_1807_06108_gb300 import mppi
    probs = _sessions()[:4]
    sizes = [mppi.mppi_jump_workspace_bytes(mppi.config_from_problem(p)) for p in probs]
    xs = _trace(probs, 3, seed=1)
    ref = mppi.Server(probs, max_inflight=4)
    try:
        tix = [[ref.submit(i, xs[i][k]) for k in range(3)] for i in range(4)]
        ref.drain()
        r_u = [[ref.wait(t) for t in ts] for ts in tix]
        r_U = [ref.controls(i) for i in range(4)]
    finally:
        ref.close()
    small = mppi.Server(probs, budget_bytes=max(sizes) + min(sizes), max_inflight=4)
    try:
        tix = []
        for k in range(3):  # round robin: every request needs an eviction
            tix.append([small.submit(i, xs[i][k]) for i in range(4)])
        small.drain()
        st = small.stats()
        assert st["evictions"] > 0 and st["resident_bytes"] <= max(sizes) + min(sizes)
        for i in range(4):
            for k in range(3):
                np.testing.assert_array_equal(small.wait(tix[k][i]), r_u[i][k])
            np.testing.assert_array_equal(small.controls(i), r_U[i])
    finally:
        small.close()


def test_bad_requests_rejected(cuda):
    from paper_1807_06108_gb300 import mppi
    probs = _sessions()[:2]
    with pytest.raises(mppi.MppiError):
        mppi.Server(probs, budget_bytes=1024)
    srv = mppi.Server(probs)
    try:
        with pytest.raises(mppi.MppiError):
            srv.submit(7, np.zeros(12))
    finally:
        srv.close()


def test_served_workload_alone_equals_in_mix(cuda):
    """The 64 sessions of the served workload (mixed plants, K up to 16384,
    T up to 200, one or ten iterations per request) under the 20 GB budget:
    three requests per session, all submitted at once and interleaved, so
    that up to 32 run concurrently; every session's u0 sequence and final
    controls equal, bit for bit, the same requests run alone through the
    plain context path."""
    from paper_1807_06108_gb300 import mppi
    probs = W.served_sessions()
    assert len(probs) == 64 and max(p["K"] for p in probs) == 16384
    assert max(p["T"] for p in probs) == 200
    xs = _trace(probs, 3, seed=4)
    srv = mppi.Server(probs, budget_bytes=20 << 30, max_inflight=32)
    try:
        tickets = [[srv.submit(i, xs[i][k]) for i in range(len(probs))] for k in range(3)]
        srv.drain(300)
        mix = [[srv.wait(tickets[k][i]) for k in range(3)] for i in range(len(probs))]
        U_mix = [srv.controls(i) for i in range(len(probs))]
        st = srv.stats()
        assert st["completed"] == 3 * len(probs) and st["evictions"] == 0
    finally:
        srv.close()
    for i, p in enumerate(probs):
        s = mppi.Solver(p)
        try:
            alone = [s.step(x) for x in xs[i]]
            U_alone = s.controls()
        finally:
            s.close()
        m = len(alone[0])
        for a, b in zip(alone, mix[i]):
            np.testing.assert_array_equal(a, b[:m])
        np.testing.assert_array_equal(U_alone, U_mix[i])
