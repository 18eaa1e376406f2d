"""GPU tests of rollout sharding through the C ABI: one problem's rollouts
split over shard contexts (configuration K = the shard's rollouts, rollout
offset = its first rollout), each exporting its partial record (rho_g, Z_g,
N_g) from the kernels; every shard applies all records and must end with
controls identical to the other shards', equal to the unsharded update and
to the oracle's full update (Eq. 37 over all rollouts).  Also a two-process
exchange of the library's records over gloo, a sharded MPC step, both
record sources (the update kernel's export and the rollout blocks' records)
and a shard with no finite cost."""

import math
import os
import socket

import numpy as np
import pytest

import oracle
from paper_1807_06108_gb300 import dist as D
from paper_1807_06108_gb300 import workloads as W

pytestmark = pytest.mark.gpu

U_RTOL = 1e-4


def _rel(dU, dU_ref):
    return float(np.max(np.abs(dU - dU_ref)) / max(np.max(np.abs(dU_ref)), 1e-30))


def _shards(prob, ranges, tile=None):
    from paper_1807_06108_gb300 import mppi
    out = []
    for k0, k1 in ranges:
        s = mppi.Solver(dict(prob, K=k1 - k0))
        if tile:
            mppi.mppi_jump_set_tuning(s.ctx, *tile)
        s.set_rollout_offset(k0)
        out.append(s)
    return out


CASES = {
    "quadrotor_K2333_T40": (W.quadrotor_k4096(K=2333, T=40, lam=20.0), [(0, 1000), (1000, 2333)]),
    "cartpole_K3001_T31_bf16": (W.cartpole_k1000(K=3001, T=31, nu=6.0, noise_dtype="bf16"),
                                [(0, 1024), (1024, 1025), (1025, 3001)]),
    "quadrotor_control_K1500_T20": (W.quadrotor_k4096(K=1500, T=20, nu=6.0, jump_channel="control",
                                                      mark_scale=0.3, lam=30.0), [(0, 700), (700, 1500)]),
}


@pytest.mark.parametrize("tile", [None, (3, 128, 8), (4, 128, 8), (4, 64, 16), (2, 64, 4)],
                         ids=["default", "staged", "block_records", "block_records_64", "split"])
@pytest.mark.parametrize("name", list(CASES))
def test_sharded_update_equals_unsharded_and_oracle(cuda, name, tile):
    torch = cuda
    from paper_1807_06108_gb300 import mppi
    prob, ranges = CASES[name]
    rng = np.random.default_rng(5)
    x0, U = W.random_state(prob, rng, 0.1), W.random_controls(prob, rng, 0.2)
    it = 4
    shards = _shards(prob, ranges, tile)
    try:
        recs = []
        for s in shards:
            s.set_controls(U)
            s.set_iteration(it)
            recs.append(s.rollout_partial(x0))
        torch.cuda.synchronize()
        recs = torch.stack(recs)
        Us = []
        for s in shards:
            s.apply_partials(recs)
            s.sync()
            Us.append(s.controls())
            assert s.iteration() == it + 1
        for Ui in Us[1:]:
            np.testing.assert_array_equal(Ui, Us[0])  # every shard holds the same controls
        rec_np = recs.cpu().numpy().astype(np.float64)
    finally:
        for s in shards:
            s.close()
    # the unsharded context
    full = mppi.Solver(prob)
    try:
        if tile:
            mppi.mppi_jump_set_tuning(full.ctx, *tile)
        full.set_controls(U)
        full.set_iteration(it)
        full.rollout_cost(x0, want_costs=False)
        full.update()
        full.sync()
        U_full = full.controls()
    finally:
        full.close()
    U0 = U.astype(np.float64)
    assert _rel(Us[0] - U0, U_full - U0) <= U_RTOL
    # the oracle's full update and each shard's record
    ref = oracle.iteration(prob, x0, U, it)
    assert _rel(Us[0] - U0, ref["U"] - U0) <= U_RTOL
    r_all = oracle.rollouts(prob, x0, U, it, 0, prob["K"], delta=True)
    # the record's rho leaves out the rollout-independent control cost
    # C = sum_j lambda/2 u_j^T Sigma^-1 u_j of the augmented cost
    C = 0.5 * prob["lam"] * float(np.sum(U0 ** 2 / np.asarray(prob["sigma"], dtype=np.float64) ** 2))
    for (k0, k1), rec in zip(ranges, rec_np):
        Sg = r_all["S"][k0:k1]
        rho_ref = Sg.min()
        assert abs(rec[0] + C - rho_ref) <= 1e-4 * max(1.0, abs(rho_ref))
        e = np.exp(-(Sg - rho_ref) / prob["lam"])
        assert abs(rec[1] - e.sum()) <= 1e-4 * e.sum()
        mean_ref = np.einsum("k,tkm->tm", e, r_all["delta"][:, k0:k1, :]).ravel() / e.sum()
        assert _rel(rec[2:] / rec[1], mean_ref) <= U_RTOL


def test_two_process_gloo_exchange_of_library_records(cuda):
    """Two processes on the same GPU, each a shard of one problem, exchange
    the records their kernels wrote over gloo and apply both: both end with
    the same controls, equal to the unsharded update."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    procs = [ctx.Process(target=_gloo_worker, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(2):
        item = q.get(timeout=300)
        out[item[0]] = item[1]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    np.testing.assert_array_equal(out[0], out[1])
    from paper_1807_06108_gb300 import mppi
    prob, x0, U = _gloo_problem()
    full = mppi.Solver(prob)
    try:
        full.set_controls(U)
        full.rollout_cost(x0, want_costs=False)
        full.update()
        full.sync()
        U_full = full.controls()
    finally:
        full.close()
    U0 = U.astype(np.float64)
    assert _rel(out[0] - U0, U_full - U0) <= U_RTOL


def _gloo_problem():
    prob = W.quadrotor_k4096(K=3000, T=30, lam=20.0)
    rng = np.random.default_rng(9)
    return prob, W.random_state(prob, rng, 0.1), W.random_controls(prob, rng, 0.2)


def _gloo_worker(rank, port, q):
    import torch
    import torch.distributed as dist
    from paper_1807_06108_gb300 import mppi
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=2)
    try:
        prob, x0, U = _gloo_problem()
        k0, k1 = D.shard_range(prob["K"], rank, 2)
        s = mppi.Solver(dict(prob, K=k1 - k0))
        try:
            s.set_rollout_offset(k0)
            s.set_controls(U)
            rec = s.rollout_partial(x0)
            s.stream.synchronize()
            recs = D.allgather_records(dist, rec.cpu())
            s.apply_partials(recs)  # copied to the device on the solver's stream
            s.sync()
            q.put((rank, s.controls()))
        finally:
            s.close()
    finally:
        dist.destroy_process_group()


def test_sharded_mpc_step_equals_oracle_step(cuda):
    """iters = 3 iterations of one MPC step, each exchanging records, the
    last with the shift; against the unsharded graph step and the oracle's
    Algorithm-1 step."""
    torch = cuda
    from paper_1807_06108_gb300 import mppi
    prob = W.quadrotor_k4096(K=2048, T=25, iters=3, lam=20.0, alpha_decay=0.7)
    x0 = W.initial_state(prob)
    ranges = [(0, 512), (512, 2048)]
    shards = _shards(prob, ranges)
    try:
        for r in range(prob["iters"]):
            parts = [s.rollout_partial(x0) for s in shards]
            torch.cuda.synchronize()  # the records were written on the shards' streams
            recs = torch.stack(parts)
            for s in shards:
                s.apply_partials(recs, r=r, shift=(r == prob["iters"] - 1))
        for s in shards:
            s.sync()
        u0s = [s.u0.cpu().numpy() for s in shards]
        Us = [s.controls() for s in shards]
        its = [s.iteration() for s in shards]
    finally:
        for s in shards:
            s.close()
    np.testing.assert_array_equal(u0s[0], u0s[1])
    np.testing.assert_array_equal(Us[0], Us[1])
    assert its == [3, 3]
    u0_ref, U_ref = oracle.step(prob, x0, W.initial_controls(prob), 0, prob["iters"])
    dU_ref = U_ref[:-1] - W.initial_controls(prob)[1:]
    den = max(np.max(np.abs(dU_ref)), np.max(np.abs(u0_ref - prob["u_init"])), 1e-30)
    err = max(np.max(np.abs(Us[0][:-1] - U_ref[:-1])), np.max(np.abs(u0s[0] - u0_ref))) / den
    assert err <= U_RTOL * prob["iters"], err
    np.testing.assert_array_equal(Us[0][-1], np.asarray(prob["u_init"], dtype=np.float32))


def test_shard_without_finite_costs(cuda):
    torch = cuda
    from paper_1807_06108_gb300 import mppi
    prob = W.cartpole_k1000(K=200, T=9)
    U = W.random_controls(prob, np.random.default_rng(2))
    bad = np.array([np.nan, 0, 0, 0], dtype=np.float32)
    good = W.random_state(prob, np.random.default_rng(3))
    shards = _shards(prob, [(0, 100), (100, 200)], (4, 64, 8))
    try:
        for s in shards:
            s.set_controls(U)
        rec_bad = shards[0].rollout_partial(bad)
        rec_good = shards[1].rollout_partial(good)
        torch.cuda.synchronize()
        rb = rec_bad.cpu().numpy()
        assert math.isinf(rb[0]) and rb[1] == 0.0 and not rb[2:].any()
        # only the finite shard contributes
        shards[1].apply_partials(torch.stack([rec_bad, rec_good]))
        shards[1].sync()
        U_mix = shards[1].controls()
        # every record non-finite: U unchanged and ENONFINITE at the next sync
        shards[0].apply_partials(torch.stack([rec_bad, rec_bad]))
        with pytest.raises(mppi.MppiError) as e:
            shards[0].sync()
        assert e.value.code == mppi.ENONFINITE
        np.testing.assert_array_equal(shards[0].controls(), U)
    finally:
        for s in shards:
            s.close()
    r = oracle.rollouts(prob, good, U, 0, 100, 100, delta=True)
    w, _ = oracle.softmin(r["S"], prob["lam"])
    U_ref = oracle.update(w, r["delta"], U, prob["alpha"])
    U0 = U.astype(np.float64)
    assert _rel(U_mix - U0, U_ref - U0) <= U_RTOL


def test_invalid_shard_arguments(cuda):
    torch = cuda
    from paper_1807_06108_gb300 import mppi
    s = mppi.Solver(W.cartpole_k1000(K=64, T=4))
    try:
        with pytest.raises(mppi.MppiError):
            mppi.mppi_jump_set_rollout_offset(s.ctx, (1 << 32) - 32)
        t = torch.zeros(8, device="cuda")
        with pytest.raises(mppi.MppiError):
            mppi.mppi_jump_apply_partials(s.ctx, t.data_ptr(), 0)
        with pytest.raises(mppi.MppiError):
            mppi.mppi_jump_apply_partials(s.ctx, t.data_ptr(), 100000)
    finally:
        s.close()
