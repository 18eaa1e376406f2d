"""Multi-process paths on CPU with the gloo backend (world size 2): the
per-rank problem keys and the max-over-ranks timing reduction the benchmark
uses, and the rollout-sharded exchange of Eq. 37 partials (one MIN and one
SUM all-reduce with the log-sum-exp rescale), which must reproduce the
oracle's full update over all rollouts."""

import os
import socket

import numpy as np
import pytest

import oracle
from paper_1807_06108_gb300 import dist as D
from paper_1807_06108_gb300 import workloads as W

WORLD = 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, port, q):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=WORLD)
    try:
        seed = D.rank_seed(0, rank)
        tmax = D.max_over_ranks(dist, 1.5 + rank)
        prob = W.cartpole_k1000(K=601, T=12, nu=8.0)
        x0 = W.random_state(prob, np.random.default_rng(0))
        U = W.random_controls(prob, np.random.default_rng(1))
        k0, k1 = D.shard_range(prob["K"], rank, WORLD)
        r = oracle.rollouts(prob, x0, U, 3, k0, k1 - k0, delta=True)
        rho_g, Z_g, N_g = D.partial_from_costs(r["S"], r["delta"], prob["lam"])
        dU, rho, Z = D.allreduce_partials(dist, rho_g, Z_g, N_g, prob["lam"])
        q.put((rank, seed, tmax, dU, rho, Z, (k0, k1)))
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_paths():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, port, q)) for r in range(WORLD)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(WORLD):
        item = q.get(timeout=120)
        out[item[0]] = item
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # weak scaling: distinct keys, one timing value for all ranks
    assert out[0][1] != out[1][1]
    assert out[0][2] == out[1][2] == 2.5
    # the shards tile [0, K)
    assert out[0][6][0] == 0 and out[0][6][1] == out[1][6][0] and out[1][6][1] == 601
    # the exchange reproduces the full update, identically on both ranks
    prob = W.cartpole_k1000(K=601, T=12, nu=8.0)
    x0 = W.random_state(prob, np.random.default_rng(0))
    U = W.random_controls(prob, np.random.default_rng(1))
    full = oracle.iteration(prob, x0, U, 3)
    dU_ref = full["U"] - U.astype(np.float64)
    np.testing.assert_array_equal(out[0][3], out[1][3])
    np.testing.assert_allclose(out[0][3], dU_ref, rtol=1e-10, atol=1e-12)
    assert out[0][4] == full["diag"][0]


def test_shard_range_and_single_process_combine():
    for K in (1, 7, 1000, 65536):
        for world in (1, 2, 3, 8):
            ranges = [D.shard_range(K, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == K
            assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
    prob = W.quadrotor_k4096(K=300, T=7, lam=5.0)
    x0, U = W.initial_state(prob), W.initial_controls(prob)
    r = oracle.rollouts(prob, x0, U, 0, 0, 300, delta=True)
    parts = []
    for k0, k1 in [(0, 100), (100, 101), (101, 300)]:
        parts.append(D.partial_from_costs(r["S"][k0:k1], r["delta"][:, k0:k1, :], prob["lam"]))
    dU, rho, Z = D.combine_partials(parts, prob["lam"])
    w, diag = oracle.softmin(r["S"], prob["lam"])
    np.testing.assert_allclose(dU, np.einsum("k,tkm->tm", w, r["delta"]), rtol=1e-10, atol=1e-13)
    assert rho == diag[0]
    assert Z == pytest.approx(diag[1], rel=1e-12)
