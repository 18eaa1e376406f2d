"""Multi-process paths on CPU with the gloo backend (world size 2): the
per-rank problem keys and the max-over-ranks timing reduction the benchmark
uses, and the exchange of rollout-shard partial records (an all-gather in
rank order).  The records here are built from the oracle's rollouts by the
test's own restatement of the record format (rho_g, Z_g, N_g), and their
combination with the log-sum-exp rescale must reproduce the oracle's full
update over all rollouts -- the same format the library's
mppi_jump_rollout_partial writes and mppi_jump_apply_partials combines
(checked on the GPU in test_gpu_shards.py)."""

import math
import os
import socket

import numpy as np
import pytest

import oracle
from paper_1807_06108_gb300 import dist as D
from paper_1807_06108_gb300 import workloads as W

WORLD = 2


def shard_record(S, delta, lam):
    """(rho_g, Z_g, N_g) of one shard, flattened like the library's record:
    rho_g = min S, Z_g = sum exp(-(S - rho_g)/lam), N_g = sum_k e_k delta_k."""
    S = np.asarray(S, dtype=np.float64)
    finite = np.isfinite(S)
    T, _, m = delta.shape
    if not finite.any():
        return np.concatenate([[math.inf, 0.0], np.zeros(T * m)])
    rho = float(S[finite].min())
    e = np.where(finite, np.exp(-(np.where(finite, S, rho) - rho) / lam), 0.0)
    N = np.einsum("k,tkm->tm", e, np.asarray(delta, dtype=np.float64))
    return np.concatenate([[rho, e.sum()], N.ravel()])


def combine_records(recs, lam):
    """dU = sum_g N_g s_g / sum_g Z_g s_g, s_g = exp(-(rho_g - rho)/lam)."""
    recs = np.asarray(recs, dtype=np.float64)
    rho = recs[:, 0].min()
    s = np.where(np.isfinite(recs[:, 0]), np.exp(-(recs[:, 0] - rho) / lam), 0.0)
    return (s @ recs[:, 2:]) / (s @ recs[:, 1]), rho


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    prob = W.cartpole_k1000(K=601, T=12, nu=8.0)
    x0 = W.random_state(prob, np.random.default_rng(0))
    U = W.random_controls(prob, np.random.default_rng(1))
    return prob, x0, U


def _worker(rank, port, q):
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=WORLD)
    try:
        seed = D.rank_seed(0, rank)
        tmax = D.max_over_ranks(dist, 1.5 + rank)
        prob, x0, U = _problem()
        k0, k1 = D.shard_range(prob["K"], rank, WORLD)
        r = oracle.rollouts(prob, x0, U, 3, k0, k1 - k0, delta=True)
        rec = torch.from_numpy(shard_record(r["S"], r["delta"], prob["lam"]))
        recs = D.allgather_records(dist, rec).numpy()
        dU, rho = combine_records(recs, prob["lam"])
        q.put((rank, seed, tmax, dU, rho, (k0, k1), recs))
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
    assert out[0][5][0] == 0 and out[0][5][1] == out[1][5][0] and out[1][5][1] == 601
    # both ranks received every record, in rank order
    np.testing.assert_array_equal(out[0][6], out[1][6])
    prob, x0, U = _problem()
    for rank in range(WORLD):
        k0, k1 = out[rank][5]
        r = oracle.rollouts(prob, x0, U, 3, k0, k1 - k0, delta=True)
        np.testing.assert_array_equal(out[0][6][rank], shard_record(r["S"], r["delta"], prob["lam"]))
    # the combination reproduces the full update, identically on both ranks
    full = oracle.iteration(prob, x0, U, 3)
    dU_ref = full["U"] - U.astype(np.float64)
    np.testing.assert_array_equal(out[0][3], out[1][3])
    np.testing.assert_allclose(out[0][3], dU_ref.ravel(), rtol=1e-10, atol=1e-12)
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
    recs = [shard_record(r["S"][k0:k1], r["delta"][:, k0:k1, :], prob["lam"])
            for k0, k1 in [(0, 100), (100, 101), (101, 300)]]
    dU, rho = combine_records(recs, prob["lam"])
    w, diag = oracle.softmin(r["S"], prob["lam"])
    np.testing.assert_allclose(dU, np.einsum("k,tkm->tm", w, r["delta"]).ravel(), rtol=1e-10,
                               atol=1e-13)
    assert rho == diag[0]
    # a shard with no finite cost contributes nothing
    S_bad = r["S"].copy()
    S_bad[100:101] = np.inf
    recs[1] = shard_record(S_bad[100:101], r["delta"][:, 100:101, :], prob["lam"])
    assert recs[1][0] == math.inf and recs[1][1] == 0.0 and not recs[1][2:].any()
    dU2, _ = combine_records(recs, prob["lam"])
    keep = np.r_[0:100, 101:300]
    w2, _ = oracle.softmin(r["S"][keep], prob["lam"])
    np.testing.assert_allclose(dU2, np.einsum("k,tkm->tm", w2, r["delta"][:, keep, :]).ravel(),
                               rtol=1e-10, atol=1e-13)
