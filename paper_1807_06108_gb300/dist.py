"""Multi-process helpers (one process per GPU).

The MPC path shards by problem: every rank solves its own independent
problems (a rank-specific Philox key), so nothing is exchanged in the data
path and the job scales weakly; the only collective is the timing
reduction (barrier, then the maximum of the ranks' elapsed times).

For a single problem split over ranks by rollouts, the update of Eq. 37
needs one exchange: each rank reduces its rollouts k in [k0, k1) to the
partial (rho_g = min S~_k, Z_g = sum exp(-(S~_k - rho_g)/lambda),
N_g = sum exp(-(S~_k - rho_g)/lambda) delta_k); with rho = min_g rho_g the
global sums are Z = sum_g Z_g exp(-(rho_g - rho)/lambda) and likewise N, and
dU = N / Z -- the same shift-invariant log-sum-exp rescaling the update
kernel applies across its chunks.  `combine_partials` and
`allreduce_partials` implement that exchange (T*m + 2 floats per rank).
"""

from __future__ import annotations

import math

import numpy as np


def rank_seed(seed, rank):
    """Philox key of rank `rank`'s problems: the key's high word is offset by
    rank << 8, so ranks draw disjoint random streams."""
    return (int(seed) + (int(rank) << 40)) & 0xFFFFFFFFFFFFFFFF


def shard_range(K, rank, world):
    """Contiguous rollout range [k0, k1) of `rank` out of `world`."""
    base, extra = divmod(int(K), int(world))
    k0 = rank * base + min(rank, extra)
    return k0, k0 + base + (1 if rank < extra else 0)


def partial_from_costs(S, delta, lam):
    """(rho_g, Z_g, N_g) of one shard: S [k], delta [T][k][m] (float64)."""
    S = np.asarray(S, dtype=np.float64)
    finite = np.isfinite(S)
    if not finite.any():
        return math.inf, 0.0, np.zeros(delta.shape[0::2])
    rho = float(S[finite].min())
    e = np.where(finite, np.exp(-(np.where(finite, S, rho) - rho) / lam), 0.0)
    N = np.einsum("k,tkm->tm", e, np.asarray(delta, dtype=np.float64))
    return rho, float(e.sum()), N


def combine_partials(parts, lam):
    """dU = sum_g N_g w_g / sum_g Z_g w_g with w_g = exp(-(rho_g - rho)/lam)."""
    rho = min(p[0] for p in parts)
    if not math.isfinite(rho):
        raise ValueError("every rollout cost is non-finite")
    Z = 0.0
    N = None
    for r, z, n in parts:
        w = math.exp(-(r - rho) / lam) if math.isfinite(r) else 0.0
        Z += z * w
        N = n * w if N is None else N + n * w
    return N / Z, rho, Z


def allreduce_partials(dist, rho_g, Z_g, N_g, lam):
    """The exchange across ranks of a torch.distributed group (any backend):
    one MIN all-reduce of rho_g and one SUM all-reduce of the rescaled
    (Z_g, N_g).  Returns (dU, rho, Z) on every rank."""
    import torch
    t = torch.tensor([rho_g], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MIN)
    rho = float(t.item())
    w = math.exp(-(rho_g - rho) / lam) if math.isfinite(rho_g) else 0.0
    buf = torch.cat([torch.tensor([Z_g * w], dtype=torch.float64),
                     torch.as_tensor(np.asarray(N_g, dtype=np.float64) * w).reshape(-1)])
    dist.all_reduce(buf, op=dist.ReduceOp.SUM)
    Z = float(buf[0].item())
    return (buf[1:].numpy().reshape(np.asarray(N_g).shape) / Z), rho, Z


def max_over_ranks(dist, value, device="cpu"):
    """Maximum of `value` over the ranks of `dist` (or value when dist is None)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
