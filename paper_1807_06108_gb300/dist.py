"""Multi-process helpers (one process per GPU).

Two ways to use several GPUs:

* independent problems: every rank solves its own problems (a rank-specific
  Philox key), so nothing is exchanged in the data path and the job scales
  weakly; the only collective is the timing reduction (barrier, then the
  maximum of the ranks' elapsed times);
* one problem split by rollouts: each rank is a shard context (its
  configuration's K is the shard's rollout count, its rollout offset the
  shard's first rollout, see shard_range) whose mppi_jump_rollout_partial
  writes a partial record (rho_g, Z_g, N_g[T][m]) on the device;
  allgather_records exchanges the records (an all-gather of T*m + 2 floats
  per rank), and every rank applies all of them, in rank order, with
  mppi_jump_apply_partials -- the combination (Eq. 37 over all rollouts)
  runs in the library's kernel, so the ranks keep identical controls.

This module moves data only; all arithmetic of the method is in the library.
"""

from __future__ import annotations


def rank_seed(seed, rank):
    """Philox key of rank `rank`'s problems: the key's high word is offset by
    rank << 8, so ranks draw disjoint random streams."""
    return (int(seed) + (int(rank) << 40)) & 0xFFFFFFFFFFFFFFFF


def shard_range(K, rank, world):
    """Contiguous rollout range [k0, k1) of `rank` out of `world`."""
    base, extra = divmod(int(K), int(world))
    k0 = rank * base + min(rank, extra)
    return k0, k0 + base + (1 if rank < extra else 0)


def allgather_records(dist, record):
    """All-gather of one partial record per rank (a 1-D float32 tensor of
    2 + T*m values, on the device for NCCL, on the host for gloo); returns a
    [world][2 + T*m] tensor in rank order on the same device."""
    import torch
    parts = [torch.empty_like(record) for _ in range(dist.get_world_size())]
    dist.all_gather(parts, record.contiguous())
    return torch.stack(parts)


def max_over_ranks(dist, value, device="cpu"):
    """Maximum of `value` over the ranks of `dist` (or value when dist is None)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
