"""Node-sharded iterations over several GPUs (one process per GPU).

The sampled nodes of one sweep are independent (Algorithm 1, Step 2), so one
batch of instances can be spread over ranks: every rank holds the same plan and
nodal values, samples its share of the round's (time node, spatial node) pairs
(spmc_iterate_shard), and the per-pair eps are exchanged once per iteration by
an all-reduce of zero-filled buffers (each entry is written by exactly one rank,
so the sum is exact) before every rank applies them (spmc_apply_eps) and
reconstructs redundantly.  The shares are those of the library: pair i belongs
to the rank r with floor(n r / W) <= i < floor(n (r + 1) / W).
"""
from __future__ import annotations

from typing import Tuple


def shard_range(n_pairs: int, rank: int, world: int) -> Tuple[int, int]:
    """The pairs [lo, hi) that rank `rank` of `world` samples."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world")
    return n_pairs * rank // world, n_pairs * (rank + 1) // world


def assemble(eps_local, group=None):
    """Sum the ranks' zero-filled eps buffers in place (every pair is written by
    one rank only, so the result is exact); a no-op on one rank."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(eps_local, op=dist.ReduceOp.SUM, group=group)
    return eps_local


def iterate_sharded(plan, interval: int, n_iter: int = 1, group=None) -> float:
    """n_iter iterations of `interval`, each sampled across the ranks of `group`
    and exchanged by one all-reduce; returns the last max |eps|."""
    import torch
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        rank, world = dist.get_rank(group), dist.get_world_size(group)
    else:
        rank, world = 0, 1
    n = plan.round_nodes(interval)
    mx = 0.0
    for _ in range(n_iter):
        eps = torch.zeros(n, dtype=torch.float64, device="cuda")
        plan.iterate_shard(interval, rank, world, eps)
        assemble(eps, group)
        mx = plan.apply_eps(interval, eps)
    return mx
