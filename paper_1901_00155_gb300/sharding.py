"""Row sharding across processes, one GPU per process.

The rows of a discord search are independent given the series. Shard k of G
keeps the rows at positions [floor(k N / G), floor((k + 1) N / G)) of the
mean-bucketed visit order (``shard_count`` / ``shard_index`` of the plan
options), and still scans every column. Its result is the discord among its
own rows. The discord of the series is the argmax of (nn distance, -index)
over the shard results (Algorithm 1's total order, with ties going to the
smallest index). So the only exchange is one all-gather of each shard's
(nn distance, index) pair. Each shard's tensor-core rescoring stays local.

``merge`` is the host rule. ``allgather_discord`` exchanges the shard
results over ``torch.distributed``: gloo with CPU tensors, NCCL with CUDA
tensors of the current device.
"""
from __future__ import annotations

from . import DiscordResult, Plan

__all__ = ["merge", "allgather_discord", "find_discord_sharded"]


def merge(results) -> DiscordResult:
    """The series' discord from the shard results: the largest nn_distance,
    ties to the smallest index. Pair and candidate counts are summed, and
    ``exact`` holds only if every shard's result is exact."""
    results = list(results)
    if not results:
        raise ValueError("no shard results")
    best = None
    for r in results:
        if best is None or r.nn_distance > best.nn_distance or (
                r.nn_distance == best.nn_distance and r.index < best.index):
            best = r
    return DiscordResult(best.index, best.nn_distance, all(r.exact for r in results),
                         sum(r.computed_pairs for r in results), sum(r.candidates for r in results))


def allgather_discord(result: DiscordResult, group=None) -> DiscordResult:
    """All-gather every rank's shard result and merge them (same answer on
    every rank). The five fields travel as float64: indices and counts up to
    2^53 are exact."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" \
        else torch.device("cpu")
    mine = torch.tensor([result.nn_distance, float(result.index), 1.0 if result.exact else 0.0,
                         float(result.computed_pairs), float(result.candidates)], dtype=torch.float64, device=dev)
    parts = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(parts, mine, group=group)
    rs = []
    for t in parts:
        v = t.cpu().tolist()
        rs.append(DiscordResult(int(v[1]), float(v[0]), v[2] != 0.0, int(v[3]), int(v[4])))
    return merge(rs)


def find_discord_sharded(T, n: int, precision="fp32", group=None, stream=None, **opts) -> DiscordResult:
    """Every rank searches its shard of the rows of the device series T (the
    whole series, replicated), then the shard results are all-gathered and
    merged."""
    import torch.distributed as dist
    G = dist.get_world_size(group)
    k = dist.get_rank(group)
    with Plan(T.numel(), n, precision, shard_count=G, shard_index=k, **opts) as p:
        local = p.find_discord(T, stream)
    return allgather_discord(local, group)
