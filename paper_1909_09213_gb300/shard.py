"""Host-side sharding of the search across ranks (one process per GPU).

Two ways to share work, neither with a collective on the data path:

* independent problems (batches, or one copy of a problem per rank): every rank solves its
  own units and the ranks only meet to combine statistics;
* one search tree (search-space partitioning): every rank propagates the root and explores
  the root children dealt to it round-robin (csp_set_partition); summing the ranks' counts
  and hash sums, and xoring their hash xors, gives the undivided search.

The single exchange is `combine_across_ranks`: an all-gather of a few 64-bit integers at the
end of the search.
"""
from __future__ import annotations

M64 = (1 << 64) - 1
FIELDS = ("nodes", "fails", "solutions", "sol_hash_sum", "sol_hash_xor")


def partition(rank: int, world: int):
    """(part, nparts) of this rank when one tree is shared by `world` ranks."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    return rank, world


def units_of(rank: int, world: int, count: int):
    """Indices of `count` independent units dealt round-robin to `rank`."""
    return list(range(rank, count, world))


def combine(parts):
    """Combine per-rank statistics (dicts with FIELDS): sums, hash sum mod 2^64, xor."""
    out = {"nodes": 0, "fails": 0, "solutions": 0, "sol_hash_sum": 0, "sol_hash_xor": 0}
    for p in parts:
        out["nodes"] += int(p["nodes"])
        out["fails"] += int(p["fails"])
        out["solutions"] += int(p["solutions"])
        out["sol_hash_sum"] = (out["sol_hash_sum"] + int(p["sol_hash_sum"])) & M64
        out["sol_hash_xor"] ^= int(p["sol_hash_xor"]) & M64
    return out


def _to_i64(v: int) -> int:
    v &= M64
    return v - (1 << 64) if v >= (1 << 63) else v


def combine_across_ranks(stats: dict, device="cpu"):
    """All-gather this rank's statistics and combine them (every rank gets the result).
    Works with gloo (CPU tensors) and nccl (device tensors)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size()
    mine = torch.tensor([_to_i64(int(stats[f])) for f in FIELDS], dtype=torch.int64, device=device)
    bufs = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(bufs, mine)
    parts = [{f: int(b[i].item()) & M64 for i, f in enumerate(FIELDS)} for b in bufs]
    return combine(parts)
