"""Host-side sharding of the search across ranks (one process per GPU).

Two ways to share work, neither with a collective on the data path:

* independent problems (batches, or one copy of a problem per rank): every rank solves its
  own units and the ranks only meet to combine statistics;
* one search tree (search-space partitioning, Section 1.3): the tree is cut at depth k
  (`split_units`): every rank expands the first k levels of the first-fail tree (one
  device fixpoint call per level) and gets every nparts-th of the nodes at depth k, which it
  solves as one batch of root copies (`solve_part`); rank 0 counts the expanded levels.
  csp_set_partition is the depth-1 case done inside the search kernel.  Summing the ranks'
  counts and hash sums, and xoring their hash xors, gives the undivided search.

The exchanges: `combine_across_ranks`, an all-gather of a few 64-bit integers at the end of
the search; in first-solution mode also `any_rank`, an OR of a "found" flag that the hosts
poll between chunks of units, so that every rank stops once one has a solution.
"""
from __future__ import annotations

import numpy as np

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


# ----------------------------------------------------------------------------- depth-k split

_POP8 = np.array([bin(i).count("1") for i in range(256)], dtype=np.int64)


def _sizes(doms: np.ndarray, n: int, W: int) -> np.ndarray:
    """(count, n) domain sizes of (count, n*W) uint32 bitset states"""
    b = np.ascontiguousarray(doms, dtype=np.uint32).view(np.uint8).reshape(doms.shape[0], n, W * 4)
    return _POP8[b].sum(axis=2)


def split_units(propagate, root: np.ndarray, n: int, W: int, depth: int):
    """Cut the first-fail search tree at `depth`.  Levels 0 .. depth-1 are expanded breadth
    first: each level's nodes go through `propagate` ((count, n*W) uint32 states ->
    (states, failed)) in one call, and every node that is neither failed nor fully fixed
    branches on its first-fail variable (fewest values, lowest index), values ascending.

    Returns (units, nodes, fails): units is a (count, n*W) uint32 array of the children at
    `depth` (not propagated yet) and of the fully fixed nodes met above it (solutions, which
    the rank that gets them records), in depth-first order within each level; nodes and
    fails count the expanded levels' branching and failed nodes (the fully fixed ones count
    when their unit is solved).  Every rank computes the same units."""
    level = np.asarray(root, dtype=np.uint32).reshape(1, n * W)
    units, nodes, fails = [], 0, 0
    for _ in range(depth):
        if level.shape[0] == 0:
            break
        out, failed = propagate(level)
        out = np.asarray(out, dtype=np.uint32).reshape(-1, n * W)
        sizes = _sizes(out, n, W)
        children = []
        for k in range(out.shape[0]):
            if failed[k]:
                nodes += 1
                fails += 1
                continue
            unfixed = np.flatnonzero(sizes[k] > 1)
            if unfixed.size == 0:
                units.append(out[k])
                continue
            nodes += 1
            x = int(unfixed[np.argmin(sizes[k][unfixed])])       # ties: lowest index
            words = out[k, x * W:(x + 1) * W]
            for w in range(W):
                m = int(words[w])
                while m:
                    bit = m & -m
                    m ^= bit
                    child = out[k].copy()
                    child[x * W:(x + 1) * W] = 0
                    child[x * W + w] = bit
                    children.append(child)
        level = np.array(children, dtype=np.uint32).reshape(-1, n * W)
    units.extend(level)
    return np.array(units, dtype=np.uint32).reshape(-1, n * W), nodes, fails


def any_rank(flag: bool, device="cpu") -> bool:
    """OR of a flag over all ranks (one all-reduce of one integer)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([1 if flag else 0], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return bool(t.item())


def first_over_ranks(units, part: int, nparts: int, solve_chunk, or_ranks, chunk: int):
    """First-solution search over a shared tree: this rank's units (every nparts-th) in chunks
    of `chunk`; after each chunk the ranks OR their "found" flags (or_ranks), and every rank
    stops once one has a solution.  Every rank makes the same number of or_ranks calls.
    solve_chunk(units) -> (found, solution or None, stats dict).  Returns (found anywhere,
    this rank's solution or None, this rank's summed stats, chunks run)."""
    mine = units[part::nparts]
    per_rank = -(-len(units) // nparts)
    rounds = -(-per_rank // chunk) if per_rank else 0
    stats = {f: 0 for f in FIELDS}
    sol, found_here, ran = None, False, 0
    for c in range(rounds):
        piece = mine[c * chunk:(c + 1) * chunk]
        if len(piece) and not found_here:
            f, s, st = solve_chunk(piece)
            stats = combine([stats, st])
            ran += 1
            if f:
                found_here, sol = True, s
        if or_ranks(found_here):
            return True, sol, stats, ran
    return False, None, stats, ran


def solve_part(p, part: int, nparts: int, depth: int = 3, mode: int = 0, chunk: int = 256,
               or_ranks=None, lim=None, tiling=None):
    """This rank's share of one problem's search (p: a cubics.Csp) cut at `depth`: the units
    are solved as batches of copies of the problem whose root domains are the units
    (csp_batch_create_roots); all solutions (mode 0) or the first over all ranks (mode 1, with
    or_ranks, e.g. any_rank).  Returns this rank's statistics (rank 0 includes the expanded
    levels), to be combined with combine_across_ranks, and in mode 1 (found, solution)."""
    from . import cubics as K
    n, W, _ = p.layout()
    units, nodes, fails = split_units(p.propagate, p.root_domains().ravel(), n, W, depth)
    head = {"nodes": nodes if part == 0 else 0, "fails": fails if part == 0 else 0,
            "solutions": 0, "sol_hash_sum": 0, "sol_hash_xor": 0}

    def run(piece, m):
        b = K.Batch.from_roots(p, piece)
        if tiling is not None:
            b.set_tiling(tiling)
        rc, res = b.solve(m, lim=lim)
        st = b.stats()
        return res, {"nodes": st["nodes"], "fails": st["fails"], "solutions": st["solutions"],
                     "sol_hash_sum": st["sol_hash_sum"], "sol_hash_xor": st["sol_hash_xor"]}

    if mode == K.CSP_ALL:
        mine = units[part::nparts]
        st = run(mine, K.CSP_ALL)[1] if len(mine) else {f: 0 for f in FIELDS}
        out = combine([head, st])
        out["units"], out["units_total"] = len(mine), len(units)
        return out

    def solve_chunk(piece):
        res, st = run(piece, K.CSP_FIRST)
        for r in res:
            if r["status"] == 1:
                return True, r["solution"], st
        return False, None, st

    found, sol, st, ran = first_over_ranks(units, part, nparts, solve_chunk,
                                           or_ranks or (lambda f: f), chunk)
    out = combine([head, st])
    out["units_total"], out["chunks"] = len(units), ran
    return out, (found, sol)
