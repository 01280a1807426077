"""Autotuner for the search and propagation kernels' launch shapes.

The occupancy trade of Section 2.3 (fewer threads per SM when the data cached in shared
memory grows) becomes a measured choice: warps per block (workers sharing one instance's
staged constraints and one work queue), search levels kept in shared memory per worker, and
queue capacity.  Candidates are timed on a calibration subset with CUDA events (the
library's own launch timing); the fastest is cached in a JSON file keyed by GPU, domain
width and a size bucket.  For one problem's search the axes are warps per block, threads
per node (two sibling nodes per warp or one) and the bitset width (the problem's own or
wider); for propagation alone the number of threads per node: a warp per domain state, or
a whole block per state (tune_propagate).  A tiling changes only speed, never results.
"""
from __future__ import annotations

import json
import os

from . import cubics as K

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "tune_cache.json")


def _gpu_name():
    import torch
    return torch.cuda.get_device_name()


def size_bucket(models) -> str:
    n = max(m.n for m in models)
    span = max(max(m.hi) - min(m.lo) + 1 for m in models)
    w = 1 if span <= 32 else 2 if span <= 64 else 4 if span <= 128 else 8
    nb = 1 << max(0, (n - 1).bit_length())
    kinds = "".join(k for k, attr in (("n", "ne"), ("l", "lin"), ("a", "alldiff"), ("t", "tables"))
                    if any(getattr(m, attr) for m in models))
    return f"W{w}-n{nb}-{kinds}"


def _load():
    try:
        return json.load(open(CACHE))
    except (OSError, ValueError):
        return {}


def _store(cache):
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


BATCH_CANDIDATES = [
    dict(warps_per_block=w, smem_levels=l)
    for w in (1, 2, 4, 8) for l in (8, 24)
]
def single_candidates(model):
    """Warps per block x threads per node (16: two sibling nodes per warp, where the problem
    allows it; 32: one node per warp) x bitset width (the problem's own, and twice that)."""
    W = K.Csp(model).layout()[1]
    widths = [0] + ([2 * W] if 2 * W <= 8 else [])
    return [dict(warps_per_block=w, threads_per_node=t, domain_words=dw)
            for w in (4, 8, 16) for t in (16, 32) for dw in widths]


def tune_batch(models, mode=K.CSP_FIRST, calib=256, reps=2, use_cache=True, verbose=False):
    """Best csp_tiling for a batch like `models`, timed on its first `calib` instances."""
    key = f"{_gpu_name()}|batch|{mode}|{size_bucket(models)}"
    cache = _load() if use_cache else {}
    if key in cache:
        return K.tiling(**cache[key]["tiling"]), cache[key]
    sub = [K.Csp(m) for m in models[:calib]]
    results = []
    for cand in BATCH_CANDIDATES:
        b = K.Batch(sub)
        b.set_tiling(K.tiling(**cand))
        try:
            b.bind(mode)
        except K.CspError:
            continue
        best = None
        for _ in range(reps + 1):
            rc, _ = b.solve(mode, bind=False)
            ms = b.stats()["ms"]
            best = ms if best is None else min(best, ms)
        results.append((best, cand))
        if verbose:
            print(f"tune batch {cand}: {best:.2f} ms", flush=True)
    best_ms, best = min(results, key=lambda r: r[0])
    entry = {"tiling": best, "ms": best_ms, "calib": len(sub),
             "candidates": [[r[0], r[1]] for r in results]}
    if use_cache:
        cache[key] = entry
        _store(cache)
    return K.tiling(**best), entry


def tune_single(model, mode=K.CSP_ALL, reps=2, use_cache=True, verbose=False):
    """Best csp_tiling for one problem, timed on the problem itself (the search's device
    time); shapes the problem does not admit (CSP_EINVAL) are skipped."""
    key = f"{_gpu_name()}|single|{mode}|{size_bucket([model])}|{model.name}"
    cache = _load() if use_cache else {}
    if key in cache:
        return K.tiling(**cache[key]["tiling"]), cache[key]
    results = []
    for cand in single_candidates(model):
        p = K.Csp(model)
        p.set_tiling(K.tiling(**cand))
        best = None
        try:
            for _ in range(reps + 1):
                rc, st, _ = p.solve(mode, 0)
                best = st["ms"] if best is None else min(best, st["ms"])
        except K.CspError:
            continue
        results.append((best, cand))
        if verbose:
            print(f"tune single {cand}: {best:.2f} ms", flush=True)
    best_ms, best = min(results, key=lambda r: r[0])
    entry = {"tiling": best, "ms": best_ms, "candidates": [[r[0], r[1]] for r in results]}
    if use_cache:
        cache[key] = entry
        _store(cache)
    return K.tiling(**best), entry


PROPAGATE_CANDIDATES = [dict(threads_per_node=t) for t in (32, 64, 128, 256, 512, 1024)]


def tune_propagate(model, states, reps=2, use_cache=True, verbose=False):
    """Threads per node for csp_propagate on states like `states` ((count, n*W) uint32): a
    warp per state, or a block of 64..1024 threads per state with the constraints shared out
    among its warps; each candidate timed on the states themselves (the kernel's device time
    that csp_propagate reports).  A choice of speed only: every candidate reaches the same
    fixpoints."""
    key = f"{_gpu_name()}|propagate|{size_bucket([model])}|{model.name}|{len(states)}"
    cache = _load() if use_cache else {}
    if key in cache:
        return K.tiling(**cache[key]["tiling"]), cache[key]
    results = []
    for cand in PROPAGATE_CANDIDATES:
        p = K.Csp(model)
        p.set_tiling(K.tiling(**cand))
        best = None
        try:
            for _ in range(reps + 1):
                p.propagate(states)
                ms = p.stats()["ms"]
                best = ms if best is None else min(best, ms)
        except K.CspError:
            continue
        results.append((best, cand))
        if verbose:
            print(f"tune propagate {cand}: {best:.3f} ms", flush=True)
    best_ms, best = min(results, key=lambda r: r[0])
    entry = {"tiling": best, "ms": best_ms, "states": len(states),
             "candidates": [[r[0], r[1]] for r in results]}
    if use_cache:
        cache[key] = entry
        _store(cache)
    return K.tiling(**best), entry
