"""Parallel large neighbourhood search over the batched search (Section 4, first direction).

Once a solution is known, the paper proposes to search many copies of the problem at once,
each with a different random subset of domains reset, and to share the intermediate
solutions so that no copy looks for a worse one.  Here one round is one batched launch:

* copy j of the round keeps the variables of its neighbourhood (a random subset) at their
  root domains and fixes every other variable to the incumbent's value: the copies of a
  round share one encoding of the model and differ only in their root domains
  (csp_batch_create_roots; `neighbourhood` builds one copy as a problem of its own);
* every copy carries the bound  sum_i c_i x_i <= f* - 1  (f* the incumbent's objective), an
  int_lin_le row, so it can only return a better solution;
* all copies are searched in one persistent launch (first solution each, a node limit per
  copy); the best solution of the round becomes the incumbent of the next round, on every
  rank when several take part (`share_best`).

The neighbourhood size grows when a round brings no improvement; a copy whose neighbourhood
is the whole problem and which is proved infeasible (status UNSAT, not undecided) proves the
incumbent optimal, and the search stops.

Every search step runs in the library's kernels; this module draws the neighbourhoods,
builds the copies through the C ABI and keeps the incumbent.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import cubics as K
from . import instances as I


def objective_value(obj, sol) -> int:
    coefs, vars_ = obj
    s = np.asarray(sol, dtype=np.int64)
    return int(sum(int(a) * int(s[v]) for a, v in zip(coefs, vars_)))


def neighbourhood(base: K.Csp, incumbent, mask, obj, bound: int) -> K.Csp:
    """Copy of `base`: variables outside `mask` fixed to the incumbent, objective <= bound."""
    c = base.clone()
    fixed = np.nonzero(~np.asarray(mask, dtype=bool))[0]
    if fixed.size:
        c.fix_values(fixed, np.asarray(incumbent, dtype=np.int64)[fixed])
    c.post_lin(obj[0], obj[1], bound)
    return c


def neighbourhood_roots(root, lo0: int, incumbent, masks) -> np.ndarray:
    """Root domains of the copies: (copies, n, W) words; variable x of copy j keeps its root
    domain where masks[j, x], else the single value incumbent[x]."""
    root = np.asarray(root, dtype=np.uint32)
    n, W = root.shape
    b = np.asarray(incumbent, dtype=np.int64) - lo0
    single = np.zeros((n, W), dtype=np.uint32)
    single[np.arange(n), b // 32] = (np.uint32(1) << (b % 32).astype(np.uint32))
    return np.where(np.asarray(masks, dtype=bool)[:, :, None], root[None], single[None])


def share_best(value, sol):
    """Across torch.distributed ranks (if initialised): the best (lowest value) incumbent,
    ties to the lowest rank; every rank returns the same pair.  value None = no solution."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value, sol
    allv = [None] * dist.get_world_size()
    dist.all_gather_object(allv, (value, None if sol is None else [int(v) for v in sol]))
    best = None
    for r, (v, s) in enumerate(allv):
        if v is not None and (best is None or v < best[0]):
            best = (v, s)
    if best is None:
        return None, None
    return best[0], np.asarray(best[1], dtype=np.int32)


@dataclass
class RoundResult:
    round: int
    frac: float
    copies: int
    sat: int
    unsat: int
    undecided: int
    nodes: int
    kernel_ms: float
    wall_ms: float
    best: int | None
    improved: bool
    proved_optimal: bool


@dataclass
class LNSResult:
    best: int | None
    solution: np.ndarray | None
    optimal: bool
    rounds: list = field(default_factory=list)
    initial: int | None = None
    nodes: int = 0
    kernel_ms: float = 0.0
    wall_ms: float = 0.0


class LNS:
    """Minimise sum c_i x_i over the solutions of `model` by parallel LNS.

    copies: neighbourhoods per round (one batched launch); frac: initial share of variables
    reset; grow: factor applied to frac after a round without improvement (capped at 1);
    node_limit: nodes per copy; seed: neighbourhood draws (instances.relax_masks, offset by
    the rank so that ranks search different neighbourhoods); share: exchange the incumbent
    with the other torch.distributed ranks after every round (every rank must then run the
    same number of rounds); False keeps the search on this rank.  always_reset: variables
    every neighbourhood resets (an objective variable, variables defined by others): fixing
    them to the incumbent would leave no better solution in any neighbourhood."""

    def __init__(self, model, obj, copies: int = 256, frac: float = 0.2, grow: float = 1.5,
                 node_limit: int = 20_000, seed: int = 1, tiling: K.csp_tiling | None = None,
                 stream=None, rank: int = 0, share: bool = True, always_reset=()):
        self.model, self.obj = model, obj
        self.always_reset = np.asarray(list(always_reset), dtype=np.int64)
        self.copies, self.frac, self.grow = copies, frac, grow
        self.node_limit, self.seed, self.rank, self.share = node_limit, seed, rank, share
        self.tiling, self.stream = tiling, stream
        self.base = K.Csp(model)
        self.incumbent = None
        self.value = None

    def initial(self):
        """First solution of the plain problem (csp_solve, first solution)."""
        rc, st, sols = self.base.solve(K.CSP_FIRST, 1)
        if rc != 0 or st["solutions"] == 0:
            return None
        self.incumbent = np.asarray(sols[0], dtype=np.int32)
        self.value = objective_value(self.obj, self.incumbent)
        return self.value

    def round(self, r: int, proof_time_ns: int = 0) -> RoundResult:
        """One batched launch over `copies` neighbourhoods.  Once every variable is reset
        (frac = 1) the round is one copy, the whole problem under the bound, searched without
        a node limit (within proof_time_ns, 0 = none; run() gives 60 s without a budget): its
        UNSAT proves optimality."""
        t0 = time.perf_counter()
        n = self.model.n
        if self.frac >= 1.0:
            masks = np.ones((1, n), dtype=bool)
            lim = K.limits(time_limit_ns=proof_time_ns)
        else:
            masks = I.relax_masks(n, self.copies, self.frac, r, self.seed + 7919 * self.rank)
            if self.always_reset.size:
                masks[:, self.always_reset] = True
            lim = K.limits(node_limit=self.node_limit)
        # the model under the bound, encoded once; the copies differ in their root domains
        bounded = self.base.clone()
        bounded.post_lin(self.obj[0], self.obj[1], self.value - 1)
        _, _, lo0 = bounded.layout()
        b = K.Batch.from_roots(bounded, neighbourhood_roots(bounded.root_domains(), lo0,
                                                            self.incumbent, masks))
        if self.tiling is not None:
            b.set_tiling(self.tiling)
        if self.stream is not None:
            b.stream = self.stream
        rc, res = b.solve(K.CSP_FIRST, lim)
        st = b.stats()
        best_v, best_s = None, None
        proved = False
        full = masks.all(axis=1)
        for j, rj in enumerate(res):
            if rj["status"] == 1:
                v = objective_value(self.obj, rj["solution"])
                if best_v is None or v < best_v:
                    best_v, best_s = v, np.array(rj["solution"], dtype=np.int32)
            elif rj["status"] == 0 and full[j]:
                proved = True           # no solution better than the incumbent exists at all
        if self.share:
            best_v, best_s = share_best(best_v, best_s)
        improved = best_v is not None and best_v < self.value
        if improved:
            self.value, self.incumbent = best_v, best_s
            proved = False              # the proof was for the previous bound
        else:
            self.frac = min(1.0, self.frac * self.grow)
        if self.share:
            proved = _all_ranks(proved)
        sat = sum(x["status"] == 1 for x in res)
        unsat = sum(x["status"] == 0 for x in res)
        return RoundResult(r, float(masks.mean()), len(res), sat, unsat, len(res) - sat - unsat,
                           int(sum(x["nodes"] for x in res)), float(st["ms"]),
                           1e3 * (time.perf_counter() - t0), self.value, improved, proved)

    def run(self, rounds: int = 50, time_budget_s: float | None = None) -> LNSResult:
        t0 = time.perf_counter()
        v0 = self.initial()
        out = LNSResult(best=v0, solution=self.incumbent, optimal=False, initial=v0)
        if v0 is None:
            return out
        for r in range(rounds):
            left = None if time_budget_s is None else time_budget_s - (time.perf_counter() - t0)
            rr = self.round(r, int(max(left, 0.1) * 1e9) if left is not None else 60_000_000_000)
            out.rounds.append(rr)
            out.nodes += rr.nodes
            out.kernel_ms += rr.kernel_ms
            if rr.proved_optimal:
                out.optimal = True
                break
            if time_budget_s is not None and time.perf_counter() - t0 > time_budget_s:
                break
        out.best, out.solution = self.value, self.incumbent
        out.wall_ms = 1e3 * (time.perf_counter() - t0)
        return out


def _all_ranks(flag: bool) -> bool:
    """True on every rank if it is true on some rank (a proof on one rank holds for all)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return flag
    allf = [None] * dist.get_world_size()
    dist.all_gather_object(allf, bool(flag))
    return any(allf)
