"""Oracle for the large neighbourhood search rounds (test infrastructure only).

Section 4 (first direction) describes the method: after a solution is found, copies of the
problem with some domains reset are searched for a better solution.  What a round must
compute has a plain definition, written out here on the oracle's own model objects:

* the neighbourhood of incumbent a under reset set R and bound f* - 1 is the problem with
  D(x) = {a(x)} for every x outside R, plus the row  sum_i c_i x_i <= f* - 1;
* its verdict is whether that problem has a solution (the oracle's exhaustive search);
* the optimum of  min sum_i c_i x_i  over the solutions is found by bound tightening: any
  solution gives an upper bound f, and the search under  objective <= f - 1  either finds a
  better one or proves f optimal.  Each step is an exact oracle search.

Nothing here is shared with the library's LNS driver; both sides take the reset sets from
the seeded generator (instances.relax_masks).
"""
from __future__ import annotations

import copy

from . import oracle as O


def objective(obj, values) -> int:
    coefs, vars_ = obj
    return int(sum(int(c) * int(values[v]) for c, v in zip(coefs, vars_)))


def neighbourhood_model(model, incumbent, reset, obj, bound):
    """The problem restricted to the neighbourhood: a CspModel (plain copy of `model`)."""
    m = copy.deepcopy(model)
    for x in range(model.n):
        if not reset[x]:
            keep = int(incumbent[x])
            for v in range(int(model.lo[x]), int(model.hi[x]) + 1):
                if v != keep:
                    m.removed.append((x, v))
    m.lin.append((list(obj[0]), list(obj[1]), int(bound)))
    return m


def verdict(model, node_limit: int = 0) -> int:
    """1 SAT, 0 UNSAT, -5 undecided within node_limit (oracle first-solution search)."""
    r = O.solve(O.OracleModel(model), mode=1, cap=1, variant=1, node_limit=node_limit)
    return int(r.status)


def optimum(model, obj):
    """(optimal value, a solution reaching it), or (None, None) when there is no solution."""
    best, sol = None, None
    cur = model
    while True:
        r = O.solve(O.OracleModel(cur), mode=1, cap=1, variant=1)
        if r.status != 1:
            return best, sol
        sol = r.sols[0].copy()
        best = objective(obj, sol)
        cur = copy.deepcopy(model)
        cur.lin.append((list(obj[0]), list(obj[1]), best - 1))


def brute_force_optimum(model, obj, cap: int = 1 << 20):
    """Minimum over every solution, enumerated from the full product of domains (tiny models
    only; the oracle's brute force, no propagation)."""
    cnt, _, _, sols = O.brute_force(O.OracleModel(model), cap=cap)
    assert cnt <= cap, "model too large for enumeration"
    if cnt == 0:
        return None
    return min(objective(obj, s) for s in sols)
