"""Oracle: bounds-consistent alldifferent (the stronger propagation Section 4 proposes as its
second direction).  The C oracle decides supports by bipartite matching; here the same
closure is recomputed by enumerating the interval relaxation, and checked against closed
forms, brute-force solutions and evaluation order.  The device propagator is checked against
this oracle in tests/test_gpu_alldiff_bc.py."""
import itertools

import pytest

from oracle import oracle as O
from paper_1909_09213_gb300 import instances as I


def _model(lo, hi, removed=(), bc=True, ve=False):
    m = I.CspModel(n=len(lo), lo=list(lo), hi=list(hi), removed=list(removed))
    if bc:
        m.alldiff_bc.append(list(range(len(lo))))
    if ve:
        m.alldiff.append(list(range(len(lo))))
    return m


def _fix(m, variant=1, seed=1):
    om = O.OracleModel(m)
    failed, d = O.propagate(om, om.root_flags(), variant=variant, seed=seed)
    return failed, (None if failed else om.flags_to_sets(d))


@pytest.mark.parametrize("lo,hi,removed,want", [
    ([1, 1, 1], [2, 2, 2], [], None),                                  # pigeonhole on [1, 2]
    ([1, 1, 1], [2, 2, 3], [], [[1, 2], [1, 2], [3]]),                 # Hall interval [1, 2]
    ([2, 2, 1], [3, 3, 4], [], [[2, 3], [2, 3], [1, 2, 3, 4]]),        # bounds only: 2, 3 stay
    ([2, 2, 2], [3, 3, 5], [], [[2, 3], [2, 3], [4, 5]]),
    ([1, 1, 1, 1], [3, 3, 3, 6], [(3, 4)], [[1, 2, 3]] * 3 + [[5, 6]]),  # next bound is a hole
    ([0, 5], [0, 9], [], [[0], [5, 6, 7, 8, 9]]),                      # disjoint: nothing to do
    ([3, 3], [3, 4], [], [[3], [4]]),                                  # k = 2 acts as int_ne
])
def test_closed_forms(lo, hi, removed, want):
    failed, d = _fix(_model(lo, hi, removed))
    assert (failed, d) == (want is None, want)


def _closure_by_enumeration(doms):
    """Remove unsupported bounds until every bound has a support in the interval relaxation
    (supports found by enumerating assignments of the other members)."""
    doms = [sorted(d) for d in doms]
    while True:
        if any(not d for d in doms):
            return None
        changed = False
        for i in range(len(doms)):
            for pick in (0, -1):
                while doms[i]:
                    v = doms[i][pick]
                    others = [range(doms[j][0], doms[j][-1] + 1) for j in range(len(doms)) if j != i]
                    ok = any(len(set(a)) == len(a) and v not in a for a in itertools.product(*others))
                    if ok:
                        break
                    doms[i].remove(v)
                    changed = True
                if not doms[i]:
                    return None
        if not changed:
            return doms


@pytest.mark.parametrize("seed", range(120))
def test_matching_closure_equals_enumeration(seed):
    s = I.Stream(I.seed_for(I.CFG_TINY, 97000 + seed))
    k = s.int(2, 5)
    lo = [int(s.int(0, 4)) for _ in range(k)]
    hi = [lo[i] + int(s.int(0, 4)) for i in range(k)]
    removed = [(i, int(s.int(lo[i], hi[i]))) for i in range(k) if hi[i] > lo[i] and s.int(0, 2) == 0]
    m = _model(lo, hi, removed)
    failed, d = _fix(m)
    om = O.OracleModel(m)
    want = _closure_by_enumeration(om.flags_to_sets(om.root_flags()))
    assert (failed, d) == (want is None, want)


@pytest.mark.parametrize("seed", range(60))
def test_sound_and_order_independent(seed):
    s = I.Stream(I.seed_for(I.CFG_TINY, 98000 + seed))
    k = s.int(2, 6)
    lo = [int(s.int(0, 3)) for _ in range(k)]
    hi = [lo[i] + int(s.int(1, 5)) for i in range(k)]
    m = _model(lo, hi)
    m.lin.append(([1] * k, list(range(k)), int(s.int(k, 4 * k))))   # other constraints too
    results = {v: _fix(m, variant=v, seed=seed + 1) for v in (0, 1, 2)}
    assert results[0] == results[1] == results[2]
    failed, d = results[1]
    cnt, _, _, sols = O.brute_force(O.OracleModel(m), cap=1 << 16)
    if failed:
        assert cnt == 0
    else:
        for sol in sols:                                     # no solution value was removed
            assert all(int(sol[i]) in d[i] for i in range(m.n))


@pytest.mark.parametrize("seed", range(30))
def test_search_keeps_the_solution_set(seed):
    s = I.Stream(I.seed_for(I.CFG_TINY, 99000 + seed))
    k = s.int(3, 6)
    lo = [int(s.int(0, 2)) for _ in range(k)]
    hi = [lo[i] + int(s.int(2, 5)) for i in range(k)]
    plain = _model(lo, hi, bc=False, ve=True)
    both = _model(lo, hi, bc=True, ve=True)
    rp = O.solve(O.OracleModel(plain), variant=1)
    rb = O.solve(O.OracleModel(both), variant=1)
    assert (rb.solutions, rb.hash_sum, rb.hash_xor) == (rp.solutions, rp.hash_sum, rp.hash_xor)


def test_library_accepts_groups_and_validates_them():
    """Host side of csp_post_alldiff_bc: groups are accepted (the device propagator exists);
    repeated or bad variables are CSP_EINVAL, more than 32 members CSP_ETOOBIG."""
    import ctypes as C
    from paper_1909_09213_gb300 import cubics as K
    K.Csp(_model([0, 0], [1, 1]))
    L = K.lib()
    h = C.c_void_p()
    lo = (C.c_int32 * 40)(*([0] * 40))
    hi = (C.c_int32 * 40)(*([50] * 40))
    assert L.csp_create(C.byref(h), 40, lo, hi) == 0
    try:
        assert L.csp_post_alldiff_bc(h, 2, (C.c_int32 * 2)(3, 3)) == K.CSP_EINVAL
        assert L.csp_post_alldiff_bc(h, 2, (C.c_int32 * 2)(3, 40)) == K.CSP_EINVAL
        assert L.csp_post_alldiff_bc(h, 33, (C.c_int32 * 33)(*range(33))) == K.CSP_ETOOBIG
        assert L.csp_post_alldiff_bc(h, 32, (C.c_int32 * 32)(*range(32))) == 0
    finally:
        L.csp_destroy(h)


def _hall_interval_closure(doms):
    """The reasoning planned for the device propagator, written plainly: while some interval
    [a, b] (a a lower, b an upper bound of members) holds as many members' [min, max] as it
    has values, no other member may take a bound inside it (its min moves above b, its max
    below a); more members than values fails.  Holes are kept: a bound moves to the next
    value of the domain."""
    doms = [sorted(d) for d in doms]
    while True:
        if any(not d for d in doms):
            return None
        lo = [d[0] for d in doms]
        hi = [d[-1] for d in doms]
        changed = False
        for a in sorted(set(lo)):
            for b in sorted(set(hi)):
                if b < a:
                    continue
                inside = [i for i in range(len(doms)) if a <= lo[i] and hi[i] <= b]
                if len(inside) > b - a + 1:
                    return None
                if len(inside) < b - a + 1:
                    continue
                for j in range(len(doms)):
                    if j in inside:
                        continue
                    keep = list(doms[j])
                    if a <= lo[j] <= b:                  # the min moves above the interval
                        keep = [v for v in keep if v > b]
                    if a <= hi[j] <= b:                  # the max moves below it
                        keep = [v for v in keep if v < a]
                    if keep != doms[j]:
                        doms[j] = keep
                        changed = True
                        if not keep:
                            return None
                lo = [d[0] if d else None for d in doms]
                hi = [d[-1] if d else None for d in doms]
                if any(d is None for d in lo):
                    return None
        if not changed:
            return doms


@pytest.mark.parametrize("seed", range(300))
def test_hall_interval_reasoning_reaches_the_matching_closure(seed):
    s = I.Stream(I.seed_for(I.CFG_TINY, 96000 + seed))
    k = s.int(2, 6) if seed < 150 else s.int(5, 10)
    w = 5 if seed < 150 else 9
    lo = [int(s.int(0, w)) for _ in range(k)]
    hi = [lo[i] + int(s.int(0, w)) for i in range(k)]
    removed = [(i, int(s.int(lo[i], hi[i]))) for i in range(k) if hi[i] > lo[i] and s.int(0, 2) == 0]
    m = _model(lo, hi, removed)
    failed, d = _fix(m)
    om = O.OracleModel(m)
    want = _hall_interval_closure(om.flags_to_sets(om.root_flags()))
    assert (failed, d) == (want is None, want)
