"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: the worked example of
Section 1.1, the published N-queens counts, splitmix64 reference vectors, brute-force
enumeration of the solution set, and the defining properties of each propagator's fixpoint
(soundness, consistency, maximality, order independence, idempotence).
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_09213_gb300 import instances as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [list(map(int, ln.split())) for ln in f if ln.strip() and not ln.startswith("#")]


# ----------------------------------------------------------------------------- hashing

def test_splitmix64_reference_vectors():
    G, M = 0x9E3779B97F4A7C15, (1 << 64) - 1
    for row in _rows("splitmix64.txt"):
        seed, outs = row[0], row[1:]
        assert [O.splitmix64((seed + k * G) & M) for k in range(len(outs))] == outs


def test_solution_hash_is_the_documented_fold():
    vals = [3, -1, 7, 0]
    h = 0x9E3779B97F4A7C15
    for i, v in enumerate(vals):
        h = O.splitmix64(h ^ ((i << 32) | (v & 0xFFFFFFFF)))
    assert O.solution_hash(vals) == h
    assert O.solution_hash([3, 7]) != O.solution_hash([7, 3])


# ----------------------------------------------------------------------------- worked example

@pytest.mark.parametrize("c1", ["domain", "lin"])
@pytest.mark.parametrize("c2", ["lin", "table"])
def test_worked_example_eleven_solutions(c1, c2):
    expect = sorted(tuple(r) for r in _rows("worked_example.txt"))
    assert len(expect) == 11
    om = O.OracleModel(I.worked_example(c1, c2))
    for variant in (0, 1, 2):
        r = O.solve(om, cap=64, variant=variant)
        assert r.solutions == 11 and r.status == 1
        assert sorted(map(tuple, r.sols.tolist())) == expect
    cnt, hs, hx, sols = O.brute_force(om)
    assert cnt == 11 and sorted(map(tuple, sols.tolist())) == expect
    r = O.solve(om, cap=64)
    assert (r.hash_sum, r.hash_xor) == (hs, hx)


def test_worked_example_root_fixpoint():
    # c1 and c2 alone already fix the bounds: x1 in {4, 5}, x2 in {5..10}
    om = O.OracleModel(I.worked_example("lin", "lin"))
    failed, f = O.propagate(om, om.root_flags())
    assert not failed
    assert om.flags_to_sets(f) == [[4, 5], list(range(5, 11))]


# ----------------------------------------------------------------------------- N-queens

@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7, 8, 9, 10])
def test_queens_counts(N):
    expect = {r[0]: r[1] for r in _rows("queens_counts.txt")}[N]
    om = O.OracleModel(I.queens(N))
    r = O.solve(om)
    assert r.solutions == expect
    assert r.status == (1 if expect else 0)


@pytest.mark.slow
def test_queens_12_count():
    om = O.OracleModel(I.queens(12))
    assert O.solve(om).solutions == 14200


def test_queens_full_size_oracle_rows():
    # the stored full-size oracle searches (N = 14..16, written by the oracle alone) against
    # the published counts, and the shape of a d-way tree: every internal node has at least
    # two children, so leaves (fails + solutions) < nodes < 2 * leaves; 12 bytes per wake
    counts = {r[0]: r[1] for r in _rows("queens_counts.txt")}
    rows = _rows("queens_oracle.txt")
    assert sorted(r[0] for r in rows) == [14, 15, 16]
    for N, nodes, fails, sols, _hs, _hx, evals, work in rows:
        assert sols == counts[N]
        leaves = fails + sols
        assert leaves < nodes < 2 * leaves
        assert work == 12 * evals


def test_queens_model_size():
    for N in (8, 14, 16):
        assert len(I.queens(N).ne) == 3 * N * (N - 1) // 2
    assert len(I.queens(8).ne) == 84


def test_queens_fixpoint_variants_give_same_tree():
    om = O.OracleModel(I.queens(8))
    rs = [O.solve(om, variant=v) for v in (0, 1, 2)]
    assert len({(r.nodes, r.fails, r.solutions, r.hash_sum, r.hash_xor) for r in rs}) == 1


def test_first_mode_stops_at_first_solution():
    om = O.OracleModel(I.queens(8))
    r = O.solve(om, mode=1, cap=1)
    assert r.solutions == 1 and r.status == 1
    allr = O.solve(om, mode=0, cap=100)
    assert tuple(r.sols[0]) == tuple(allr.sols[0])      # DFS order: first found is first listed
    assert O.check_solution(om, r.sols[0])
    assert r.nodes < allr.nodes


def test_node_limit_status():
    om = O.OracleModel(I.queens(8))
    r = O.solve(om, node_limit=10)
    assert r.status == -5 and r.nodes == 10


# ----------------------------------------------------------------------------- brute force

def _tiny_models(count, seed0=0):
    return [I.random_tiny(I.seed_for(I.CFG_TINY, seed0 + i)) for i in range(count)]


def test_search_equals_brute_force_on_tiny_csps():
    models = _tiny_models(2500)
    kinds = {"ne": 0, "lin": 0, "alldiff": 0, "table": 0}
    sat = 0
    for m in models:
        om = O.OracleModel(m)
        cnt, hs, hx, bsols = O.brute_force(om, cap=20000)
        r = O.solve(om, cap=20000, variant=1)
        assert (r.solutions, r.hash_sum, r.hash_xor) == (cnt, hs, hx), m.name
        assert sorted(map(tuple, r.sols.tolist())) == sorted(map(tuple, bsols.tolist())), m.name
        for s in r.sols:
            assert O.check_solution(om, s)
        sat += cnt > 0
        for k in kinds:
            kinds[k] += len(getattr(m, "tables" if k == "table" else k)) > 0
    # the sample exercises every constraint kind and both outcomes
    assert min(kinds.values()) > 300
    assert 200 < sat < len(models) - 200


def test_first_mode_matches_brute_force_status():
    for m in _tiny_models(600, 10000):
        om = O.OracleModel(m)
        cnt = O.brute_force(om, cap=1)[0]
        r = O.solve(om, mode=1, cap=1)
        assert r.status == (1 if cnt else 0)
        if cnt:
            assert O.check_solution(om, r.sols[0])


# ----------------------------------------------------------------------------- fixpoint properties

def _random_subdomain(om, rng, p_keep=0.7):
    f = om.root_flags().copy()
    keep = rng.random(f.shape[0]) < p_keep
    return (f & keep).astype(np.uint8)


def test_propagation_is_sound():
    """Root fixpoint never removes a value used by a brute-force solution."""
    for m in _tiny_models(800, 20000):
        om = O.OracleModel(m)
        cnt, _, _, sols = O.brute_force(om, cap=20000)
        failed, f = O.propagate(om, om.root_flags(), variant=1)
        if cnt:
            assert not failed
            sets = om.flags_to_sets(f)
            for s in sols:
                for i, v in enumerate(s):
                    assert v in sets[i]


def test_fixpoint_variants_agree_and_are_idempotent():
    rng = np.random.default_rng(7)
    n_fail = 0
    for m in _tiny_models(800, 30000):
        om = O.OracleModel(m)
        for _ in range(3):
            d = _random_subdomain(om, rng)
            outs = [O.propagate(om, d, variant=v, seed=s) for v, s in ((0, 1), (1, 1), (2, 3), (2, 99))]
            fails = {o[0] for o in outs}
            assert len(fails) == 1
            if outs[0][0]:
                n_fail += 1
                continue
            for o in outs[1:]:
                assert np.array_equal(o[1], outs[0][1])
            again = O.propagate(om, outs[0][1], variant=0)
            assert not again[0] and np.array_equal(again[1], outs[0][1])
    assert n_fail > 50


def _sets_model(m, sets):
    """flags for explicit per-variable value sets"""
    om = O.OracleModel(m)
    f = np.zeros(int(om.off[-1]), np.uint8)
    for i, s in enumerate(sets):
        for v in s:
            f[om.off[i] + v - om.lo[i]] = 1
    return om, f


def _min_term(a, dom):
    return min(a * u for u in dom)


def test_lin_single_row_fixpoint_is_bounds_consistent_and_greatest():
    """For one row sum a_i x_i <= b, the fixpoint D* must satisfy, for every i,
    D*_i = {v in D_i : a_i v + sum_{j != i} min_{u in D*_j} a_j u <= b}  (bounds support),
    and D* must contain every value of every solution (greatest)."""
    rng = np.random.default_rng(11)
    checked = 0
    for t in range(1500):
        k = int(rng.integers(1, 5))
        n = k
        lo = [int(x) for x in rng.integers(-4, 3, n)]
        hi = [lo[i] + int(rng.integers(0, 7)) for i in range(n)]
        coefs = [int(c) for c in rng.choice([-4, -3, -2, -1, 1, 2, 3, 4], k)]
        vars_ = list(range(k))
        mid = sum(a * (lo[v] + hi[v]) // 2 for a, v in zip(coefs, vars_))
        b = mid + int(rng.integers(-6, 4))
        m = I.CspModel(n=n, lo=lo, hi=hi, lin=[(coefs, vars_, b)])
        om = O.OracleModel(m)
        d = _random_subdomain(om, rng, 0.8)
        failed, f = O.propagate(om, d)
        before = om.flags_to_sets(d)
        sols = [s for s in __import__("itertools").product(*before)
                if sum(a * s[v] for a, v in zip(coefs, vars_)) <= b]
        if failed:
            assert not sols
            continue
        after = om.flags_to_sets(f)
        for i in range(n):
            others = sum(_min_term(coefs[j], after[j]) for j in range(n) if j != i)
            expect = [v for v in before[i] if coefs[i] * v + others <= b]
            assert after[i] == expect, (coefs, b, before, after)
        for s in sols:
            assert all(s[i] in after[i] for i in range(n))
        checked += 1
    assert checked > 500


def test_lin_one_term_is_unary_bound():
    """a x <= b keeps exactly the values v of D with a*v <= b (textbook unary bound)."""
    for a in (-7, -3, -1, 1, 2, 5):
        for b in range(-12, 13):
            m = I.CspModel(n=1, lo=[-6], hi=[6], lin=[([a], [0], b)])
            om = O.OracleModel(m)
            failed, f = O.propagate(om, om.root_flags())
            expect = [v for v in range(-6, 7) if a * v <= b]
            assert failed == (not expect)
            if expect:
                assert om.flags_to_sets(f)[0] == expect


def test_lin_merges_repeated_variables():
    # x + x <= 3 is 2x <= 3, so x <= 1; unmerged reasoning would only give x <= 3 - min = 3
    m = I.CspModel(n=1, lo=[0], hi=[5], lin=[([1, 1], [0, 0], 3)])
    om = O.OracleModel(m)
    failed, f = O.propagate(om, om.root_flags())
    assert not failed and om.flags_to_sets(f)[0] == [0, 1]
    # x - x <= -1 is 0 <= -1: unsatisfiable
    m = I.CspModel(n=1, lo=[0], hi=[5], lin=[([1, -1], [0, 0], -1)])
    om = O.OracleModel(m)
    assert O.propagate(om, om.root_flags())[0]
    assert O.solve(om).status == 0


def test_table_fixpoint_is_arc_consistent_and_greatest():
    rng = np.random.default_rng(5)
    for t in range(600):
        sx, sy = int(rng.integers(1, 7)), int(rng.integers(1, 7))
        al = rng.random((sx, sy)) < rng.uniform(0.1, 0.9)
        m = I.CspModel(n=2, lo=[0, 2], hi=[sx - 1, sy + 1], tables=[(0, 1, al)])
        om = O.OracleModel(m)
        d = _random_subdomain(om, rng, 0.8)
        before = om.flags_to_sets(d)
        failed, f = O.propagate(om, d)
        sup_x = [a for a in before[0] if any(al[a, b - 2] for b in before[1])]
        sup_y = [b for b in before[1] if any(al[a, b - 2] for a in before[0])]
        if failed:
            assert not any(al[a, b - 2] for a in before[0] for b in before[1])
            continue
        after = om.flags_to_sets(f)
        assert after[0] == [a for a in before[0] if any(al[a, b - 2] for b in after[1])]
        assert after[1] == [b for b in before[1] if any(al[a, b - 2] for a in after[0])]
        # one binary constraint: AC after one revision of each side is already the fixpoint
        assert after[0] == sup_x and after[1] == sup_y


def test_table_full_matrix_is_noop():
    rng = np.random.default_rng(3)
    for t in range(200):
        m = I.CspModel(n=2, lo=[0, 0], hi=[4, 6], tables=[(0, 1, np.ones((5, 7), bool))])
        om = O.OracleModel(m)
        d = _random_subdomain(om, rng, 0.6)
        failed, f = O.propagate(om, d)
        empty = any(len(s) == 0 for s in om.flags_to_sets(d))
        assert failed == empty
        if not failed:
            assert np.array_equal(f, d)


def test_alldiff_of_two_equals_ne():
    rng = np.random.default_rng(9)
    for t in range(600):
        lo = [int(x) for x in rng.integers(-2, 2, 2)]
        hi = [lo[i] + int(rng.integers(0, 4)) for i in range(2)]
        ma = I.CspModel(n=2, lo=lo, hi=hi, alldiff=[[0, 1]])
        mn = I.CspModel(n=2, lo=lo, hi=hi, ne=[(0, 1, 0)])
        oa, on = O.OracleModel(ma), O.OracleModel(mn)
        d = _random_subdomain(oa, rng, 0.7)
        fa, da = O.propagate(oa, d)
        fn, dn = O.propagate(on, d)
        assert fa == fn
        if not fa:
            assert np.array_equal(da, dn)


def test_alldiff_pigeonhole_and_elimination():
    # three variables over two values cannot be pairwise distinct (pigeonhole)
    m = I.CspModel(n=3, lo=[0, 0, 0], hi=[1, 1, 1], alldiff=[[0, 1, 2]])
    om = O.OracleModel(m)
    assert O.propagate(om, om.root_flags())[0]
    # x0 = 2 removes 2 from the others but leaves the rest
    m = I.CspModel(n=3, lo=[2, 0, 0], hi=[2, 3, 3], alldiff=[[0, 1, 2]])
    om = O.OracleModel(m)
    failed, f = O.propagate(om, om.root_flags())
    assert not failed and om.flags_to_sets(f) == [[2], [0, 1, 3], [0, 1, 3]]


def test_ne_fixpoint_definition():
    rng = np.random.default_rng(13)
    for t in range(600):
        c = int(rng.integers(-3, 4))
        m = I.CspModel(n=2, lo=[0, 0], hi=[5, 5], ne=[(0, 1, c)])
        om = O.OracleModel(m)
        d = _random_subdomain(om, rng, 0.4)
        before = om.flags_to_sets(d)
        failed, f = O.propagate(om, d)
        x, y = list(before[0]), list(before[1])
        # apply the definition until nothing changes
        while True:
            nx = [v for v in x if not (len(y) == 1 and v == y[0] + c)]
            ny = [v for v in y if not (len(nx) == 1 and v == nx[0] - c)]
            if (nx, ny) == (x, y):
                break
            x, y = nx, ny
        assert failed == (not x or not y)
        if not failed:
            assert om.flags_to_sets(f) == [x, y]


def test_unary_ne():
    m = I.CspModel(n=1, lo=[0], hi=[3], ne=[(0, -1, 2)])
    om = O.OracleModel(m)
    assert om.flags_to_sets(O.propagate(om, om.root_flags())[1]) == [[0, 1, 3]]


def test_work_bytes_counts_ne_wakes():
    om = O.OracleModel(I.queens(6))
    r = O.solve(om, variant=1, W=1)
    assert r.work_bytes == 12.0 * r.evals[0]


# Hand-traced FIFO fixpoints of all-solution searches (first-fail, lowest index on ties,
# values ascending).  At the root every propagator is queued once; at a child only those
# over the branched variable; a propagator that changes a domain is queued again (it is in
# the scope of the variable it changed).  Bytes per evaluation, with sizes taken before it:
# int_ne 12; table 4 (|D(x)| + 2) + 4 (|D(y)| + 2); int_lin_le 4 W (2k + changed);
# alldifferent 4 W 2k.

def test_work_bytes_one_ne_by_hand():
    # x, y in {0, 1}, x != y.  Root: 12 (nothing fixed).  x = 0: y loses 0 (12), queued
    # again, nothing left to remove (12); x = 1 the same.  3 nodes, 2 solutions.
    m = I.CspModel(n=2, lo=[0, 0], hi=[1, 1], ne=[(0, 1, 0)])
    r = O.solve(O.OracleModel(m), variant=1, W=1)
    assert (r.nodes, r.solutions) == (3, 2)
    assert r.work_bytes == 12 + 2 * (12 + 12)


def test_work_bytes_one_table_by_hand():
    # x, y in {0, 1, 2} with every pair allowed: no evaluation changes anything.  Root:
    # 4 (3 + 2) + 4 (3 + 2) = 40.  x = v: 4 (1 + 2) + 4 (3 + 2) = 32, then y = w:
    # 4 (1 + 2) + 4 (1 + 2) = 24 for each of 3 values.  13 nodes.
    m = I.CspModel(n=2, lo=[0, 0], hi=[2, 2], tables=[(0, 1, np.ones((3, 3), bool))])
    r = O.solve(O.OracleModel(m), variant=1, W=1)
    assert (r.nodes, r.solutions) == (13, 9)
    assert r.work_bytes == 40 + 3 * (32 + 3 * 24)
    # table sizes do not depend on W
    assert O.solve(O.OracleModel(m), variant=1, W=4).work_bytes == r.work_bytes


@pytest.mark.parametrize("W", [1, 2, 8])
def test_work_bytes_one_row_by_hand(W):
    # x, y in {0..3}, x + y <= 3 (k = 2): an evaluation is 4 W (4 + changed).
    # Root: 4W*4 (no change).  x = 0: 16W, then y = 0..3: 4 x 16W.  x = 1: y <= 2 (20W),
    # queued again (16W), then y = 0..2: 3 x 16W.  x = 2: 20W + 16W + 2 x 16W.  x = 3: y <= 0
    # fixes y (20W + 16W): a solution without branching.  14 nodes, 10 solutions.
    m = I.CspModel(n=2, lo=[0, 0], hi=[3, 3], lin=[([1, 1], [0, 1], 3)])
    r = O.solve(O.OracleModel(m), variant=1, W=W)
    assert (r.nodes, r.solutions) == (14, 10)
    assert r.work_bytes == W * (16 + (16 + 64) + (36 + 48) + (36 + 32) + 36)


@pytest.mark.parametrize("W", [1, 4])
def test_work_bytes_one_alldiff_by_hand(W):
    # x, y, z in {0, 1, 2}, all different (k = 3): an evaluation is 4 W 6.  Root: one
    # evaluation.  x = v: v leaves y and z (one evaluation, queued again, a second one);
    # then y (size 2, lowest index) = w: w leaves z (two evaluations again).  10 nodes.
    m = I.CspModel(n=3, lo=[0, 0, 0], hi=[2, 2, 2], alldiff=[[0, 1, 2]])
    r = O.solve(O.OracleModel(m), variant=1, W=W)
    assert (r.nodes, r.solutions) == (10, 6)
    e = 24 * W
    assert r.work_bytes == e + 3 * (2 * e + 2 * (2 * e))


# ----------------------------------------------------------------------------- generators

def test_model_rb_shape():
    p = I.rb_tightness()
    assert abs(p - (1 - math.exp(-0.8 / 0.7))) < 1e-15 and abs(p - 0.681093) < 1e-6
    m = I.model_rb(123, 30, 16)
    assert len(m.tables) == round(0.7 * 30 * math.log(30)) == 71
    for (x, y, al) in m.tables:
        assert x != y and al.shape == (16, 16)
        assert int((~al).sum()) == round(p * 256) == 174
    m = I.model_rb(5, 80, 20)
    assert len(m.tables) == 245 and int((~m.tables[0][2]).sum()) == 272


def test_model_rb_threshold_tightness():
    # at p*, ln E[#solutions] = n ln d + m ln(1 - p*) with m = r n ln n is exactly zero
    for n, d in ((80, 20), (30, 16), (20, 8), (60, 32)):
        p = I.rb_threshold_tightness(n, d)
        assert abs(n * math.log(d) + 0.7 * n * math.log(n) * math.log(1 - p)) < 1e-9
    assert abs(I.rb_threshold_tightness(80, 20) - 0.6234) < 1e-4
    # the learning configuration's evaluation set at the configured p is far above it:
    # ln E = 80 ln 20 + 245 ln(1 - 0.681093) = -40.3
    assert abs(80 * math.log(20) + 245 * math.log(1 - I.rb_tightness()) + 40.3) < 0.1


def test_generators_are_deterministic():
    a, b = I.rb_batch(3), I.rb_batch(3)
    for ma, mb in zip(a, b):
        assert ma.n == mb.n and len(ma.tables) == len(mb.tables)
        assert all(np.array_equal(ta[2], tb[2]) for ta, tb in zip(ma.tables, mb.tables))
    la, lb = I.lin_alldiff(1), I.lin_alldiff(1)
    assert la.lin == lb.lin and la.alldiff == lb.alldiff
    assert sorted(v for g in la.alldiff for v in g) == list(range(200))
