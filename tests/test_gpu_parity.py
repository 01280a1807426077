"""GPU parity: the CUDA path against the oracle on the same seeded inputs.

Propagation must be bit-exact (same fixpoint domains, same failure flag); search must give
the same solution count, solution-set hash, sorted solution list, node count and fail count
as the oracle's sequential search (the tree is fixed by the per-node fixpoints and the
first-fail rule, so it does not depend on how workers share it).
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_1909_09213_gb300 import cubics as K
from paper_1909_09213_gb300 import instances as I

from _util import bits_to_flags, flags_to_bits, random_subdomains, sorted_rows

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def queens_count(N):
    for ln in open(os.path.join(GOLDEN, "queens_counts.txt")):
        if ln.strip() and not ln.startswith("#"):
            a, b = map(int, ln.split())
            if a == N:
                return b
    raise KeyError(N)


def mixed_model(seed, span=40, n=7):
    """Every constraint kind over a window wider than one word (W = 2 or more)."""
    s = I.Stream(seed)
    lo = [int(v) for v in s.ints(-3, 3, n)]
    hi = [lo[i] + int(s.int(span // 2, span - 7)) for i in range(n)]
    m = I.CspModel(n=n, lo=lo, hi=hi, name=f"mixed-{span}-{seed}")
    for i in range(n):
        for _ in range(3):
            m.removed.append((i, s.int(lo[i], hi[i])))
    m.ne.append((0, 1, 3))
    m.ne.append((2, -1, lo[2] + 1))
    m.ne.append((3, 4, -7))
    last = n - 1
    m.lin.append(([2, -3, 1], [0, 1, 2], 5))
    m.lin.append(([-1, -1, 1, 4], [3, 4, last, last], -2))    # repeated variable: merged
    m.alldiff.append([1, 3, 5, 6] if n >= 7 else [1, n - 2, last])
    sx, sy = hi[2] - lo[2] + 1, hi[last] - lo[last] + 1
    al = (s.ints(0, 2, sx * sy) > 0).reshape(sx, sy)
    m.tables.append((2, last, al))
    return m


def strided_queens(N, stride, alldiff=False, rows=False):
    """N-queens over the values 0, stride, ..., (N-1) stride: the same search tree as
    N-queens (the map k -> k stride is an isomorphism of the constraints), on a window of
    (N-1) stride + 1 values, so W = 4 (stride 13) or W = 8 (stride 31).  With alldiff the
    column constraints become one alldifferent group; rows adds two int_lin_le rows."""
    hi = (N - 1) * stride
    m = I.CspModel(n=N, lo=[0] * N, hi=[hi] * N, name=f"queens{N}x{stride}")
    m.removed = [(i, v) for i in range(N) for v in range(hi + 1) if v % stride]
    for i in range(N):
        for j in range(i + 1, N):
            if not alldiff:
                m.ne.append((i, j, 0))
            m.ne.append((i, j, stride * (i - j)))
            m.ne.append((i, j, stride * (j - i)))
    if alldiff:
        m.alldiff.append(list(range(N)))
    if rows:
        m.lin.append(([1, 1], [0, 1], stride * (N - 1)))
        m.lin.append(([1] * N, list(range(N)), stride * (N * (N - 1) // 2)))
    return m


def pooled_wide_model(seed, span, n=8, pool=9, keep=5):
    """Every constraint kind over one window of `span` values; each domain keeps `keep`
    values of a pool of `pool` values spread over the window (so that domains overlap)."""
    s = I.Stream(seed)
    lo0 = int(s.int(-20, 20))
    m = I.CspModel(n=n, lo=[lo0] * n, hi=[lo0 + span - 1] * n, name=f"pooled-{span}-{seed}")
    P = sorted(lo0 + int(v) for v in s.perm(span)[:pool])
    for i in range(n):
        kept = set(P[int(k)] for k in s.perm(pool)[:keep])
        m.removed += [(i, v) for v in range(lo0, lo0 + span) if v not in kept]
    m.ne += [(0, 1, 0), (2, 3, 0), (6, 7, 0), (1, 6, 0), (4, -1, P[0])]
    m.lin.append(([1, -1, 2], [1, 2, 5], lo0 + int(s.int(span // 3, span // 2))))
    m.lin.append(([-1, -1, 1], [0, 3, 6], -(lo0 + int(s.int(span // 4, span // 2)))))
    m.alldiff.append([0, 2, 4, 5, 7])
    m.tables.append((1, 5, (s.ints(0, 3, span * span) > 0).reshape(span, span)))
    return m


# ----------------------------------------------------------------------------- propagation

def propagate_parity(m, rng, count):
    om = O.OracleModel(m)
    p = K.Csp(m)
    n, W, lo0 = p.layout()
    subs = random_subdomains(om, rng, count)
    din = np.stack([flags_to_bits(om, f, n, W, lo0) for f in subs])
    dout, failed = p.propagate(din)
    n_fail = 0
    for k, f in enumerate(subs):
        of, od = O.propagate(om, f, variant=1)
        assert bool(failed[k]) == of, (m.name, k)
        if of:
            n_fail += 1
            continue
        got = bits_to_flags(om, dout[k], n, W, lo0)
        assert np.array_equal(got, od), (m.name, k, om.flags_to_sets(od), om.flags_to_sets(got))
    ok = ~failed
    if ok.any():                                         # idempotence on the device
        d2, f2 = p.propagate(dout[ok])
        assert not f2.any() and np.array_equal(d2, dout[ok])
    return n_fail


def test_propagate_tiny_random():
    rng = np.random.default_rng(1)
    fails = 0
    for i in range(250):
        m = I.random_tiny(I.seed_for(I.CFG_TINY, 50000 + i))
        fails += propagate_parity(m, rng, 6)
    assert fails > 50


@pytest.mark.parametrize("span", [40, 100, 250])
def test_propagate_multiword(span):
    rng = np.random.default_rng(span)
    for seed in range(6):
        propagate_parity(mixed_model(seed, span), rng, 20)


def test_propagate_queens_rb_linad():
    rng = np.random.default_rng(2)
    propagate_parity(I.queens(8), rng, 64)
    propagate_parity(I.queens(16), rng, 64)
    propagate_parity(I.model_rb(11, 20, 8), rng, 32)
    propagate_parity(I.model_rb(12, 30, 32), rng, 32)
    propagate_parity(I.lin_alldiff(13, n=40, rows=12, groups=4), rng, 16)


def test_propagate_root_linad_full_size():
    rng = np.random.default_rng(3)
    propagate_parity(I.lin_alldiff(I.seed_for(I.CFG_LINAD, 0)), rng, 4)


def test_propagate_empty_and_singletons():
    m = I.queens(6)
    om = O.OracleModel(m)
    p = K.Csp(m)
    n, W, lo0 = p.layout()
    empty = np.zeros(n * W, np.uint32)
    single = np.zeros(n * W, np.uint32)
    for i in range(n):                                     # a full solution: 1 3 5 0 2 4
        single[i] = 1 << [1, 3, 5, 0, 2, 4][i]
    dout, failed = p.propagate(np.stack([empty, single]))
    assert failed[0] and not failed[1] and np.array_equal(dout[1], single)


# ----------------------------------------------------------------------------- search

TILINGS = {
    "auto": None,                          # all-solution search split at depth 3 by default
    "shared": K.tiling(split_depth=-1),    # one queue shared by every worker
    "one-worker": K.tiling(blocks=1, warps_per_block=1, split_depth=-1),
    "spilling": K.tiling(blocks=3, warps_per_block=4, smem_levels=2, queue_records=8, split_depth=-1),
    # all-solution search split at depth k into units solved by per-block teams
    "split1": K.tiling(split_depth=1),
    "split3": K.tiling(split_depth=3, warps_per_block=4),
    "split8": K.tiling(split_depth=8, blocks=5, warps_per_block=2, smem_levels=2),
    # a warp per node also where two sibling nodes per warp would apply (the default there)
    "warp": K.tiling(threads_per_node=32, split_depth=-1),
    "warp-split": K.tiling(threads_per_node=32, warps_per_block=4),
}


def search_parity(m, tiling=None, cap=5000):
    om = O.OracleModel(m)
    r = O.solve(om, cap=cap, variant=1)
    p = K.Csp(m)
    if tiling is not None:
        p.set_tiling(tiling)
    rc, st, sols = p.solve(K.CSP_ALL, cap)
    assert rc == 0, m.name
    assert st["solutions"] == r.solutions, m.name
    assert (st["sol_hash_sum"], st["sol_hash_xor"]) == (r.hash_sum, r.hash_xor), m.name
    assert (st["nodes"], st["fails"]) == (r.nodes, r.fails), m.name
    if r.solutions <= cap:
        assert sorted_rows(sols) == sorted_rows(r.sols), m.name
    return st


@pytest.mark.parametrize("tname", list(TILINGS))
def test_search_queens_small(tname):
    for N in range(1, 11):
        st = search_parity(I.queens(N), TILINGS[tname])
        assert st["solutions"] == queens_count(N)


@pytest.mark.parametrize("c1", ["domain", "lin"])
@pytest.mark.parametrize("c2", ["lin", "table"])
def test_search_worked_example(c1, c2):
    st = search_parity(I.worked_example(c1, c2))
    assert st["solutions"] == 11


@pytest.mark.parametrize("tname", list(TILINGS))
def test_search_tiny_random(tname):
    for i in range(120):
        search_parity(I.random_tiny(I.seed_for(I.CFG_TINY, 70000 + i)), TILINGS[tname])


def test_search_multiword_and_rb():
    for seed in range(4):
        search_parity(mixed_model(100 + seed, 40, 5), cap=100000)
    for k in range(6):
        search_parity(I.model_rb(I.seed_for(I.CFG_RB, 900 + k), 12, 6), cap=100000)


@pytest.mark.parametrize("tname", ["auto", "spilling"])
@pytest.mark.parametrize("N,stride,W", [(9, 13, 4), (10, 13, 4), (8, 31, 8), (9, 31, 8)])
def test_search_strided_queens_wide_domains(N, stride, W, tname):
    m = strided_queens(N, stride)
    assert K.Csp(m).layout()[1] == W
    st = search_parity(m, TILINGS[tname], cap=1000)
    q = O.solve(O.OracleModel(I.queens(N)), variant=1)
    assert (st["nodes"], st["fails"], st["solutions"]) == (q.nodes, q.fails, q.solutions)
    assert st["solutions"] == queens_count(N)


@pytest.mark.parametrize("stride,W", [(13, 4), (31, 8)])
def test_search_alldiff_and_rows_wide_domains(stride, W):
    for N in (8, 9):
        m = strided_queens(N, stride, alldiff=True, rows=True)
        assert K.Csp(m).layout()[1] == W
        search_parity(m, cap=1000)


@pytest.mark.parametrize("span,W", [(100, 4), (250, 8)])
def test_search_every_kind_wide_domains(span, W):
    for seed in range(6):
        m = pooled_wide_model(1000 + seed, span)
        assert K.Csp(m).layout()[1] == W
        search_parity(m, cap=20000)
        search_parity(m, TILINGS["spilling"], cap=0)


def random_ne_model(seed, n, dmax, m):
    """One-word int_ne-only problems: domains of up to dmax values (holes included) inside
    one 32-value window, binary constraints with offsets up to +-40 (beyond one word as
    well), unary ones, and self constraints x != x + c."""
    s = I.Stream(seed)
    lo0 = int(s.int(-5, 5))
    lo, hi = [], []
    for i in range(n):
        a = lo0 + int(s.int(0, 31 - dmax))
        lo.append(a)
        hi.append(a + int(s.int(1, dmax - 1)))
    M = I.CspModel(n=n, lo=lo, hi=hi, name=f"ne-{n}-{seed}")
    for i in range(n):
        if s.int(0, 3) == 0:
            M.removed.append((i, int(s.int(lo[i], hi[i]))))
    for _ in range(m):
        x, k = int(s.int(0, n - 1)), int(s.int(0, 19))
        if k == 0:
            M.ne.append((x, -1, int(s.int(lo0, lo0 + 31))))
        elif k == 1:
            M.ne.append((x, x, int(s.int(-2, 2))))
        elif k == 2:
            M.ne.append((x, x, int(s.int(1, 3))))
        else:
            y = int(s.int(0, n - 1))
            M.ne.append((x, y, int(s.int(-40, 40)) if k < 6 else int(s.int(-6, 6))))
    return M


PAIR_TILINGS = {
    "pairs": K.tiling(threads_per_node=16),
    "pairs-shared": K.tiling(threads_per_node=16, split_depth=-1),
    "pairs-one-worker": K.tiling(threads_per_node=16, blocks=1, warps_per_block=1, split_depth=-1),
    # two shared-memory levels: pairs push two levels at once through the spill path
    "pairs-spilling": K.tiling(threads_per_node=16, blocks=3, warps_per_block=4, smem_levels=2,
                               queue_records=8, split_depth=-1),
    "pairs-split8": K.tiling(threads_per_node=16, split_depth=8, blocks=5, warps_per_block=2,
                             smem_levels=2),
}


@pytest.mark.parametrize("tname", list(PAIR_TILINGS))
def test_two_nodes_per_warp(tname):
    """Two sibling nodes per warp (a half-warp each) on one-word int_ne models of at most 16
    variables: nodes, fails, solutions, both hashes and the stored solutions equal the
    oracle's depth-first search, in every tiling; the stack never needs more than 2n - 1
    levels."""
    t = PAIR_TILINGS[tname]
    for N in range(1, 13):
        st = search_parity(I.queens(N), t)
        assert st["solutions"] == queens_count(N)
        assert st["max_depth"] <= max(1, 2 * N - 1)
    compared = 0
    for seed in range(30):
        n = 6 + seed % 11                                   # 6 .. 16 variables
        M = random_ne_model(9100 + seed, n, 8 if n < 10 else 6, 2 * n + 6)
        r = O.solve(O.OracleModel(M), cap=0, variant=1, node_limit=100_000)
        if r.status < 0:
            continue
        search_parity(M, t, cap=3000)
        compared += 1
    assert compared >= 15


@pytest.mark.parametrize("dw", [2, 4, 8])
def test_search_at_wider_domain_words(dw):
    """csp_tiling.domain_words: the same searches with wider bitsets (upper words empty) give
    the oracle's counts, hashes and stored solutions; propagation keeps the problem's layout
    and fixpoints."""
    models = [I.queens(8), random_ne_model(9500, 12, 6, 30),
              I.model_rb(I.seed_for(I.CFG_RB, 77), 14, 7), I.worked_example("lin", "table"),
              mixed_model(120, 30, 5), strided_queens(7, 13)]
    for m in models:
        if K.Csp(m).layout()[1] > dw:
            continue
        search_parity(m, K.tiling(domain_words=dw), cap=2000)
        search_parity(m, K.tiling(domain_words=dw, split_depth=-1), cap=2000)
    p = K.Csp(I.queens(10))
    root = p.root_domains().reshape(1, -1)
    out0, f0 = p.propagate(root)
    p.set_tiling(K.tiling(domain_words=dw))
    out1, f1 = p.propagate(root)
    assert np.array_equal(out0, out1) and np.array_equal(f0, f1)


def test_tuned_single_shape_keeps_the_results():
    """The autotuner's axes for one problem (warps per block, two nodes or one per warp, the
    problem's own or a wider bitset): every shape it times gives the oracle's counts, and so
    does the shape it picks.  Two nodes per warp need one-word domains, so they are tried at
    the problem's own width only."""
    from paper_1909_09213_gb300 import tune
    m = I.queens(10)
    t, entry = tune.tune_single(m, reps=0, use_cache=False)
    tried = {(c["threads_per_node"], c["domain_words"]) for _, c in entry["candidates"]}
    assert tried == {(16, 0), (32, 0), (32, 2)}
    search_parity(m, t)
    m2 = I.model_rb(I.seed_for(I.CFG_RB, 78), 20, 8)            # tables: one node per warp
    t2, entry2 = tune.tune_single(m2, reps=0, use_cache=False)
    assert all(c["threads_per_node"] == 32 for _, c in entry2["candidates"])
    search_parity(m2, t2)


def test_two_nodes_per_warp_limits_and_modes():
    p = K.Csp(I.queens(12))
    p.set_tiling(K.tiling(threads_per_node=16, blocks=2, warps_per_block=2, split_depth=-1))
    rc, st, _ = p.solve(K.CSP_ALL, 0, K.limits(node_limit=5_000))
    assert rc == K.CSP_ELIMIT and st["nodes"] >= 5_000
    with pytest.raises(K.CspError) as e:             # pairs are for all-solution search only
        p.solve(K.CSP_FIRST)
    assert e.value.code == K.CSP_EINVAL
    # a batch of such problems: pairs in its all-solution launches, a warp per node otherwise
    models = [I.queens(N) for N in (6, 8, 9, 10)] + [random_ne_model(9300 + k, 12, 6, 30)
                                                    for k in range(4)]
    b = K.Batch([K.Csp(m) for m in models])
    rc, res = b.solve(K.CSP_ALL)
    for m, r in zip(models, res):
        o = O.solve(O.OracleModel(m), cap=0, variant=1)
        assert (r["nodes"], r["fails"], r["solutions"]) == (o.nodes, o.fails, o.solutions), m.name
    rc, res = b.solve(K.CSP_FIRST)
    for m, r in zip(models, res):
        o = O.solve(O.OracleModel(m), mode=1, cap=1, variant=1)
        assert r["status"] == o.status, m.name


@pytest.mark.parametrize("n,dmax,m", [(6, 8, 12), (12, 6, 30), (20, 5, 70), (32, 3, 110), (33, 3, 110)])
def test_search_random_ne_one_word(n, dmax, m):
    """The register-held kernel (n <= 32) and the shared-memory one (n = 33) on random
    int_ne models that the oracle decides within 200 000 nodes."""
    compared, big = 0, 0
    for seed in range(40):
        M = random_ne_model(500 + 7 * seed + n, n, dmax, m)
        r = O.solve(O.OracleModel(M), cap=0, variant=1, node_limit=200_000)
        if r.status < 0:
            continue
        search_parity(M, cap=2000)
        compared += 1
        big += r.nodes >= 1000
    assert compared >= 10 and big >= 2, (compared, big)


def test_search_spill_heavy_deep_stack():
    # 12-queens with 2 shared-memory levels per worker: most levels live in global memory
    for split in (-1, 0):
        st = search_parity(I.queens(12), K.tiling(blocks=4, warps_per_block=8, smem_levels=2,
                                                  split_depth=split), cap=10)
        assert st["spills"] > 0


def test_first_mode_status_and_validity():
    for i in range(150):
        m = I.random_tiny(I.seed_for(I.CFG_TINY, 80000 + i))
        om = O.OracleModel(m)
        r = O.solve(om, mode=1, cap=1)
        p = K.Csp(m)
        rc, st, sols = p.solve(K.CSP_FIRST)
        assert rc == 0
        assert st["solutions"] == (1 if r.status == 1 else 0), m.name
        if r.status == 1:
            assert O.check_solution(om, sols[0]), m.name


def test_first_mode_single_worker_is_the_oracle_order():
    for m in [I.queens(8), I.queens(12), I.model_rb(I.seed_for(I.CFG_RB, 7), 25, 10)]:
        om = O.OracleModel(m)
        r = O.solve(om, mode=1, cap=1)
        p = K.Csp(m)
        p.set_tiling(K.tiling(blocks=1, warps_per_block=1))
        rc, st, sols = p.solve(K.CSP_FIRST)
        assert rc == 0 and st["solutions"] == r.solutions
        assert (st["nodes"], st["fails"]) == (r.nodes, r.fails)
        if r.solutions:
            assert tuple(sols[0]) == tuple(r.sols[0])


def oracle_reference(N):
    """Full-size oracle results written by tests/golden/make_queens_reference.py."""
    path = os.path.join(GOLDEN, "queens_oracle.txt")
    for ln in open(path):
        if ln.strip() and not ln.startswith("#"):
            f = list(map(int, ln.split()[:6]))
            if f[0] == N:
                return dict(zip(["N", "nodes", "fails", "solutions", "hash_sum", "hash_xor"], f))
    pytest.skip(f"no oracle reference for N={N}")


@pytest.mark.parametrize("split", [-1, 0])
@pytest.mark.parametrize("N", [14, 15, 16])
def test_queens_full_size_against_oracle_reference(N, split):
    # one shared queue, and the default split of the first levels
    ref = oracle_reference(N)
    p = K.Csp(I.queens(N))
    p.set_tiling(K.tiling(split_depth=split))
    rc, st, _ = p.solve(K.CSP_ALL, 0)
    assert rc == 0 and st["solutions"] == queens_count(N) == ref["solutions"]
    assert (st["nodes"], st["fails"]) == (ref["nodes"], ref["fails"])
    assert (st["sol_hash_sum"], st["sol_hash_xor"]) == (ref["hash_sum"], ref["hash_xor"])


def test_queens_14_full_size():
    p = K.Csp(I.queens(14))
    rc, st, _ = p.solve(K.CSP_ALL, 0)
    assert rc == 0 and st["solutions"] == queens_count(14)


def test_queens_16_full_size_and_sampled_subtrees():
    """16-queens in the benchmark's launch shape (one shared queue) and split: the published
    count; nodes, fails and the solution hash of sampled subtrees (x0, x1 fixed) against the
    oracle."""
    for split in (-1, 0):
        p = K.Csp(I.queens(16))
        p.set_tiling(K.tiling(split_depth=split))
        rc, st, _ = p.solve(K.CSP_ALL, 0)
        assert rc == 0 and st["solutions"] == queens_count(16)
        assert st["steals"] > 0
    for (a, b) in [(0, 2), (7, 3)]:
        m = I.queens(16)
        m.removed += [(0, v) for v in range(16) if v != a] + [(1, v) for v in range(16) if v != b]
        search_parity(m, cap=0)


@pytest.mark.parametrize("nparts", [2, 3, 5])
def test_partitioned_tree_sums_to_the_whole(nparts):
    """The parts of a shared tree (csp_set_partition), run one after another on this GPU,
    combine to the undivided search: what ranks on separate GPUs would exchange."""
    from paper_1909_09213_gb300 import shard
    for m in [I.queens(12), I.model_rb(I.seed_for(I.CFG_RB, 11), 14, 7), mixed_model(210, 40, 5)]:
        whole = K.Csp(m)
        rc, st_whole, _ = whole.solve(K.CSP_ALL, 0)
        assert rc == 0
        parts = []
        for part in range(nparts):
            p = K.Csp(m)
            p.set_partition(part, nparts)
            rc, st, _ = p.solve(K.CSP_ALL, 0)
            assert rc == 0
            parts.append(st)
        got = shard.combine(parts)
        for k in shard.FIELDS:
            assert got[k] == st_whole[k], (m.name, k)


@pytest.mark.parametrize("depth,nparts", [(2, 2), (3, 3), (4, 8)])
def test_tree_cut_at_depth_k_sums_to_the_whole(depth, nparts):
    """shard.solve_part: the tree cut at depth k (levels expanded with csp_propagate, units
    solved as batches of root copies); the parts, run one after another on this GPU, combine
    to the undivided search.  In first-solution mode some part finds a valid solution."""
    from paper_1909_09213_gb300 import shard
    for m in [I.queens(12), I.model_rb(I.seed_for(I.CFG_RB, 11), 14, 7), mixed_model(210, 40, 5),
              strided_queens(9, 31)]:
        rc, whole, _ = K.Csp(m).solve(K.CSP_ALL, 0)
        assert rc == 0
        parts = [shard.solve_part(K.Csp(m), part, nparts, depth) for part in range(nparts)]
        assert sum(pt["units"] for pt in parts) == parts[0]["units_total"]
        got = shard.combine(parts)
        for k in shard.FIELDS:
            assert got[k] == whole[k], (m.name, k)
        found = []
        for part in range(nparts):
            st, (f, sol) = shard.solve_part(K.Csp(m), part, nparts, depth, mode=K.CSP_FIRST, chunk=8)
            if f:
                assert O.check_solution(O.OracleModel(m), sol), m.name
            found.append(f)
        assert any(found) == (whole["solutions"] > 0), m.name


@pytest.mark.parametrize("N,depth", [(14, 3), (16, 3), (16, 4)])
def test_split_full_size_against_oracle_reference(N, depth):
    """The benchmark's trees split at depth k: nodes, fails, solutions and both hashes equal
    the oracle's full-size run."""
    from paper_1909_09213_gb300 import shard
    ref = oracle_reference(N)
    p = K.Csp(I.queens(N))
    p.set_tiling(K.tiling(split_depth=depth))
    rc, st, _ = p.solve(K.CSP_ALL, 0)
    assert rc == 0
    assert (st["nodes"], st["fails"], st["solutions"], st["sol_hash_sum"], st["sol_hash_xor"]) == (
        ref["nodes"], ref["fails"], ref["solutions"], ref["hash_sum"], ref["hash_xor"])
    # the subtrees solved: the same cut made on the host from csp_propagate's fixpoints
    n, W = p.layout()[:2]
    units, nodes, fails = shard.split_units(p.propagate, p.root_domains().ravel(), n, W, depth)
    assert st["units"] == len(units)
    q = K.Csp(I.queens(N))
    q.set_tiling(K.tiling(split_depth=-1))
    rc, st1, _ = q.solve(K.CSP_ALL, 0)
    assert rc == 0 and st1["units"] == 1 and st1["nodes"] == st["nodes"]


def test_tiny_units_with_many_helper_blocks_repeated():
    """Small trees split into a few tiny units, most blocks helping other blocks' teams: the
    owner of a team reuses its queue for its next unit only once no helper is left, so no
    record is taken twice.  Repeated solves (the interleavings vary), and a batch of many
    tiny instances, per instance."""
    for N in (6, 7, 8, 9):
        r = O.solve(O.OracleModel(I.queens(N)), cap=0, variant=1)
        p = K.Csp(I.queens(N))
        p.bind(K.CSP_ALL, 0)
        p.upload(K.CSP_ALL, 0)
        for _ in range(40):
            p.launch()
            assert p.collect(None) == 0
            st = p.stats()
            assert (st["nodes"], st["fails"], st["solutions"], st["sol_hash_sum"],
                    st["sol_hash_xor"]) == (r.nodes, r.fails, r.solutions, r.hash_sum,
                                            r.hash_xor), N
    models = [I.queens(4 + k % 5) for k in range(96)]
    refs = {m.n: O.solve(O.OracleModel(m), cap=0, variant=1) for m in models}
    b = K.Batch([K.Csp(m) for m in models])
    for _ in range(10):
        rc, res = b.solve(K.CSP_ALL)
        assert rc == 0
        for m, x in zip(models, res):
            o = refs[m.n]
            assert (x["nodes"], x["fails"], x["solutions"]) == (o.nodes, o.fails, o.solutions), m.name


def test_split_level_overflow_keeps_the_last_level_that_fits():
    """16-queens split at depth 6: a level of more than 2^16 states (the level buffers of a
    16-variable problem) is not expanded, and the level above it becomes the units; the
    counts still equal the oracle's full-size run."""
    from paper_1909_09213_gb300 import shard
    ref = oracle_reference(16)
    p = K.Csp(I.queens(16))
    p.set_tiling(K.tiling(split_depth=6))
    rc, st, _ = p.solve(K.CSP_ALL, 0)
    assert rc == 0
    assert (st["nodes"], st["fails"], st["solutions"], st["sol_hash_sum"], st["sol_hash_xor"]) == (
        ref["nodes"], ref["fails"], ref["solutions"], ref["hash_sum"], ref["hash_xor"])
    n, W = p.layout()[:2]
    root = p.root_domains().ravel()
    cuts = {d: len(shard.split_units(p.propagate, root, n, W, d)[0]) for d in (4, 5)}
    assert cuts[4] <= 1 << 16 < cuts[5]              # the level at depth 5 does not fit
    assert st["units"] == cuts[4]


@pytest.mark.parametrize("tname", ["split1", "split3"])
def test_split_wide_domains_and_every_kind(tname):
    for m in [strided_queens(9, 31), strided_queens(8, 13, alldiff=True, rows=True),
              pooled_wide_model(1003, 250), mixed_model(101, 40, 5),
              I.model_rb(I.seed_for(I.CFG_RB, 902), 12, 6)]:
        search_parity(m, TILINGS[tname], cap=20000)


def test_split_repeated_launches_and_stored_solutions():
    """One upload, several launches: each launch restarts the split from the root; the
    stored solutions are the oracle's."""
    m = I.queens(9)
    r = O.solve(O.OracleModel(m), cap=400, variant=1)
    p = K.Csp(m)
    p.set_tiling(K.tiling(split_depth=2))
    p.bind(K.CSP_ALL, 400)
    p.upload(K.CSP_ALL, 400)
    for _ in range(3):
        sols = np.zeros((400, 9), np.int32)
        p.launch()
        assert p.collect(sols) == 0
        st = p.stats()
        assert (st["nodes"], st["fails"], st["solutions"]) == (r.nodes, r.fails, r.solutions)
        assert sorted_rows(sols[:st["stored"]]) == sorted_rows(r.sols)


def test_split_limits_are_global_and_partitions_unsplit():
    p = K.Csp(I.queens(12))
    p.set_tiling(K.tiling(split_depth=3, blocks=2, warps_per_block=2))
    rc, st, _ = p.solve(K.CSP_ALL, 0, K.limits(node_limit=5_000))
    assert rc == K.CSP_ELIMIT
    # a partitioned handle keeps the shared-queue search: the parts still sum to the whole
    from paper_1909_09213_gb300 import shard
    m = I.queens(10)
    rc, whole, _ = K.Csp(m).solve(K.CSP_ALL, 0)
    parts = []
    for part in range(3):
        q = K.Csp(m)
        q.set_tiling(K.tiling(split_depth=3))
        q.set_partition(part, 3)
        rc, st, _ = q.solve(K.CSP_ALL, 0)
        assert rc == 0
        parts.append(st)
    got = shard.combine(parts)
    assert all(got[k] == whole[k] for k in shard.FIELDS)
    # first-solution search is not split
    q = K.Csp(I.queens(10))
    q.set_tiling(K.tiling(split_depth=3))
    rc, st, sols = q.solve(K.CSP_FIRST)
    assert rc == 0 and st["solutions"] == 1 and O.check_solution(O.OracleModel(I.queens(10)), sols[0])


# ----------------------------------------------------------------------------- limits, errors

@pytest.mark.parametrize("split", [-1, 0])
def test_node_limit(split):
    p = K.Csp(I.queens(11))
    # limits are checked every 64 nodes
    p.set_tiling(K.tiling(blocks=1, warps_per_block=2, split_depth=split))
    rc, st, _ = p.solve(K.CSP_ALL, 0, K.limits(node_limit=200))
    assert rc == K.CSP_ELIMIT and st["nodes"] >= 200


def test_wait_limit_returns_timeout():
    # no worker ever donates, so every idle worker waits until the limit runs out
    p = K.Csp(I.queens(13))
    p.set_tiling(K.tiling(split_depth=-1))                  # one queue for the whole tree
    rc, st, _ = p.solve(K.CSP_ALL, 0, K.limits(wait_limit_ns=20_000_000, flags=K.CSP_F_NO_DONATE))
    assert rc == K.CSP_ETIMEOUT
    rc, st, _ = p.solve(K.CSP_ALL, 0)                       # the context is still usable
    assert rc == 0 and st["solutions"] == queens_count(13)


def test_small_workspace_is_enomem():
    import ctypes as C
    p = K.Csp(I.queens(8))
    ws = torch.empty(1024, dtype=torch.uint8, device="cuda")
    L = K.lib()
    assert L.csp_bind(p.h, C.c_void_p(ws.data_ptr()), 1024, None) == 0
    sols = np.zeros((1, 8), np.int32)
    assert L.csp_solve(p.h, K.CSP_ALL, 0, sols.ctypes.data_as(K._I32P), None) == K.CSP_ENOMEM


def test_failed_upload_leaves_the_previous_upload_usable():
    """On error the handle is unchanged: an upload that does not fit the bound workspace
    (a larger cap) leaves the earlier upload in place, and it still launches correctly."""
    m = I.queens(10)
    orc = O.solve(O.OracleModel(m), cap=0, variant=1)
    p = K.Csp(m)
    p.bind(K.CSP_ALL, 0)
    p.upload(K.CSP_ALL, 0)
    assert K.lib().csp_upload(p.h, K.CSP_ALL, 10_000_000) == K.CSP_ENOMEM
    p.launch()
    assert p.collect() == 0
    st = p.stats()
    assert (st["solutions"], st["nodes"], st["fails"], st["sol_hash_sum"], st["sol_hash_xor"]) == (
        orc.solutions, orc.nodes, orc.fails, orc.hash_sum, orc.hash_xor)


def test_block_beyond_register_budget_is_einval():
    # the one-word first-fail kernel is capped at 80 registers per thread: a 32-warp block
    # (32 x 32 x 80 > 64 K registers) does not fit, a 16-warp block does
    m = I.model_rb(I.seed_for(I.CFG_RB, 5), 14, 6)
    p = K.Csp(m)
    p.set_tiling(K.tiling(warps_per_block=32))
    with pytest.raises(K.CspError) as e:
        p.workspace_bytes(K.CSP_ALL, 0)
    assert e.value.code == K.CSP_EINVAL
    p.set_tiling(K.tiling(warps_per_block=16))
    search_parity(m, K.tiling(warps_per_block=16))
    # the register-held int_ne kernel (64 registers) takes a whole 32-warp block
    p = K.Csp(I.queens(8))
    p.set_tiling(K.tiling(warps_per_block=32))
    rc, st, _ = p.solve(K.CSP_ALL, 0)
    assert rc == 0 and st["solutions"] == queens_count(8) and st["workers"] % 32 == 0


# ----------------------------------------------------------------------------- batches

def _rb_small(count, first=0):
    return I.rb_batch(count, n_range=(8, 16), d_range=(4, 9), config_id=I.CFG_RB + 100, first=first)


def test_batch_first_matches_oracle_status():
    models = _rb_small(96)
    probs = [K.Csp(m) for m in models]
    b = K.Batch(probs)
    rc, res = b.solve(K.CSP_FIRST)
    assert rc == 0
    sat = 0
    for m, r in zip(models, res):
        om = O.OracleModel(m)
        o = O.solve(om, mode=1, cap=1)
        assert r["status"] == o.status, m.name
        if o.status == 1:
            sat += 1
            assert O.check_solution(om, r["solution"]), m.name
    assert 0 < sat < len(models)


def test_batch_all_counts_and_graph_replay():
    models = _rb_small(48, first=500)
    b = K.Batch([K.Csp(m) for m in models])
    rc, res = b.solve(K.CSP_ALL)
    assert rc == 0
    for m, r in zip(models, res):
        o = O.solve(O.OracleModel(m), variant=1)
        assert (r["solutions"], r["nodes"], r["fails"]) == (o.solutions, o.nodes, o.fails), m.name
    rc, res_g = b.solve(K.CSP_ALL, use_graph=True)
    rc2, res_g2 = b.solve(K.CSP_ALL, use_graph=True)
    assert rc == 0 and rc2 == 0
    strip = lambda rs: [(r["status"], r["solutions"], r["nodes"]) for r in rs]
    assert strip(res_g) == strip(res) == strip(res_g2)


def test_batch_node_limit_is_per_instance():
    """A batch node limit stops only the instances that reach it: they report CSP_ELIMIT and
    the others keep their exact verdicts."""
    easy = _rb_small(24, first=1300)
    hard = I.queens(13)                                     # 4.2 M nodes in all-solution mode
    models = easy[:12] + [hard] + easy[12:]
    b = K.Batch([K.Csp(m) for m in models])
    rc, res = b.solve(K.CSP_ALL, lim=K.limits(node_limit=100_000))
    assert rc == 0
    assert res[12]["status"] == K.CSP_ELIMIT
    for m, r in zip(easy, res[:12] + res[13:]):
        o = O.solve(O.OracleModel(m), variant=1)
        assert (r["status"], r["solutions"], r["nodes"]) == (o.status, o.solutions, o.nodes), m.name


def test_batch_tilings_do_not_change_results():
    models = _rb_small(40, first=900)
    probs = [K.Csp(m) for m in models]
    out = []
    for t in [K.tiling(warps_per_block=1), K.tiling(warps_per_block=8, smem_levels=2),
              K.tiling(blocks=5, warps_per_block=4)]:
        b = K.Batch(probs)
        b.set_tiling(t)
        rc, res = b.solve(K.CSP_ALL)
        assert rc == 0
        out.append([(r["solutions"], r["nodes"], r["fails"]) for r in res])
    assert out[0] == out[1] == out[2]


def test_batch_full_size_model_rb_verdicts_against_oracle_file():
    """The benchmark's model-RB workload at full size (instances 0..511 of the 4096; n up to
    60, d up to 32): every verdict equals the one the oracle wrote to
    tests/golden/rb4096_oracle.txt (where it decided within its node budget), and every SAT
    instance's solution satisfies the model.  The undecided ones get a node limit."""
    golden = {}
    for ln in open(os.path.join(GOLDEN, "rb4096_oracle.txt")):
        if ln.strip() and not ln.startswith("#"):
            i, n, d, status, nodes = map(int, ln.split())
            golden[i] = (n, d, status)
    models = I.rb_batch(512)
    b = K.Batch([K.Csp(m) for m in models])
    rc, res = b.solve(K.CSP_FIRST, lim=K.limits(node_limit=50_000_000), use_graph=True)
    assert rc == 0
    decided = 0
    for i, (m, r) in enumerate(zip(models, res)):
        n, d, status = golden[i]
        assert (m.n, len(m.lo)) == (n, n)
        if status >= 0:
            decided += 1
            assert r["status"] == status, (i, r["status"], status)
        if r["status"] == 1:
            assert O.check_solution(O.OracleModel(m), r["solution"]), i
    assert decided >= 500


def test_batch_transfer_byte_accounting():
    """csp_stats of a batch: h2d_bytes counts the upload since the previous successful
    collect (the encoded instances plus 16 bytes of offsets per instance), d2h_bytes the
    launch counters, the per-instance records and, when asked for, the solutions."""
    import ctypes as C
    models = _rb_small(16, first=40)
    b = K.Batch([K.Csp(m) for m in models])
    rc, _ = b.solve(K.CSP_FIRST)                  # uploads, launches, collects with solutions
    assert rc == 0
    st = b.stats()
    words = K.lib().csp_batch_solution_words(b.b)
    assert st["h2d_bytes"] > 16 * len(models) and st["h2d_bytes"] % 4 == 0
    res = (K.csp_result * len(models))()
    sol = np.zeros(max(words, 1), np.int32)
    K._check(K.lib().csp_batch_launch(b.b, None, 0), "launch")
    assert K.lib().csp_batch_collect(b.b, res, None) == 0
    st_none = b.stats()
    assert st_none["h2d_bytes"] == 0                  # nothing uploaded since the last collect
    K._check(K.lib().csp_batch_launch(b.b, None, 0), "launch")
    assert K.lib().csp_batch_collect(b.b, res, sol.ctypes.data_as(K._I32P)) == 0
    st_sol = b.stats()
    assert st_sol["d2h_bytes"] - st_none["d2h_bytes"] == 4 * words
    b.set_tiling(K.tiling(warps_per_block=2))          # forces a new upload
    rc, _ = b.solve(K.CSP_FIRST)
    assert rc == 0 and b.stats()["h2d_bytes"] == st["h2d_bytes"]
