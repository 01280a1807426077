"""GPU parity of the bounds-consistent alldifferent propagator (Section 4, second direction)
against the oracle, which decides bound supports by bipartite matching on the interval
relaxation: bit-exact fixpoints (alone and among the other constraint kinds, one- and
multi-word domains, groups up to 32 members) and search parity (nodes, fails, solutions,
hashes)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_1909_09213_gb300 import cubics as K
from paper_1909_09213_gb300 import instances as I

from _util import bits_to_flags, flags_to_bits, random_subdomains, sorted_rows

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def group_model(seed, k, width, extra=False, ve=False, off=0, keep=None):
    """k members whose domains are random intervals with holes inside a window of `width`
    values starting at `off` (so that several words are in play when width > 32); `keep`:
    at most that many values besides the bounds stay in each domain; with `extra`, an int_ne,
    a linear row and a table over the members too."""
    s = I.Stream(I.seed_for(I.CFG_TINY, 120000 + seed))
    lo = [off + int(s.int(0, width // 2)) for _ in range(k)]
    hi = [min(off + width - 1, lo[i] + int(s.int(0, width // 2))) for i in range(k)]
    lo[0], hi[-1] = off, off + width - 1                  # the window spans `width` values
    m = I.CspModel(n=k, lo=lo, hi=hi, name=f"adbc-{k}-{width}-{seed}")
    for i in range(k):
        for _ in range(int(s.int(0, 3))):
            m.removed.append((i, int(s.int(lo[i], hi[i]))))
        if keep is not None and hi[i] - lo[i] > keep + 1:
            inner = list(range(lo[i] + 1, hi[i]))
            kept = set(inner[int(j)] for j in s.perm(len(inner))[:keep])
            m.removed += [(i, v) for v in inner if v not in kept]
    m.alldiff_bc.append(list(range(k)))
    if ve:
        m.alldiff.append(list(range(k)))
    if extra and k >= 3:
        m.ne.append((0, 1, int(s.int(-3, 3))))
        m.lin.append(([1, 2, -1], [0, 1, 2], int(sum(hi[:2]) - lo[2])))
        sx, sy = hi[1] - lo[1] + 1, hi[2] - lo[2] + 1
        m.tables.append((1, 2, (s.ints(0, 3, sx * sy) > 0).reshape(sx, sy)))
    return m


def propagate_parity(m, rng, count):
    om = O.OracleModel(m)
    p = K.Csp(m)
    n, W, lo0 = p.layout()
    subs = [om.root_flags()] + random_subdomains(om, rng, count)
    din = np.stack([flags_to_bits(om, f, n, W, lo0) for f in subs])
    dout, failed = p.propagate(din)
    fails = 0
    for k, f in enumerate(subs):
        of, od = O.propagate(om, f, variant=1)
        assert bool(failed[k]) == of, (m.name, k)
        if of:
            fails += 1
            continue
        got = bits_to_flags(om, dout[k], n, W, lo0)
        assert np.array_equal(got, od), (m.name, k, om.flags_to_sets(od), om.flags_to_sets(got))
    return fails, len(subs)


@pytest.mark.parametrize("width,W", [(12, 1), (30, 1), (60, 2), (120, 4), (250, 8)])
def test_propagate_groups_bit_exact(width, W):
    rng = np.random.default_rng(width)
    fails = total = 0
    for seed in range(40):
        k = 2 + seed % 9
        m = group_model(1000 * W + seed, k, width, extra=seed % 2 == 1, ve=seed % 3 == 0,
                        off=int(rng.integers(-20, 20)))
        assert K.Csp(m).layout()[1] == W, m.name
        f, t = propagate_parity(m, rng, 12)
        fails, total = fails + f, total + t
    assert 0 < fails < total


def test_propagate_closed_forms():
    # the oracle's pinned closed forms, on the device
    cases = [([1, 1, 1], [2, 2, 3], [], [[1, 2], [1, 2], [3]]),
             ([2, 2, 1], [3, 3, 4], [], [[2, 3], [2, 3], [1, 2, 3, 4]]),
             ([1, 1, 1, 1], [3, 3, 3, 6], [(3, 4)], [[1, 2, 3]] * 3 + [[5, 6]]),
             ([1, 1, 1], [2, 2, 2], [], None)]
    for lo, hi, removed, want in cases:
        m = I.CspModel(n=len(lo), lo=lo, hi=hi, removed=list(removed))
        m.alldiff_bc.append(list(range(len(lo))))
        om = O.OracleModel(m)
        p = K.Csp(m)
        n, W, lo0 = p.layout()
        dout, failed = p.propagate(flags_to_bits(om, om.root_flags(), n, W, lo0)[None, :])
        assert bool(failed[0]) == (want is None)
        if want is not None:
            assert om.flags_to_sets(bits_to_flags(om, dout[0], n, W, lo0)) == want


def test_propagate_full_group_of_32():
    rng = np.random.default_rng(7)
    for seed in range(6):
        m = group_model(5000 + seed, 32, 40)
        propagate_parity(m, rng, 8)


@pytest.mark.parametrize("width", [20, 100])
def test_search_parity(width):
    searched = 0
    for seed in range(24):
        m = group_model(7000 + seed, 4 + seed % 4, width, extra=seed % 2 == 0, ve=seed % 3 == 0,
                        keep=None if width <= 32 else 6)
        om = O.OracleModel(m)
        r = O.solve(om, cap=5000, variant=1, node_limit=300_000)
        if r.status < 0:
            continue
        p = K.Csp(m)
        rc, st, sols = p.solve(K.CSP_ALL, 5000)
        assert rc == 0, m.name
        assert (st["solutions"], st["sol_hash_sum"], st["sol_hash_xor"]) == (
            r.solutions, r.hash_sum, r.hash_xor), m.name
        assert (st["nodes"], st["fails"]) == (r.nodes, r.fails), m.name
        if r.solutions <= 5000:
            assert sorted_rows(sols) == sorted_rows(r.sols), m.name
        searched += 1
    assert searched >= 10


def test_search_queens_columns_as_a_bounds_consistent_group():
    """N-queens with the columns as one bounds-consistent group next to the diagonal int_ne
    constraints: the published counts, and the oracle's nodes and fails."""
    for N, count in [(6, 4), (8, 92), (9, 352)]:
        m = I.queens(N)
        m.ne = [(x, y, c) for (x, y, c) in m.ne if c != 0]
        m.alldiff_bc.append(list(range(N)))
        r = O.solve(O.OracleModel(m), variant=1)
        rc, st, _ = K.Csp(m).solve(K.CSP_ALL, 0)
        assert rc == 0 and st["solutions"] == r.solutions == count
        assert (st["nodes"], st["fails"], st["sol_hash_sum"]) == (r.nodes, r.fails, r.hash_sum)
