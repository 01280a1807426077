"""Seeded synthetic CSP instances: the inputs shared by the CUDA path and the oracle.

This module only *describes* problems.  It holds none of the solver's arithmetic (no
propagation, no search, no solution hashing); both the CUDA library and the CPU oracle
consume a ``CspModel`` and each encodes it in its own way.

A CSP is the triple (X, D, C) of the paper's Section 1.1: variables, one finite domain per
variable, and constraints, each a relation over the domains of the variables it involves.
Four constraint kinds are described here:

* ``ne``      x != y + c       (``y == -1`` means the unary x != c)
* ``lin``     sum_i a_i * x_i <= b
* ``alldiff`` pairwise distinct values over a group of variables
* ``tables``  binary relation given as a boolean matrix ``allowed[a - lo_x, b - lo_y]``

Random numbers come from a counter-based splitmix64 stream (Steele, Lea and Flood 2014),
implemented with numpy uint64 arithmetic so the same seed gives the same instance on every
machine and numpy version.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

M64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15
BASE_SEED = 20190920

# config identifiers used to derive per-instance seeds
CFG_QUEENS, CFG_RB, CFG_RB_TRAIN, CFG_RB_EVAL, CFG_LINAD, CFG_TINY = 1, 3, 40, 41, 5, 99
CFG_LNS_OBJ, CFG_LNS_RELAX = 60, 61     # objective weights; neighbourhood draws
CFG_LINAD_TRAIN = 42                    # training instances of the mixed workload's brancher


def _mix64(z: int) -> int:
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def seed_for(config_id: int, i: int, base: int = BASE_SEED) -> int:
    """Per-instance seed: one splitmix64 step of base ^ (config_id << 32) ^ i."""
    return _mix64(((base ^ (config_id << 32) ^ i) + GOLDEN) & M64)


def _mix64_np(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


class Stream:
    """Counter-based splitmix64 stream: draw i is mix(seed + (i + 1) * GOLDEN)."""

    def __init__(self, seed: int):
        self.seed = seed & M64
        self.count = 0

    def u64(self, k: int) -> np.ndarray:
        idx = np.arange(self.count + 1, self.count + 1 + k, dtype=np.uint64)
        self.count += k
        with np.errstate(over="ignore"):
            z = np.uint64(self.seed) + idx * np.uint64(GOLDEN)
        return _mix64_np(z)

    def ints(self, lo: int, hi: int, k: int) -> np.ndarray:
        """k integers uniform on [lo, hi] (multiply-high reduction of the top 32 bits)."""
        span = hi - lo + 1
        top = self.u64(k) >> np.uint64(32)
        return (lo + ((top * np.uint64(span)) >> np.uint64(32)).astype(np.int64)).astype(np.int64)

    def int(self, lo: int, hi: int) -> int:
        return int(self.ints(lo, hi, 1)[0])

    def perm(self, k: int) -> np.ndarray:
        return np.argsort(self.u64(k), kind="stable")


@dataclass
class CspModel:
    """Plain description of a CSP (X, D, C)."""

    n: int
    lo: list
    hi: list
    removed: list = field(default_factory=list)    # (var, value) pairs cut from D
    ne: list = field(default_factory=list)         # (x, y, c): x != y + c ; y = -1: x != c
    lin: list = field(default_factory=list)        # (coefs, vars, rhs): sum coefs*vars <= rhs
    alldiff: list = field(default_factory=list)    # [vars]
    tables: list = field(default_factory=list)     # (x, y, allowed bool matrix)
    name: str = ""
    alldiff_bc: list = field(default_factory=list) # [vars], bounds-consistent (oracle only)

    def n_constraints(self) -> int:
        return len(self.ne) + len(self.lin) + len(self.alldiff) + len(self.tables)


# --------------------------------------------------------------------------- fixed models

def worked_example(c1: str = "domain", c2: str = "lin") -> CspModel:
    """The worked example of Section 1.1: x1 in 1..5, x2 in 1..10, c1: x1 > 3, c2: x1 < x2.

    ``c1`` is posted as a domain cut ("domain") or as the unary row -x1 <= -4 ("lin");
    ``c2`` as the row x1 - x2 <= -1 ("lin") or as its tuple set ("table").
    Variable 0 is x1 and variable 1 is x2.
    """
    m = CspModel(n=2, lo=[1, 1], hi=[5, 10], name=f"worked-{c1}-{c2}")
    if c1 == "domain":
        m.removed += [(0, 1), (0, 2), (0, 3)]
    else:
        m.lin.append(([-1], [0], -4))
    if c2 == "lin":
        m.lin.append(([1, -1], [0, 1], -1))
    else:
        allowed = np.zeros((5, 10), dtype=bool)
        for a in range(1, 6):
            for b in range(1, 11):
                allowed[a - 1, b - 1] = a < b
        m.tables.append((0, 1, allowed))
    return m


def queens(N: int) -> CspModel:
    """N-queens with one variable per column (value = row): for i < j,
    x_i != x_j, x_i - x_j != i - j and x_i - x_j != j - i (3 * C(N, 2) ne constraints)."""
    m = CspModel(n=N, lo=[0] * N, hi=[N - 1] * N, name=f"queens-{N}")
    for i in range(N):
        for j in range(i + 1, N):
            m.ne.append((i, j, 0))
            m.ne.append((i, j, i - j))
            m.ne.append((i, j, j - i))
    return m


# --------------------------------------------------------------------------- model RB

def rb_tightness(alpha: float = 0.8, r: float = 0.7) -> float:
    """Tightness p = 1 - exp(-alpha / r) of model RB (Xu and Li 2000)."""
    return 1.0 - math.exp(-alpha / r)


def rb_threshold_tightness(n: int, d: int, r: float = 0.7) -> float:
    """The tightness at which the expected number of solutions of model RB is 1 (first-moment
    threshold): n ln d + r n ln n ln(1 - p) = 0, so p* = 1 - exp(-ln d / (r ln n))."""
    return 1.0 - math.exp(-math.log(d) / (r * math.log(n)))


def model_rb(seed: int, n: int, d: int, alpha: float = 0.8, r: float = 0.7,
             p: float | None = None) -> CspModel:
    """One model-RB instance: m = round(r n ln n) binary tables, each over two distinct
    variables drawn uniformly (scopes may repeat), each forbidding exactly round(p d^2)
    distinct value pairs drawn uniformly without replacement; domains are 0..d-1."""
    if p is None:
        p = rb_tightness(alpha, r)
    s = Stream(seed)
    m_cons = int(math.floor(r * n * math.log(n) + 0.5))
    t = int(math.floor(p * d * d + 0.5))
    xs = s.ints(0, n - 1, m_cons)
    ys = s.ints(0, n - 2, m_cons)
    ys = ys + (ys >= xs)
    keys = s.u64(m_cons * d * d).reshape(m_cons, d * d)
    order = np.argsort(keys, axis=1, kind="stable")[:, :t]
    forb = np.zeros((m_cons, d * d), dtype=bool)
    np.put_along_axis(forb, order, True, axis=1)
    allowed = ~forb.reshape(m_cons, d, d)
    model = CspModel(n=n, lo=[0] * n, hi=[d - 1] * n, name=f"rb-n{n}-d{d}-s{seed & 0xffff:04x}")
    model.tables = [(int(xs[k]), int(ys[k]), allowed[k]) for k in range(m_cons)]
    return model


def rb_batch(count: int, n_range=(20, 60), d_range=(8, 32), config_id: int = CFG_RB,
             alpha: float = 0.8, r: float = 0.7, p: float | None = None, first: int = 0):
    """``count`` model-RB instances with n ~ U[n_range], d ~ U[d_range] (inclusive),
    each from its own derived seed."""
    out = []
    for i in range(first, first + count):
        sd = seed_for(config_id, i)
        s = Stream(sd ^ 0x5555)
        n = s.int(*n_range)
        d = s.int(*d_range)
        out.append(model_rb(sd, n, d, alpha, r, p))
    return out


# --------------------------------------------------------------------------- linear + alldiff

# Right-hand-side position between row minimum and maximum.  Measured on dev seeds with the
# GPU search (first solution, 30 M nodes each): theta <= 0.15 fails at the root, theta in
# [0.2, 0.45] leaves most instances undecided, theta = 0.5 finds a solution for most within
# ~1e5 nodes.  0.5 is the frozen value; instances a search cannot decide are reported as such.
LINAD_THETA = 0.5


def lin_alldiff(seed: int, n: int = 200, dmax: int = 255, rows: int = 60, kmin: int = 5,
                kmax: int = 20, groups: int = 20, gsize: int = 10,
                theta: float = LINAD_THETA) -> CspModel:
    """Mixed instance: n vars on 0..dmax; ``groups`` disjoint alldifferent groups of ``gsize``
    vars (a seeded permutation cut in consecutive pieces); ``rows`` linear rows of k ~ U[kmin, kmax]
    distinct vars with coefficients uniform on {-10..-1, 1..10} and
    rhs = rowmin + floor(theta * (rowmax - rowmin)), rowmin/rowmax over the domain bounds."""
    s = Stream(seed)
    m = CspModel(n=n, lo=[0] * n, hi=[dmax] * n, name=f"linad-s{seed & 0xffff:04x}")
    perm = s.perm(n)
    for g in range(groups):
        m.alldiff.append([int(v) for v in perm[g * gsize:(g + 1) * gsize]])
    for _ in range(rows):
        k = s.int(kmin, kmax)
        vars_ = [int(v) for v in s.perm(n)[:k]]
        raw = s.ints(0, 19, k)
        coefs = [int(v - 10) if v < 10 else int(v - 9) for v in raw]
        rowmin = sum(a * dmax for a in coefs if a < 0)
        rowmax = sum(a * dmax for a in coefs if a > 0)
        rhs = rowmin + int(math.floor(theta * (rowmax - rowmin)))
        m.lin.append((coefs, vars_, rhs))
    return m


def linad_batch(count: int, theta: float = LINAD_THETA, config_id: int = CFG_LINAD,
                first: int = 0, **kw):
    return [lin_alldiff(seed_for(config_id, i), theta=theta, **kw)
            for i in range(first, first + count)]


# --------------------------------------------------------------------------- tiny random CSPs

def random_tiny(seed: int, n_max: int = 6, d_max: int = 5, kinds=("ne", "lin", "alldiff", "table"),
                density: float = 1.0) -> CspModel:
    """Small random CSP with every constraint kind, for brute-force agreement tests.
    Domains are ranges inside [-2, 7] with random holes; rows may repeat a variable and
    carry zero coefficients (merged and dropped when posted)."""
    s = Stream(seed)
    n = s.int(1, n_max)
    lo, hi = [], []
    for _ in range(n):
        a = s.int(-2, 3)
        lo.append(a)
        hi.append(a + s.int(0, d_max - 1))
    m = CspModel(n=n, lo=lo, hi=hi, name=f"tiny-{seed & 0xffffffff:08x}")
    for i in range(n):
        if hi[i] > lo[i] and s.int(0, 3) == 0:
            m.removed.append((i, s.int(lo[i], hi[i])))
    ncons = int(s.int(0, 2 + int(density * 2 * n)))
    for _ in range(ncons):
        kind = kinds[s.int(0, len(kinds) - 1)]
        if kind == "ne":
            x = s.int(0, n - 1)
            if n == 1 or s.int(0, 4) == 0:
                m.ne.append((x, -1, s.int(-2, 7)))
            else:
                y = s.int(0, n - 2)
                y += y >= x
                m.ne.append((x, y, s.int(-2, 2)))
        elif kind == "lin":
            k = s.int(1, 4)
            vars_ = [s.int(0, n - 1) for _ in range(k)]
            coefs = [s.int(-3, 3) for _ in range(k)]
            mid = sum(a * (lo[v] + hi[v]) // 2 for a, v in zip(coefs, vars_))
            m.lin.append((coefs, vars_, mid + s.int(-3, 3)))
        elif kind == "alldiff":
            if n < 2:
                continue
            k = s.int(2, min(4, n))
            m.alldiff.append([int(v) for v in s.perm(n)[:k]])
        else:
            if n < 2:
                continue
            x = s.int(0, n - 1)
            y = s.int(0, n - 2)
            y += y >= x
            sx, sy = hi[x] - lo[x] + 1, hi[y] - lo[y] + 1
            thr = s.int(1, 3)
            allowed = (s.ints(0, 3, sx * sy) >= thr).reshape(sx, sy)
            m.tables.append((x, y, allowed))
    return m


# ----------------------------------------------------------------------------- optimisation

def objective_weights(seed: int, n: int, wmin: int = 1, wmax: int = 9):
    """Objective minimise sum_i w_i x_i with w_i uniform on [wmin, wmax]: (coefs, vars)."""
    s = Stream(seed_for(CFG_LNS_OBJ, seed))
    return [int(w) for w in s.ints(wmin, wmax, n)], list(range(n))


def relax_masks(n: int, copies: int, frac: float, round_id: int, seed: int) -> np.ndarray:
    """Neighbourhoods of one search round: (copies, n) booleans, True = the variable is reset
    to its root domain.  Each variable is reset with probability frac (a uniform draw on
    [0, 2^32) below frac * 2^32); a copy that resets none resets one drawn variable."""
    s = Stream(seed_for(CFG_LNS_RELAX, (seed & 0xffffffff) ^ (round_id << 20)))
    u = (s.u64(copies * n) >> np.uint64(32)).reshape(copies, n)
    masks = u < np.uint64(int(frac * 4294967296.0))
    pick = s.ints(0, n - 1, copies)
    for c in range(copies):
        if not masks[c].any():
            masks[c, pick[c]] = True
    return masks


def small_optimisation(seed: int, n: int = 9, d: int = 9, rows: int = 3):
    """A small optimisation problem for exact checks: n vars on 0..d-1, one alldifferent over
    all of them, `rows` linear rows (as in lin_alldiff, theta 0.6), weights on [1, 9]."""
    m = lin_alldiff(seed, n=n, dmax=d - 1, rows=rows, kmin=2, kmax=min(5, n), groups=1, gsize=n,
                    theta=0.6)
    m.name = f"opt-s{seed & 0xffff:04x}"
    return m, objective_weights(seed, n)

