"""FlatZinc-subset front end (host only): parsed problems against the oracle and against the
models they were written from.  The FlatZinc texts are written here or by flatzinc.write."""
import numpy as np
import pytest

from oracle import lns_ref as L
from oracle import oracle as O
from paper_1909_09213_gb300 import flatzinc as F
from paper_1909_09213_gb300 import instances as I


def queens_fzn(N):
    """N-queens in the usual flat form: rows 1..N, one alldifferent, two diagonal int_lin_ne
    per pair."""
    out = [f"var 1..{N}: q{i};" for i in range(1, N + 1)]
    qs = ", ".join(f"q{i}" for i in range(1, N + 1))
    out.append(f"array [1..{N}] of var int: q :: output_array([1..{N}]) = [{qs}];")
    out.append("constraint all_different_int(q);")
    for i in range(1, N + 1):
        for j in range(i + 1, N + 1):
            out.append(f"constraint int_lin_ne([1, -1], [q{i}, q{j}], {i - j});")
            out.append(f"constraint int_lin_ne([1, -1], [q[{i}], q[{j}]], {j - i});")
    out.append("solve satisfy;")
    return "\n".join(out) + "\n"


WORKED = """
% the worked example of Section 1.1: x1 in 1..5, x2 in 1..10, x1 > 3, x1 < x2
var 1..5: x1 :: output_var;
var 1..10: x2 :: output_var;
constraint int_lt(3, x1);
constraint int_lt(x1, x2);
solve satisfy;
"""


def count(model):
    r = O.solve(O.OracleModel(model), variant=1)
    return r.solutions, r.hash_sum, r.hash_xor


def test_worked_example_has_eleven_solutions():
    p = F.parse(WORKED)
    assert p.names == ["x1", "x2"] and p.solve == "satisfy"
    assert count(p.model)[0] == 11


@pytest.mark.parametrize("N,want", [(4, 2), (6, 4), (8, 92)])
def test_queens_counts(N, want):
    p = F.parse(queens_fzn(N))
    assert p.model.n == N and len(p.model.alldiff) == 1 and len(p.model.ne) == N * (N - 1)
    assert count(p.model)[0] == want


@pytest.mark.parametrize("k", range(40))
def test_write_then_parse_keeps_the_solution_set(k):
    m = I.random_tiny(I.seed_for(I.CFG_TINY, 91000 + k))
    p = F.parse(F.write(m))

    def values(mm, i):
        cut = {v for (x, v) in mm.removed if x == i}
        return [v for v in range(mm.lo[i], mm.hi[i] + 1) if v not in cut]

    assert p.model.n == m.n
    for i in range(m.n):
        if values(m, i):                    # an empty domain is written as an unsatisfiable row
            assert values(p.model, i) == values(m, i)
    assert count(p.model) == count(m)


def test_set_domains_tables_and_params():
    text = """
    int: k = 2;
    array [1..4] of int: pairs = [0, 1, 2, 0];
    var {0, 2, 3}: a;
    var 0..3: b;
    constraint table_int([a, b], pairs);
    constraint int_ne(b, k);
    solve satisfy;
    """
    p = F.parse(text)
    assert sorted(p.model.removed) == [(0, 1)]
    r = O.solve(O.OracleModel(p.model), cap=10, variant=1)
    # (a, b) in {(0, 1), (2, 0)}, b != 2
    assert sorted(map(tuple, r.sols.tolist())) == [(0, 1), (2, 0)]


def test_lin_eq_and_le_rows():
    text = """
    var 0..9: x; var 0..9: y; var 0..30: s;
    constraint int_lin_eq([1, 2, -1], [x, y, s], 0);
    constraint int_le(s, 5);
    constraint int_eq(x, 1);
    solve satisfy;
    """
    p = F.parse(text)
    r = O.solve(O.OracleModel(p.model), cap=100, variant=1)
    got = sorted(map(tuple, r.sols.tolist()))
    assert got == [(1, y, 1 + 2 * y) for y in range(0, 3)]


def test_minimize_reads_the_objective():
    # an objective variable tied to a weighted sum over a permutation
    w = [4, 1, 3]
    text = """
    var 0..2: a; var 0..2: b; var 0..2: c; var 0..40: f;
    constraint all_different_int([a, b, c]);
    constraint int_lin_eq([4, 1, 3, -1], [a, b, c, f], 0);
    solve minimize f;
    """
    p = F.parse(text)
    assert p.solve == "minimize" and p.objective == ([1], [3])
    best, _ = L.optimum(p.model, p.objective)
    assert best == sum(k * wk for k, wk in enumerate(sorted(w, reverse=True)))
    q = F.parse(text.replace("minimize", "maximize"))
    best_max, _ = L.optimum(q.model, q.objective)
    assert -best_max == sum(k * wk for k, wk in enumerate(sorted(w)))


@pytest.mark.parametrize("bad", [
    "var 0..3: x; var 0..3: y; constraint int_times(x, y, x); solve satisfy;",
    "var float: f; solve satisfy;",
    "var 0..3: x; var int: y = x; solve satisfy;",
    "var 0..3: x; var 0..3: y; var 0..3: z; constraint table_int([x, y, z], [0, 0, 0]); solve satisfy;",
    "var 0..3: x; var 0..3: y; var 0..3: z; constraint int_lin_ne([1, 1, 1], [x, y, z], 3); solve satisfy;",
    "var 0..300: x; solve satisfy;",
    "var 0..3: x; constraint int_ne(x, y); solve satisfy;",
    "var 0..3: x;",
])
def test_outside_the_subset_is_rejected(bad):
    with pytest.raises(ValueError):
        F.parse(bad)


def test_solution_output_format():
    p = F.parse(queens_fzn(4))
    s = F.format_solution(p, np.array([2, 4, 1, 3]))
    assert s.splitlines() == ["q = array1d(1..4, [2, 4, 1, 3]);", "----------"]
    w = F.parse(WORKED)
    assert F.format_solution(w, [4, 7]).splitlines() == ["x1 = 4;", "x2 = 7;", "----------"]


# ---------------------------------------------------------------------------- booleans, reification

def _solutions(text, n_orig, functional=True):
    """Solutions of the parsed model projected on its first n_orig (declared) variables."""
    p = F.parse(text)
    r = O.solve(O.OracleModel(p.model), cap=1 << 16, variant=1)
    assert r.solutions < 1 << 16
    proj = sorted({tuple(int(v) for v in s[:n_orig]) for s in r.sols})
    if functional:                           # hidden variables are functions of the declared ones
        assert len(proj) == r.solutions
    return proj


def _enumerate(doms, pred):
    import itertools
    return sorted(t for t in itertools.product(*doms) if pred(*t))


R4, B = range(0, 4), range(0, 2)
CASES = [
    ("var 0..3: x; var 0..3: y; var bool: r; constraint int_le_reif(x, y, r);",
     [R4, R4, B], lambda x, y, r: r == (x <= y)),
    ("var 0..3: x; var 0..3: y; var bool: r; constraint int_lt_reif(x, y, r);",
     [R4, R4, B], lambda x, y, r: r == (x < y)),
    ("var 0..3: x; var 0..3: y; var bool: r; constraint int_eq_reif(x, y, r);",
     [R4, R4, B], lambda x, y, r: r == (x == y)),
    ("var 0..3: x; var 0..3: y; var bool: r; constraint int_ne_reif(x, y, r);",
     [R4, R4, B], lambda x, y, r: r == (x != y)),
    ("var 0..3: x; var bool: r; constraint int_eq_reif(x, 2, r);",
     [R4, B], lambda x, r: r == (x == 2)),
    ("var 0..3: x; var 0..3: y; var bool: r; constraint int_lin_le_reif([2, -1], [x, y], 1, r);",
     [R4, R4, B], lambda x, y, r: r == (2 * x - y <= 1)),
    ("var 0..3: x; var 0..3: y; var bool: r; constraint int_lin_eq_reif([1, 1], [x, y], 3, r);",
     [R4, R4, B], lambda x, y, r: r == (x + y == 3)),
    ("var 0..3: x; var 0..3: y; var bool: r; constraint int_lin_ne_reif([1, -2], [x, y], 0, r);",
     [R4, R4, B], lambda x, y, r: r == (x - 2 * y != 0)),
    ("var 0..3: x; var 0..3: y; constraint int_le_reif(x, y, true);",
     [R4, R4], lambda x, y: x <= y),
    ("var 0..3: x; var 0..3: y; constraint int_eq_reif(x, y, false);",
     [R4, R4], lambda x, y: x != y),
    ("var bool: a; var bool: b; var bool: c; constraint bool_clause([a, b], [c]);",
     [B, B, B], lambda a, b, c: a or b or not c),
    ("var bool: a; var bool: b; var bool: r; constraint array_bool_or([a, b], r);",
     [B, B, B], lambda a, b, r: r == (a or b)),
    ("var bool: a; var bool: b; var bool: r; constraint array_bool_and([a, b], r);",
     [B, B, B], lambda a, b, r: r == (a and b)),
    ("var bool: a; var bool: b; constraint array_bool_or([a, b], true);",
     [B, B], lambda a, b: a or b),
    ("var bool: a; var bool: b; constraint array_bool_and([a, b], false);",
     [B, B], lambda a, b: not (a and b)),
    ("var bool: a; var 0..1: i; constraint bool2int(a, i);",
     [B, B], lambda a, i: a == i),
    ("var bool: a; var bool: b; constraint bool_not(a, b);",
     [B, B], lambda a, b: a != b),
    ("var bool: a; var bool: b; var bool: r; constraint bool_eq_reif(a, b, r);",
     [B, B, B], lambda a, b, r: r == (a == b)),
    ("var bool: a; var bool: b; constraint bool_lt(a, b);",
     [B, B], lambda a, b: a < b),
    ("var bool: a; var bool: b; var bool: c; constraint bool_lin_le([1, 1, 1], [a, b, c], 1);",
     [B, B, B], lambda a, b, c: a + b + c <= 1),
    ("var 0..3: x; var 0..3: y = x; var int: z = 2; constraint int_ne(x, z);",
     [R4, R4, range(2, 3)], lambda x, y, z: y == x and x != 2),
    ("var 0..3: x; var 0..3: y; var 0..6: z; constraint int_plus(x, y, z);",
     [R4, R4, range(0, 7)], lambda x, y, z: z == x + y),
    ("var 0..3: x; var 0..3: y; var -3..3: z; constraint int_minus(x, y, z);",
     [R4, R4, range(-3, 4)], lambda x, y, z: z == x - y),
    ("var 0..3: x; var 0..9: z; constraint int_times(3, x, z);",
     [R4, range(0, 10)], lambda x, z: z == 3 * x),
    ("var -3..3: x; var 0..2: y; constraint int_abs(x, y);",
     [range(-3, 4), range(0, 3)], lambda x, y: y == abs(x)),
    ("var 0..4: i; var 0..9: v; constraint array_int_element(i, [5, 2, 7], v);",
     [range(0, 5), range(0, 10)], lambda i, v: 1 <= i <= 3 and v == [5, 2, 7][i - 1]),
    ("var 0..3: i; constraint array_int_element(i, [4, 6, 4], 4);",
     [R4], lambda i: i in (1, 3)),
    ("var -2..3: x; var 0..3: y; var -2..3: z; constraint int_max(x, y, z);",
     [range(-2, 4), R4, range(-2, 4)], lambda x, y, z: z == max(x, y), False),
    ("var -2..3: x; var 0..3: y; var -2..3: z; constraint int_min(x, y, z);",
     [range(-2, 4), R4, range(-2, 4)], lambda x, y, z: z == min(x, y), False),
    ("var 0..5: x; constraint set_in(x, {1, 3, 9});",
     [range(0, 6)], lambda x: x in (1, 3)),
    ("var 0..5: x; constraint set_in(x, 2..4);",
     [range(0, 6)], lambda x: 2 <= x <= 4),
]


@pytest.mark.parametrize("k", range(len(CASES)))
def test_boolean_and_reified_constraints(k):
    text, doms, pred = CASES[k][:3]
    functional = CASES[k][3] if len(CASES[k]) > 3 else True    # max/min: a free choice when equal
    assert _solutions(text + " solve satisfy;", len(doms), functional) == _enumerate(doms, pred)


def test_bool_output_and_arrays():
    text = """
    array [1..3] of bool: pat = [true, false, true];
    var bool: a :: output_var;
    var bool: b;
    array [1..2] of var bool: ab :: output_array([1..2]) = [a, b];
    constraint bool_clause([a], [b]);
    solve satisfy;
    """
    p = F.parse(text)
    assert p.bools == {0, 1}
    out = F.format_solution(p, [1, 0])
    assert out.splitlines() == ["a = true;", "ab = array1d(1..2, [true, false]);", "----------"]


def test_minimize_marks_the_variables_a_neighbourhood_must_reset():
    text = """
    var 0..3: a; var 0..3: b;
    var 0..20: cost :: output_var :: is_defined_var;
    var bool: t :: var_is_introduced;
    constraint int_lin_eq([2, 3, -1], [a, b, cost], 0) :: defines_var(cost);
    constraint int_le_reif(a, b, t);
    constraint int_eq_reif(a, 2, t);
    solve minimize cost;
    """
    p = F.parse(text)
    names = p.names
    assert [names[i] for i in p.free] == ["cost", "t"] + [n for n in names if n.startswith("__aux")]
    assert p.objective == ([1], [names.index("cost")])
    best, _ = L.optimum(p.model, p.objective)
    # t = (a <= b) = (a == 2): (a, b) in {(0..1, 0..a-1)} U {(2, 2..3)}; cheapest: a = 1, b = 0
    assert best == 2


def test_strings_and_comments_in_output_items():
    text = """
    var 1..3: x :: output_var;   % a comment; with a semicolon
    constraint int_ne(x, 2);
    solve satisfy;
    output ["x = ", show(x), ";\\n", "100%"];
    """
    p = F.parse(text)
    assert p.names == ["x"] and count(p.model)[0] == 2
