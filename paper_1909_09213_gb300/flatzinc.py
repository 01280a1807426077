"""FlatZinc-subset front end: the problem is parsed on the host (Section 2.1: the CPU reads
and builds the problem, the GPU solves it) into the CSP triple of Section 1.1.

Supported subset (anything else is rejected with a ValueError naming the item):

* variables: ``var lo..hi: x;``, ``var {v1, v2, ...}: x;`` (integer domains of at most 256
  consecutive values), ``var bool: b;`` (0/1, printed false/true), ``var int: x = 3;`` and
  ``var ...: x = y;`` (fixed values and aliases); parameter arrays ``array [1..k] of int: a =
  [...];`` (also of bool) and variable arrays ``array [1..k] of var int: xs = [x1, ...];``
  (with ``output_array``);
* constraints: ``int_ne``, ``int_eq``, ``int_le``, ``int_lt``, ``int_lin_ne`` (the forms
  x != c and a x - a y != c), ``int_lin_le``, ``int_lin_eq`` (two rows), ``all_different_int``
  (also ``fzn_all_different_int``), ``table_int`` over two variables; the boolean
  ``bool_eq/ne/le/lt``, ``bool2int``, ``bool_not``, ``bool_clause``, ``array_bool_or``,
  ``array_bool_and``, ``bool_lin_le/eq``; and the reified ``int_le/lt/eq/ne_reif``,
  ``bool_le/lt/eq_reif``, ``int_lin_le/eq/ne_reif`` (linear rows with big-M terms from the
  domain bounds, exact for these bounded domains; reified equalities add two hidden 0/1
  variables); ``int_plus``, ``int_minus``, ``int_times`` with a constant factor,
  ``int_max``, ``int_min`` (one hidden 0/1 variable), ``int_abs``, ``int_negate`` and
  ``array_int_element`` (binary tables of the function), ``set_in``;
* ``solve satisfy;``, ``solve minimize x;``, ``solve maximize x;``.

Every search step then runs in the library (``cubics.Csp``, ``lns.LNS``); this module only
turns text into a ``CspModel`` and solutions back into FlatZinc output.
"""
from __future__ import annotations

import re
import sys
from dataclasses import dataclass, field

from .instances import CspModel


@dataclass
class FznProblem:
    model: CspModel
    names: list                                    # variable index -> name
    index: dict                                    # name -> variable index
    outputs: list = field(default_factory=list)   # ("var", name) | ("array", name, [dims], [idx])
    solve: str = "satisfy"                         # satisfy | minimize | maximize
    objective: tuple | None = None                 # (coefs, vars) to minimise
    bools: set = field(default_factory=set)        # bool variables (printed true / false)
    free: list = field(default_factory=list)       # variables a neighbourhood always resets:
                                                   # introduced / defined, hidden, the objective


_INT = r"-?\d+"


def _split_statements(text: str):
    """Statements separated by ';' outside brackets and string literals; comments (% to the
    end of the line, outside string literals) removed."""
    lines = []
    for ln in text.splitlines():
        quoted = False
        for k, ch in enumerate(ln):
            if ch == '"':
                quoted = not quoted
            elif ch == "%" and not quoted:
                ln = ln[:k]
                break
        lines.append(ln)
    body = " ".join(lines)
    out, depth, cur, quoted = [], 0, [], False
    for ch in body:
        if ch == '"':
            quoted = not quoted
        elif quoted:
            pass
        elif ch in "[({":
            depth += 1
        elif ch in "])}":
            depth -= 1
        if ch == ";" and depth == 0 and not quoted:
            s = "".join(cur).strip()
            if s:
                out.append(s)
            cur = []
        else:
            cur.append(ch)
    if "".join(cur).strip():
        raise ValueError("missing ';' after the last statement")
    return out


def _strip_annotations(s: str) -> str:
    """Remove '::' annotations that are not inside brackets."""
    depth = 0
    for i, ch in enumerate(s):
        if ch in "[({":
            depth += 1
        elif ch in "])}":
            depth -= 1
        elif ch == ":" and depth == 0 and s[i:i + 2] == "::":
            return s[:i].strip()
    return s.strip()


def _args(s: str):
    """Top-level comma-separated arguments of 'name(args)'."""
    out, depth, cur = [], 0, []
    for ch in s:
        if ch in "[({":
            depth += 1
        elif ch in "])}":
            depth -= 1
        if ch == "," and depth == 0:
            out.append("".join(cur).strip())
            cur = []
        else:
            cur.append(ch)
    if "".join(cur).strip():
        out.append("".join(cur).strip())
    return out


class _Builder:
    def __init__(self):
        self.lo, self.hi, self.removed = [], [], []
        self.names, self.index = [], {}
        self.params = {}                   # name -> int or list of ints
        self.var_arrays = {}               # name -> list of var indices
        self.model = None
        self.outputs = []
        self.bools = set()                 # indices of bool variables (printed true/false)
        self.introduced = set()            # variables annotated as introduced / defined
        self.aliases = []                  # (var, token) from `var ...: x = token`

    # -- terms
    def var(self, tok: str) -> int:
        tok = tok.strip()
        m = re.fullmatch(r"([A-Za-z_][\w]*)\[(\d+)\]", tok)
        if m:
            arr = self.var_arrays.get(m.group(1))
            if arr is None:
                raise ValueError(f"unknown variable array {m.group(1)}")
            return arr[int(m.group(2)) - 1]
        if tok not in self.index:
            raise ValueError(f"unknown variable {tok}")
        return self.index[tok]

    def is_int(self, tok: str) -> bool:
        tok = tok.strip()
        return (re.fullmatch(_INT, tok) is not None or tok in ("true", "false") or
                (tok in self.params and isinstance(self.params[tok], int)))

    def int(self, tok: str) -> int:
        tok = tok.strip()
        if re.fullmatch(_INT, tok):
            return int(tok)
        if tok in ("true", "false"):
            return 1 if tok == "true" else 0
        if tok in self.params and isinstance(self.params[tok], int):
            return self.params[tok]
        raise ValueError(f"expected an integer, got {tok}")

    def list_of(self, tok: str, kind: str):
        tok = tok.strip()
        if tok.startswith("["):
            items = _args(tok[1:-1]) if tok[1:-1].strip() else []
            return [self.int(t) for t in items] if kind == "int" else [self.var(t) for t in items]
        if kind == "int" and isinstance(self.params.get(tok), list):
            return list(self.params[tok])
        if kind == "var" and tok in self.var_arrays:
            return list(self.var_arrays[tok])
        raise ValueError(f"expected an array of {kind}, got {tok}")

    # -- declarations
    def declare(self, name: str, values):
        if name in self.index:
            raise ValueError(f"variable {name} declared twice")
        lo, hi = min(values), max(values)
        if hi - lo + 1 > 256:
            raise ValueError(f"domain of {name} spans more than 256 values")
        i = len(self.names)
        self.index[name] = i
        self.names.append(name)
        self.lo.append(lo)
        self.hi.append(hi)
        present = set(values)
        self.removed += [(i, v) for v in range(lo, hi + 1) if v not in present]
        return i


def parse(text: str) -> FznProblem:
    b = _Builder()
    constraints, solve = [], None
    for st in _split_statements(text):
        head = st.split(None, 1)[0]
        if head == "predicate":
            raise ValueError("predicate declarations are outside the supported subset")
        if head == "constraint":
            constraints.append(_strip_annotations(st[len("constraint"):]))
            continue
        if head == "solve":
            solve = _strip_annotations(st[len("solve"):]).strip()
            continue
        if head == "var":
            m = re.fullmatch(r"var\s+(.+?)\s*:\s*([A-Za-z_]\w*)\s*(::[^=]*)?(=\s*(.+))?", st)
            if not m:
                raise ValueError(f"cannot read declaration: {st}")
            dom, name, ann = m.group(1).strip(), m.group(2), m.group(3) or ""
            r = re.fullmatch(rf"({_INT})\s*\.\.\s*({_INT})", dom)
            if r:
                values = list(range(int(r.group(1)), int(r.group(2)) + 1))
            elif dom.startswith("{") and dom.endswith("}"):
                values = [int(t) for t in _args(dom[1:-1])]
            elif dom == "bool":
                values = [0, 1]
            elif dom == "int" and m.group(5) is not None and b.is_int(m.group(5)):
                values = [b.int(m.group(5))]               # a constant declared as a variable
            else:
                raise ValueError(f"unsupported domain for {name}: {dom}")
            if not values:
                raise ValueError(f"empty domain for {name}")
            i = b.declare(name, values)
            if dom == "bool":
                b.bools.add(i)
            if m.group(5) is not None:
                b.aliases.append((i, m.group(5).strip()))
            if "output_var" in ann:
                b.outputs.append(("var", name))
            if "var_is_introduced" in ann or "is_defined_var" in ann:
                b.introduced.add(i)
            continue
        if head == "array":
            m = re.fullmatch(r"array\s*\[(.+?)\]\s*of\s+(var\s+)?(int|[^:]+?)\s*:\s*([A-Za-z_]\w*)\s*"
                             r"(::.*?)?\s*=\s*(\[.*\])", st)
            if not m:
                raise ValueError(f"cannot read array: {st}")
            is_var, name, ann, body = m.group(2) is not None, m.group(4), m.group(5) or "", m.group(6)
            if is_var:
                b.var_arrays[name] = b.list_of(body, "var")
                o = re.search(r"output_array\s*\(\s*\[(.*?)\]\s*\)", ann)
                if o:
                    dims = [tuple(int(x) for x in d.split("..")) for d in _args(o.group(1))]
                    b.outputs.append(("array", name, dims, b.var_arrays[name]))
            else:
                b.params[name] = b.list_of(body, "int")
            continue
        if re.fullmatch(rf"int\s*:\s*[A-Za-z_]\w*\s*=\s*{_INT}", st):
            name, val = re.fullmatch(rf"int\s*:\s*([A-Za-z_]\w*)\s*=\s*({_INT})", st).groups()
            b.params[name] = int(val)
            continue
        if head == "output":
            continue
        raise ValueError(f"statement outside the supported subset: {st}")
    if solve is None:
        raise ValueError("no solve item")

    model = CspModel(n=len(b.names), lo=list(b.lo), hi=list(b.hi), removed=list(b.removed),
                     name="fzn")
    for i, tok in b.aliases:                       # var ...: x = 3  /  var ...: x = y
        _post(b, model, f"int_eq({b.names[i]}, {tok})")
    for c in constraints:
        _post(b, model, c)
    prob = FznProblem(model=model, names=list(b.names), index=dict(b.index), outputs=b.outputs,
                      bools=set(b.bools))
    if solve == "satisfy":
        prob.solve = "satisfy"
    else:
        m = re.fullmatch(r"(minimize|maximize)\s+(.+)", solve)
        if not m:
            raise ValueError(f"unsupported solve item: {solve}")
        v = b.var(m.group(2))
        prob.solve = m.group(1)
        prob.objective = ([1], [v]) if m.group(1) == "minimize" else ([-1], [v])
        hidden = {i for i, nm in enumerate(prob.names) if nm.startswith("__aux")}
        prob.free = sorted(b.introduced | hidden | {v})
    if not prob.outputs:
        prob.outputs = [("var", n) for n in b.names]
    return prob


class _Poster:
    """Posts FlatZinc constraints as the library's constraint kinds.  Reified comparisons
    become linear rows with big-M terms taken from the domain bounds (exact for bounded
    integer domains); an equality's reification goes through two auxiliary booleans."""

    def __init__(self, b: _Builder, model: CspModel):
        self.b, self.m = b, model

    # -- helpers
    def term(self, tok):
        """(1, var) for a variable token, (None, value) for a constant."""
        return (None, self.b.int(tok)) if self.b.is_int(tok) else (1, self.b.var(tok))

    def row(self, coefs, vars_, rhs):
        self.m.lin.append((list(coefs), list(vars_), int(rhs)))

    def eq_row(self, coefs, vars_, rhs):
        self.row(coefs, vars_, rhs)
        self.row([-a for a in coefs], vars_, -rhs)

    def aux_bool(self):
        i = self.m.n
        name = f"__aux{i}"
        self.m.n += 1
        self.m.lo.append(0)
        self.m.hi.append(1)
        self.b.index[name] = i
        self.b.names.append(name)
        return i

    def bounds(self, coefs, vars_):
        lo = sum(min(a * self.m.lo[v], a * self.m.hi[v]) for a, v in zip(coefs, vars_))
        hi = sum(max(a * self.m.lo[v], a * self.m.hi[v]) for a, v in zip(coefs, vars_))
        return lo, hi

    def linear(self, pairs):
        """pairs of (coef, token) -> (coefs, vars, constant part)"""
        coefs, vars_, const = [], [], 0
        for a, tok in pairs:
            c, v = self.term(tok)
            if c is None:
                const += a * v
            else:
                coefs.append(a)
                vars_.append(v)
        return coefs, vars_, const

    def reif_le(self, coefs, vars_, c, r_tok):
        """r <-> (sum coefs * vars <= c)"""
        if self.b.is_int(r_tok):
            if self.b.int(r_tok):
                self.row(coefs, vars_, c)
            else:
                self.row([-a for a in coefs], vars_, -(c + 1))
            return
        r = self.b.var(r_tok)
        smin, smax = self.bounds(coefs, vars_)
        # r = 1 -> S <= c:       S + (smax - c) r <= smax
        self.row(list(coefs) + [smax - c], list(vars_) + [r], smax)
        # r = 0 -> S >= c + 1:  -S - (c + 1 - smin) r <= -(c + 1)
        self.row([-a for a in coefs] + [-(c + 1 - smin)], list(vars_) + [r], -(c + 1))

    def reif_eq(self, coefs, vars_, c, r_tok, negate=False):
        """r <-> (S == c) (negate: r <-> (S != c)) through p <-> (S <= c), q <-> (S >= c);
        p or q always holds, so S == c is p and q"""
        p, q = self.aux_bool(), self.aux_bool()
        self.reif_le(coefs, vars_, c, self.b.names[p])
        self.reif_le([-a for a in coefs], vars_, -c, self.b.names[q])
        if self.b.is_int(r_tok):
            if bool(self.b.int(r_tok)) != negate:
                self.row([-1, -1], [p, q], -2)           # p = q = 1
            else:
                self.row([1, 1], [p, q], 1)              # not both
            return
        r = self.b.var(r_tok)
        if not negate:                                   # r = p and q
            self.row([1, -1], [r, p], 0)
            self.row([1, -1], [r, q], 0)
            self.row([1, 1, -1], [p, q, r], 1)
        else:                                            # r = not (p and q)
            self.row([-1, -1], [r, p], -1)               # r >= 1 - p
            self.row([-1, -1], [r, q], -1)               # r >= 1 - q
            self.row([1, 1, 1], [r, p, q], 2)            # p = q = 1 -> r = 0

    def function_table(self, x_tok, y_tok, f):
        """y = f(x) as a binary table over the domains (f(x) None: x has no image)"""
        b, model = self.b, self.m
        if b.is_int(x_tok):
            fx = f(b.int(x_tok))
            if fx is None:
                model.lin.append(([], [], -1))
            elif b.is_int(y_tok):
                if b.int(y_tok) != fx:
                    model.lin.append(([], [], -1))
            else:
                self.eq_row([1], [b.var(y_tok)], fx)
            return
        x = b.var(x_tok)
        if b.is_int(y_tok):
            yv = b.int(y_tok)
            model.removed += [(x, u) for u in range(model.lo[x], model.hi[x] + 1) if f(u) != yv]
            return
        y = b.var(y_tok)
        if x == y:
            model.removed += [(x, u) for u in range(model.lo[x], model.hi[x] + 1) if f(u) != u]
            return
        import numpy as np
        al = np.zeros((model.hi[x] - model.lo[x] + 1, model.hi[y] - model.lo[y] + 1), dtype=bool)
        for u in range(model.lo[x], model.hi[x] + 1):
            fu = f(u)
            if fu is not None and model.lo[y] <= fu <= model.hi[y]:
                al[u - model.lo[x], fu - model.lo[y]] = True
        model.tables.append((x, y, al))

    # -- constraints
    def post(self, c: str):
        b, model = self.b, self.m
        m = re.fullmatch(r"([A-Za-z_]\w*)\s*\((.*)\)", c)
        if not m:
            raise ValueError(f"cannot read constraint: {c}")
        name, args = m.group(1), _args(m.group(2))
        if name in ("int_ne", "bool_ne"):
            x, y = args
            if b.is_int(x) and b.is_int(y):
                if b.int(x) == b.int(y):
                    model.lin.append(([], [], -1))       # never satisfied
            elif b.is_int(y) or b.is_int(x):
                v, k = (x, y) if b.is_int(y) else (y, x)
                model.ne.append((b.var(v), -1, b.int(k)))
            else:
                model.ne.append((b.var(x), b.var(y), 0))
        elif name in ("int_eq", "int_le", "int_lt", "bool_eq", "bool_le", "bool_lt", "bool2int"):
            x, y = args
            coefs, vars_, const = self.linear([(1, x), (-1, y)])
            rhs = -const - (1 if name in ("int_lt", "bool_lt") else 0)
            if name in ("int_eq", "bool_eq", "bool2int"):
                self.eq_row(coefs, vars_, rhs)
            else:
                self.row(coefs, vars_, rhs)
        elif name == "bool_not":
            coefs, vars_, const = self.linear([(1, args[0]), (1, args[1])])
            self.eq_row(coefs, vars_, 1 - const)
        elif name in ("int_le_reif", "int_lt_reif", "bool_le_reif", "bool_lt_reif"):
            x, y, r = args
            coefs, vars_, const = self.linear([(1, x), (-1, y)])
            self.reif_le(coefs, vars_, -const - (1 if name.endswith("lt_reif") else 0), r)
        elif name in ("int_eq_reif", "int_ne_reif", "bool_eq_reif"):
            x, y, r = args
            coefs, vars_, const = self.linear([(1, x), (-1, y)])
            self.reif_eq(coefs, vars_, -const, r, negate=name == "int_ne_reif")
        elif name in ("int_lin_le", "int_lin_eq", "int_lin_ne", "bool_lin_le", "bool_lin_eq"):
            coefs, vars_, rhs = b.list_of(args[0], "int"), b.list_of(args[1], "var"), b.int(args[2])
            if len(coefs) != len(vars_):
                raise ValueError(f"{name}: {len(coefs)} coefficients for {len(vars_)} variables")
            if name.endswith("lin_le"):
                self.row(coefs, vars_, rhs)
            elif name.endswith("lin_eq"):
                self.eq_row(coefs, vars_, rhs)
            else:
                _lin_ne(model, coefs, vars_, rhs)
        elif name in ("int_lin_le_reif", "int_lin_eq_reif", "int_lin_ne_reif"):
            coefs, vars_, rhs = b.list_of(args[0], "int"), b.list_of(args[1], "var"), b.int(args[2])
            if len(coefs) != len(vars_):
                raise ValueError(f"{name}: {len(coefs)} coefficients for {len(vars_)} variables")
            if name == "int_lin_le_reif":
                self.reif_le(coefs, vars_, rhs, args[3])
            else:
                self.reif_eq(coefs, vars_, rhs, args[3], negate=name == "int_lin_ne_reif")
        elif name == "bool_clause":
            pos, neg = b.list_of(args[0], "var"), b.list_of(args[1], "var")
            # sum pos + sum (1 - neg) >= 1
            self.row([-1] * len(pos) + [1] * len(neg), pos + neg, len(neg) - 1)
        elif name in ("array_bool_or", "array_bool_and"):
            xs, r = b.list_of(args[0], "var"), args[1]
            k = len(xs)
            if b.is_int(r):
                if name == "array_bool_or":
                    self.row([-1] * k, xs, -1) if b.int(r) else self.row([1] * k, xs, 0)
                else:
                    self.row([-1] * k, xs, -k) if b.int(r) else self.row([1] * k, xs, k - 1)
                return
            rv = b.var(r)
            if name == "array_bool_or":                  # r = max(xs)
                for x in xs:
                    self.row([1, -1], [x, rv], 0)
                self.row([1] + [-1] * k, [rv] + xs, 0)
            else:                                        # r = min(xs)
                for x in xs:
                    self.row([1, -1], [rv, x], 0)
                self.row([1] * k + [-1], xs + [rv], k - 1)
        elif name in ("int_plus", "int_minus"):          # a + b = c  /  a - b = c
            a, bb, cc = args
            sign = 1 if name == "int_plus" else -1
            coefs, vars_, const = self.linear([(1, a), (sign, bb), (-1, cc)])
            self.eq_row(coefs, vars_, -const)
        elif name == "int_times":                        # a * b = c, one factor constant
            a, bb, cc = args
            if b.is_int(a) or b.is_int(bb):
                k, v = (b.int(a), bb) if b.is_int(a) else (b.int(bb), a)
                coefs, vars_, const = self.linear([(k, v), (-1, cc)])
                self.eq_row(coefs, vars_, -const)
            else:
                raise ValueError("int_times of two variables is outside the supported subset")
        elif name in ("int_abs", "int_negate"):          # b = |a|  /  b = -a: a binary table
            self.function_table(args[0], args[1], abs if name == "int_abs" else (lambda v: -v))
        elif name == "array_int_element":                # c = as[idx] (1-based): a binary table
            idx, arr, cc = args
            vals = b.list_of(arr, "int")
            self.function_table(idx, cc, lambda i: vals[i - 1] if 1 <= i <= len(vals) else None)
        elif name in ("int_max", "int_min"):             # c = max(a, b)  /  c = min(a, b)
            a, bb, cc = args
            sgn = 1 if name == "int_max" else -1
            # c >= a, c >= b (max) and c <= a or c <= b, chosen by a hidden 0/1 variable s
            for t in (a, bb):
                coefs, vars_, const = self.linear([(sgn, t), (-sgn, cc)])
                self.row(coefs, vars_, -const)
            s_ = self.aux_bool()
            for t, on in ((a, 1), (bb, 0)):
                coefs, vars_, const = self.linear([(sgn, cc), (-sgn, t)])
                lo, hi = self.bounds(coefs, vars_)
                big = max(hi + const, 0)
                # s = on -> sgn (c - t) <= 0, else relaxed by `big`
                self.row(coefs + [big if on else -big], vars_ + [s_], -const + (big if on else 0))
        elif name == "set_in":                           # x in {..} or x in a..b
            x, st = args
            if st.startswith("{"):
                keep = {b.int(t) for t in _args(st[1:-1])}
            else:
                r = re.fullmatch(rf"({_INT})\s*\.\.\s*({_INT})", st)
                if not r:
                    raise ValueError(f"set_in: unsupported set {st}")
                keep = set(range(int(r.group(1)), int(r.group(2)) + 1))
            v = b.var(x)
            model.removed += [(v, u) for u in range(model.lo[v], model.hi[v] + 1) if u not in keep]
        elif name in ("all_different_int", "fzn_all_different_int"):
            vars_ = b.list_of(args[0], "var")
            if len(set(vars_)) != len(vars_):
                raise ValueError("all_different_int over a repeated variable")
            model.alldiff.append(vars_)
        elif name == "table_int":
            vars_, flat = b.list_of(args[0], "var"), b.list_of(args[1], "int")
            if len(vars_) != 2 or vars_[0] == vars_[1]:
                raise ValueError("table_int is supported over two distinct variables only")
            if len(flat) % 2:
                raise ValueError("table_int: odd number of tuple entries")
            x, y = vars_
            import numpy as np
            al = np.zeros((model.hi[x] - model.lo[x] + 1, model.hi[y] - model.lo[y] + 1), dtype=bool)
            for a, c2 in zip(flat[0::2], flat[1::2]):
                if model.lo[x] <= a <= model.hi[x] and model.lo[y] <= c2 <= model.hi[y]:
                    al[a - model.lo[x], c2 - model.lo[y]] = True
            model.tables.append((x, y, al))
        else:
            raise ValueError(f"constraint {name} is outside the supported subset")


def _post(b: _Builder, model: CspModel, c: str):
    _Poster(b, model).post(c)


def _lin_ne(model: CspModel, coefs, vars_, rhs):
    """sum a_i x_i != rhs in the forms the library has: a x != c, a x - a y != c."""
    terms = {}
    for a, v in zip(coefs, vars_):
        terms[v] = terms.get(v, 0) + a
    terms = [(a, v) for v, a in terms.items() if a != 0]
    if not terms:
        if rhs == 0:
            model.lin.append(([], [], -1))
        return
    if len(terms) == 1:
        a, v = terms[0]
        if rhs % a == 0:
            model.ne.append((v, -1, rhs // a))
        return
    if len(terms) == 2 and terms[0][0] == -terms[1][0]:
        (a, x), (_, y) = terms
        # a x - a y != rhs  <=>  x != y + rhs / a  (nothing to post if a does not divide rhs)
        if rhs % a == 0:
            model.ne.append((x, y, rhs // a))
        return
    raise ValueError("int_lin_ne is supported as a x != c or a x - a y != c only")


# ----------------------------------------------------------------------------- writing

def write(model: CspModel, names=None, solve: str = "satisfy", objective=None) -> str:
    """FlatZinc text of a CspModel (int_ne as int_ne / int_lin_ne, rows as int_lin_le,
    alldifferent as all_different_int, tables as table_int)."""
    names = names or [f"x{i}" for i in range(model.n)]
    removed = {}
    for v, val in model.removed:
        removed.setdefault(v, set()).add(val)
    out = []
    for i in range(model.n):
        lo, hi = model.lo[i], model.hi[i]
        vals = [v for v in range(lo, hi + 1) if v not in removed.get(i, ())]
        dom = f"{lo}..{hi}" if len(vals) == hi - lo + 1 else "{" + ", ".join(map(str, vals)) + "}"
        if not vals:
            dom = f"{lo}..{hi}"
        out.append(f"var {dom}: {names[i]} :: output_var;")
    for i in range(model.n):
        lo, hi = model.lo[i], model.hi[i]
        if not [v for v in range(lo, hi + 1) if v not in removed.get(i, ())]:
            out.append(f"constraint int_lin_le([], [], -1);")        # an empty domain
    for x, y, c in model.ne:
        if y < 0:
            out.append(f"constraint int_ne({names[x]}, {c});")
        elif c == 0:
            out.append(f"constraint int_ne({names[x]}, {names[y]});")
        else:
            out.append(f"constraint int_lin_ne([1, -1], [{names[x]}, {names[y]}], {c});")
    for coefs, vars_, rhs in model.lin:
        out.append(f"constraint int_lin_le([{', '.join(map(str, coefs))}], "
                   f"[{', '.join(names[v] for v in vars_)}], {rhs});")
    for g in model.alldiff:
        out.append(f"constraint all_different_int([{', '.join(names[v] for v in g)}]);")
    for x, y, al in model.tables:
        pairs = []
        for a in range(len(al)):
            for c in range(len(al[a])):
                if al[a][c]:
                    pairs += [model.lo[x] + a, model.lo[y] + c]
        out.append(f"constraint table_int([{names[x]}, {names[y]}], [{', '.join(map(str, pairs))}]);")
    if solve == "satisfy":
        out.append("solve satisfy;")
    else:
        out.append(f"solve {solve} {names[objective]};")
    return "\n".join(out) + "\n"


def format_solution(prob: FznProblem, values) -> str:
    """One solution in FlatZinc output form, followed by the separator line."""
    def show(i):
        v = int(values[i])
        return ("true" if v else "false") if i in prob.bools else str(v)

    lines = []
    for o in prob.outputs:
        if o[0] == "var":
            lines.append(f"{o[1]} = {show(prob.index[o[1]])};")
        else:
            _, name, dims, idx = o
            d = ", ".join(f"{a}..{c}" for a, c in dims)
            lines.append(f"{name} = array{len(dims)}d({d}, [{', '.join(show(i) for i in idx)}]);")
    lines.append("----------")
    return "\n".join(lines)


def main(argv=None):
    """Solve a FlatZinc file on the GPU: all solutions (-a), or the first; minimize/maximize
    by parallel large neighbourhood search."""
    import argparse
    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("file")
    ap.add_argument("-a", "--all", action="store_true", help="all solutions")
    ap.add_argument("--cap", type=int, default=1000, help="solutions printed with -a")
    ap.add_argument("--time", type=float, default=30.0, help="optimisation time budget (s)")
    a = ap.parse_args(argv)
    prob = parse(open(a.file).read())
    from . import cubics as K
    if prob.solve == "satisfy":
        rc, st, sols = K.Csp(prob.model).solve(K.CSP_ALL if a.all else K.CSP_FIRST,
                                               a.cap if a.all else 1)
        if rc != 0:
            raise SystemExit(f"search failed: {rc}")
        for s in sols:
            print(format_solution(prob, s))
        print("==========" if st["solutions"] else "=====UNSATISFIABLE=====")
        return
    from . import lns
    res = lns.LNS(prob.model, prob.objective, always_reset=prob.free).run(rounds=10**6,
                                                                          time_budget_s=a.time)
    if res.best is None:
        print("=====UNSATISFIABLE=====")
        return
    print(format_solution(prob, res.solution))
    if res.optimal:
        print("==========")


if __name__ == "__main__":
    main(sys.argv[1:])
