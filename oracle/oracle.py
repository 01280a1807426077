"""ctypes wrapper of the C oracle (test infrastructure only).

Converts a ``CspModel`` into the oracle's flat arrays.  Domains cross this boundary as
per-value byte flags: variable i owns flags ``off[i] .. off[i+1]-1`` for values lo_i..hi_i.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import build as _build

_I32P = C.POINTER(C.c_int32)
_I64P = C.POINTER(C.c_int64)
_U8P = C.POINTER(C.c_uint8)


class _Model(C.Structure):
    _fields_ = [("n", C.c_int32), ("lo", _I32P), ("hi", _I32P),
                ("n_ne", C.c_int32), ("ne_x", _I32P), ("ne_y", _I32P), ("ne_c", _I32P),
                ("n_lin", C.c_int32), ("lin_start", _I32P), ("lin_coef", _I32P),
                ("lin_var", _I32P), ("lin_rhs", _I32P),
                ("n_ad", C.c_int32), ("ad_start", _I32P), ("ad_var", _I32P),
                ("n_tab", C.c_int32), ("tab_x", _I32P), ("tab_y", _I32P),
                ("tab_off", _I64P), ("tab_allowed", _U8P),
                ("n_adb", C.c_int32), ("adb_start", _I32P), ("adb_var", _I32P)]


class _Stats(C.Structure):
    _fields_ = [("nodes", C.c_int64), ("fails", C.c_int64), ("solutions", C.c_int64),
                ("stored", C.c_int64), ("hash_sum", C.c_uint64), ("hash_xor", C.c_uint64),
                ("evals", C.c_int64 * 4), ("work_bytes", C.c_double),
                ("status", C.c_int32), ("max_depth", C.c_int32)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(_build.build())
        L.oracle_solve.restype = C.c_int32
        L.oracle_solve.argtypes = [C.POINTER(_Model), _U8P, C.c_int32, C.c_int64, _I32P,
                                   C.c_int32, C.c_int64, C.c_int32, C.c_uint64, C.POINTER(_Stats)]
        L.oracle_propagate.restype = C.c_int32
        L.oracle_propagate.argtypes = [C.POINTER(_Model), _U8P, C.c_int32, C.c_uint64,
                                       C.POINTER(_Stats)]
        L.oracle_check_solution.restype = C.c_int32
        L.oracle_check_solution.argtypes = [C.POINTER(_Model), _U8P, _I32P]
        L.oracle_brute_force.restype = C.c_int64
        L.oracle_brute_force.argtypes = [C.POINTER(_Model), _U8P, C.c_int64, _I32P,
                                         C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]
        L.oracle_splitmix64.restype = C.c_uint64
        L.oracle_splitmix64.argtypes = [C.c_uint64]
        L.oracle_solution_hash.restype = C.c_uint64
        L.oracle_solution_hash.argtypes = [C.c_int32, _I32P]
        _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


class OracleModel:
    """Flat arrays of one CspModel, kept alive for the C calls."""

    def __init__(self, m):
        self.model = m
        i32 = lambda v: np.ascontiguousarray(np.asarray(v, dtype=np.int32).reshape(-1))
        self.n = m.n
        self.lo = i32(m.lo)
        self.hi = i32(m.hi)
        self.size = (self.hi.astype(np.int64) - self.lo + 1)
        self.off = np.concatenate([[0], np.cumsum(self.size)]).astype(np.int64)
        ne = m.ne if m.ne else []
        self.ne_x = i32([c[0] for c in ne])
        self.ne_y = i32([c[1] for c in ne])
        self.ne_c = i32([c[2] for c in ne])
        starts, coefs, vars_, rhs = [0], [], [], []
        for (a, v, b) in m.lin:
            coefs += list(a)
            vars_ += list(v)
            starts.append(len(coefs))
            rhs.append(b)
        self.lin_start, self.lin_coef, self.lin_var, self.lin_rhs = (
            i32(starts), i32(coefs), i32(vars_), i32(rhs))
        ad_start, ad_var = [0], []
        for g in m.alldiff:
            ad_var += list(g)
            ad_start.append(len(ad_var))
        self.ad_start, self.ad_var = i32(ad_start), i32(ad_var)
        offs, mats = [], []
        o = 0
        for (x, y, al) in m.tables:
            al = np.ascontiguousarray(np.asarray(al, dtype=np.uint8))
            assert al.shape == (self.size[x], self.size[y]), "table shape must match the domains"
            offs.append(o)
            mats.append(al.reshape(-1))
            o += al.size
        self.tab_x = i32([t[0] for t in m.tables])
        self.tab_y = i32([t[1] for t in m.tables])
        self.tab_off = np.asarray(offs, dtype=np.int64)
        self.tab_allowed = (np.concatenate(mats) if mats else np.zeros(1, np.uint8)).astype(np.uint8)
        adb = getattr(m, "alldiff_bc", [])
        adb_start, adb_var = [0], []
        for g in adb:
            adb_var += list(g)
            adb_start.append(len(adb_var))
        self.adb_start, self.adb_var = i32(adb_start), i32(adb_var)
        self.c = _Model(self.n, _p(self.lo, _I32P), _p(self.hi, _I32P),
                        len(ne), _p(self.ne_x, _I32P), _p(self.ne_y, _I32P), _p(self.ne_c, _I32P),
                        len(m.lin), _p(self.lin_start, _I32P), _p(self.lin_coef, _I32P),
                        _p(self.lin_var, _I32P), _p(self.lin_rhs, _I32P),
                        len(m.alldiff), _p(self.ad_start, _I32P), _p(self.ad_var, _I32P),
                        len(m.tables), _p(self.tab_x, _I32P), _p(self.tab_y, _I32P),
                        _p(self.tab_off, _I64P), _p(self.tab_allowed, _U8P),
                        len(adb), _p(self.adb_start, _I32P), _p(self.adb_var, _I32P))

    # ---------------------------------------------------------------- domains
    def root_flags(self) -> np.ndarray:
        f = np.ones(int(self.off[-1]), dtype=np.uint8)
        for (i, v) in self.model.removed:
            if self.lo[i] <= v <= self.hi[i]:
                f[self.off[i] + v - self.lo[i]] = 0
        return f

    def flags_to_sets(self, f) -> list:
        return [[int(self.lo[i] + k) for k in range(int(self.size[i])) if f[self.off[i] + k]]
                for i in range(self.n)]


@dataclass
class SolveResult:
    status: int
    nodes: int
    fails: int
    solutions: int
    hash_sum: int
    hash_xor: int
    evals: tuple
    work_bytes: float
    max_depth: int
    sols: np.ndarray


def solve(om: OracleModel, mode: int = 0, cap: int = 0, variant: int = 0, node_limit: int = 0,
          W: int = 0, dom=None, seed: int = 1) -> SolveResult:
    """Search from ``dom`` (default: root domains); mode 0 = all solutions, 1 = first."""
    L = lib()
    d = om.root_flags() if dom is None else np.ascontiguousarray(dom, dtype=np.uint8)
    sols = np.zeros((max(cap, 1), max(om.n, 1)), dtype=np.int32)
    st = _Stats()
    L.oracle_solve(C.byref(om.c), _p(d, _U8P), mode, cap, _p(sols, _I32P), variant, node_limit,
                   W, seed, C.byref(st))
    return SolveResult(st.status, st.nodes, st.fails, st.solutions, st.hash_sum, st.hash_xor,
                       tuple(st.evals), st.work_bytes, st.max_depth, sols[:st.stored, :om.n].copy())


def propagate(om: OracleModel, flags, variant: int = 0, seed: int = 1):
    """One fixpoint from ``flags``; returns (failed, new flags)."""
    d = np.array(flags, dtype=np.uint8, copy=True)
    failed = lib().oracle_propagate(C.byref(om.c), _p(d, _U8P), variant, seed, None)
    return bool(failed), d


def check_solution(om: OracleModel, values, dom=None) -> bool:
    v = np.ascontiguousarray(values, dtype=np.int32)
    d = om.root_flags() if dom is None else np.ascontiguousarray(dom, dtype=np.uint8)
    return bool(lib().oracle_check_solution(C.byref(om.c), _p(d, _U8P), _p(v, _I32P)))


def brute_force(om: OracleModel, cap: int = 1 << 16, dom=None):
    """Every solution by enumeration of prod D_i: (count, hash_sum, hash_xor, solutions)."""
    d = om.root_flags() if dom is None else np.ascontiguousarray(dom, dtype=np.uint8)
    sols = np.zeros((max(cap, 1), max(om.n, 1)), dtype=np.int32)
    hs, hx = C.c_uint64(0), C.c_uint64(0)
    cnt = lib().oracle_brute_force(C.byref(om.c), _p(d, _U8P), cap, _p(sols, _I32P),
                                   C.byref(hs), C.byref(hx))
    return cnt, hs.value, hx.value, sols[:min(cnt, cap), :om.n].copy()


def splitmix64(x: int) -> int:
    return lib().oracle_splitmix64(x)


def solution_hash(values) -> int:
    v = np.ascontiguousarray(values, dtype=np.int32)
    return lib().oracle_solution_hash(len(v), _p(v, _I32P))
