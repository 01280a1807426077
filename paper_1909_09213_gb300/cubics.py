"""Python binding of the CUBICS C ABI (include/cubics.h): argument marshalling only.

Every step of the search runs in libcubics.so's CUDA kernels; this module only converts
Python/numpy arguments, allocates the device workspace as a torch CUDA tensor and passes a
torch stream.  There is no CPU fallback: if the library is missing, importing the names
below raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

CSP_OK, CSP_EINVAL, CSP_ENOMEM, CSP_ETOOBIG, CSP_ECUDA, CSP_ELIMIT, CSP_ETIMEOUT, CSP_ESTATE = (
    0, -1, -2, -3, -4, -5, -6, -7)
CSP_ALL, CSP_FIRST, CSP_PROPAGATE = 0, 1, 2
CSP_BR_FIRST_FAIL, CSP_BR_LEARNED = 0, 1
CSP_F_NO_DONATE = 1

_I32P = C.POINTER(C.c_int32)
_U32P = C.POINTER(C.c_uint32)
_U16P = C.POINTER(C.c_uint16)
_VP = C.c_void_p


class csp_limits(C.Structure):
    _fields_ = [("node_limit", C.c_int64), ("time_limit_ns", C.c_int64),
                ("wait_limit_ns", C.c_int64), ("flags", C.c_int32), ("reserved", C.c_int32)]


class csp_tiling(C.Structure):
    _fields_ = [("blocks", C.c_int32), ("warps_per_block", C.c_int32),
                ("smem_levels", C.c_int32), ("queue_records", C.c_int32),
                ("threads_per_node", C.c_int32), ("split_depth", C.c_int32),
                ("domain_words", C.c_int32)]


class csp_stats_t(C.Structure):
    _fields_ = [("nodes", C.c_uint64), ("fails", C.c_uint64), ("solutions", C.c_uint64),
                ("sol_hash_sum", C.c_uint64), ("sol_hash_xor", C.c_uint64),
                ("prop_evals", C.c_uint64), ("steals", C.c_uint64), ("spills", C.c_uint64),
                ("max_depth", C.c_int32), ("status", C.c_int32), ("ms", C.c_double),
                ("stored", C.c_int64), ("workers", C.c_int32), ("blocks", C.c_int32),
                ("h2d_bytes", C.c_int64), ("d2h_bytes", C.c_int64), ("wait_ns", C.c_uint64),
                ("rounds", C.c_uint64), ("kernel_ms", C.c_double), ("units", C.c_int64)]


class csp_result(C.Structure):
    _fields_ = [("status", C.c_int32), ("n", C.c_int32), ("nodes", C.c_uint64),
                ("fails", C.c_uint64), ("solutions", C.c_uint64), ("sol_offset", C.c_int64),
                ("ms", C.c_double)]


# name -> (restype, argtypes): every entry point of include/cubics.h
SIGNATURES = {
    "csp_create": (C.c_int, [C.POINTER(_VP), C.c_int32, _I32P, _I32P]),
    "csp_remove_value": (C.c_int, [_VP, C.c_int32, C.c_int32]),
    "csp_post_int_ne": (C.c_int, [_VP, C.c_int32, C.c_int32, C.c_int32]),
    "csp_post_int_lin_le": (C.c_int, [_VP, C.c_int32, _I32P, _I32P, C.c_int32]),
    "csp_post_alldiff": (C.c_int, [_VP, C.c_int32, _I32P]),
    "csp_post_alldiff_bc": (C.c_int, [_VP, C.c_int32, _I32P]),
    "csp_post_table": (C.c_int, [_VP, C.c_int32, C.c_int32, _U32P, C.c_int32]),
    "csp_layout": (C.c_int, [_VP, _I32P, _I32P, _I32P]),
    "csp_root_domains": (C.c_int, [_VP, _U32P]),
    "csp_clone": (C.c_int, [_VP, C.POINTER(_VP)]),
    "csp_fix_values": (C.c_int, [_VP, C.c_int32, _I32P, _I32P]),
    "csp_set_tiling": (C.c_int, [_VP, C.POINTER(csp_tiling)]),
    "csp_workspace_bytes": (C.c_int, [_VP, C.c_int32, C.c_int64, C.POINTER(C.c_size_t)]),
    "csp_bind": (C.c_int, [_VP, _VP, C.c_size_t, _VP]),
    "csp_set_brancher": (C.c_int, [_VP, C.c_int32, _U16P]),
    "csp_set_partition": (C.c_int, [_VP, C.c_int32, C.c_int32]),
    "csp_solve": (C.c_int, [_VP, C.c_int32, C.c_int64, _I32P, C.POINTER(csp_limits)]),
    "csp_upload": (C.c_int, [_VP, C.c_int32, C.c_int64]),
    "csp_launch": (C.c_int, [_VP, C.POINTER(csp_limits)]),
    "csp_collect": (C.c_int, [_VP, _I32P]),
    "csp_propagate": (C.c_int, [_VP, C.c_int32, _U32P, _U32P, _I32P]),
    "csp_stats": (C.c_int, [_VP, C.POINTER(csp_stats_t)]),
    "csp_destroy": (None, [_VP]),
    "csp_strerror": (C.c_char_p, [C.c_int]),
    "csp_batch_create": (C.c_int, [C.POINTER(_VP), C.POINTER(_VP), C.c_int32]),
    "csp_batch_create_roots": (C.c_int, [C.POINTER(_VP), _VP, C.c_int32, _U32P]),
    "csp_batch_set_tiling": (C.c_int, [_VP, C.POINTER(csp_tiling)]),
    "csp_batch_workspace_bytes": (C.c_int, [_VP, C.c_int32, C.POINTER(C.c_size_t)]),
    "csp_batch_bind": (C.c_int, [_VP, _VP, C.c_size_t, _VP]),
    "csp_batch_solve": (C.c_int, [_VP, C.c_int32, C.POINTER(csp_limits), C.c_int32,
                                  C.POINTER(csp_result), _I32P]),
    "csp_batch_launch": (C.c_int, [_VP, C.POINTER(csp_limits), C.c_int32]),
    "csp_batch_collect": (C.c_int, [_VP, C.POINTER(csp_result), _I32P]),
    "csp_batch_solution_words": (C.c_int64, [_VP]),
    "csp_batch_set_brancher": (C.c_int, [_VP, C.c_int32, _U16P]),
    "csp_batch_set_log": (C.c_int, [_VP, _VP, _VP, C.c_int64, C.c_uint32]),
    "csp_batch_stats": (C.c_int, [_VP, C.POINTER(csp_stats_t)]),
    "csp_batch_destroy": (None, [_VP]),
    "csp_probe_smem_bandwidth": (C.c_int, [_VP, _VP, C.c_int32, C.POINTER(C.c_double)]),
    "csp_solve_noalloc": (C.c_int, [_VP, C.c_int32, C.c_int64, _I32P, C.POINTER(csp_limits), _VP]),
    "csp_mlp_pack": (C.c_int, [_VP, _VP, _VP]),
    "csp_mlp_forward": (C.c_int, [_VP, _VP, C.c_int32, _VP, _VP]),
    "csp_mlp_grad": (C.c_int, [_VP, _VP, _VP, C.c_int32, _VP, _VP, _VP]),
    "csp_mlp_adam": (C.c_int, [_VP, _VP, _VP, _VP, C.c_int32, C.c_float, _VP, _VP]),
}

_lib = None


def lib_path() -> str:
    return _build.LIB


def lib():
    """Load libcubics.so (building it if stale).  Raises if it cannot be built or loaded."""
    global _lib
    if _lib is None:
        path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is missing; build it with build.py")
        L = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class CspError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {lib().csp_strerror(code).decode()} ({code})")


def _check(code: int, what: str) -> int:
    if code < 0:
        raise CspError(code, what)
    return code


def _i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32).reshape(-1))


def _ptr(a, t):
    return a.ctypes.data_as(t)


def limits(node_limit=0, time_limit_ns=0, wait_limit_ns=0, flags=0) -> csp_limits:
    return csp_limits(node_limit, time_limit_ns, wait_limit_ns, flags, 0)


def tiling(blocks=0, warps_per_block=0, smem_levels=0, queue_records=0,
           threads_per_node=0, split_depth=0, domain_words=0) -> csp_tiling:
    return csp_tiling(blocks, warps_per_block, smem_levels, queue_records, threads_per_node,
                      split_depth, domain_words)


def _stats_dict(s: csp_stats_t) -> dict:
    return {f: getattr(s, f) for f, _ in csp_stats_t._fields_}


def _stream_handle(stream):
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(st.cuda_stream)


def _workspace(nbytes: int):
    import torch
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device="cuda")


# ----------------------------------------------------------------------------- problems

class Csp:
    """One CSP (X, D, C) built through csp_create / csp_post_* from a CspModel."""

    def __init__(self, model):
        L = lib()
        self.model = model
        h = _VP()
        lo, hi = _i32(model.lo), _i32(model.hi)
        _check(L.csp_create(C.byref(h), model.n, _ptr(lo, _I32P), _ptr(hi, _I32P)), "csp_create")
        self.h = h
        self.ws = None
        self.stream = None
        for (v, val) in model.removed:
            _check(L.csp_remove_value(h, v, val), "csp_remove_value")
        for (x, y, c) in model.ne:
            _check(L.csp_post_int_ne(h, x, y, c), "csp_post_int_ne")
        for (coefs, vars_, rhs) in model.lin:
            a, v = _i32(coefs), _i32(vars_)
            _check(L.csp_post_int_lin_le(h, len(a), _ptr(a, _I32P), _ptr(v, _I32P), rhs),
                   "csp_post_int_lin_le")
        for g in model.alldiff:
            v = _i32(g)
            _check(L.csp_post_alldiff(h, len(v), _ptr(v, _I32P)), "csp_post_alldiff")
        for g in getattr(model, "alldiff_bc", []):
            v = _i32(g)
            _check(L.csp_post_alldiff_bc(h, len(v), _ptr(v, _I32P)), "csp_post_alldiff_bc")
        for (x, y, allowed) in model.tables:
            al = np.asarray(allowed, dtype=bool)
            rw = (al.shape[1] + 31) // 32
            bits = np.zeros((al.shape[0], rw * 32), dtype=np.uint64)
            bits[:, :al.shape[1]] = al
            shifts = np.arange(32, dtype=np.uint64)
            words = (bits.reshape(al.shape[0], rw, 32) << shifts).sum(axis=2)
            words = np.ascontiguousarray(words.astype(np.uint32))
            _check(L.csp_post_table(h, x, y, _ptr(words, _U32P), rw), "csp_post_table")

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and _lib is not None:
            _lib.csp_destroy(h)
            self.h = None

    def clone(self) -> "Csp":
        """csp_clone: an unbound copy of this problem (its model object is shared)."""
        h = _VP()
        _check(lib().csp_clone(self.h, C.byref(h)), "csp_clone")
        c = object.__new__(Csp)
        c.model, c.h, c.ws, c.stream = self.model, h, None, None
        return c

    def fix_values(self, vars_, values):
        """csp_fix_values: D(vars_[t]) := D(vars_[t]) & {values[t]}."""
        v, a = _i32(vars_), _i32(values)
        _check(lib().csp_fix_values(self.h, len(v), _ptr(v, _I32P), _ptr(a, _I32P)),
               "csp_fix_values")

    def post_lin(self, coefs, vars_, rhs: int):
        """csp_post_int_lin_le on this handle."""
        a, v = _i32(coefs), _i32(vars_)
        _check(lib().csp_post_int_lin_le(self.h, len(a), _ptr(a, _I32P), _ptr(v, _I32P), int(rhs)),
               "csp_post_int_lin_le")

    def root_domains(self) -> np.ndarray:
        """csp_root_domains: (n, W) uint32 words in the layout of csp_layout."""
        n, W, _ = self.layout()
        out = np.zeros(n * W, dtype=np.uint32)
        _check(lib().csp_root_domains(self.h, _ptr(out, _U32P)), "csp_root_domains")
        return out.reshape(n, W)

    def layout(self):
        n, W, lo0 = C.c_int32(), C.c_int32(), C.c_int32()
        _check(lib().csp_layout(self.h, C.byref(n), C.byref(W), C.byref(lo0)), "csp_layout")
        return n.value, W.value, lo0.value

    def set_tiling(self, t: csp_tiling | None):
        _check(lib().csp_set_tiling(self.h, C.byref(t) if t is not None else None), "csp_set_tiling")

    def set_partition(self, part: int, nparts: int):
        _check(lib().csp_set_partition(self.h, part, nparts), "csp_set_partition")

    def workspace_bytes(self, mode: int, cap: int) -> int:
        b = C.c_size_t()
        _check(lib().csp_workspace_bytes(self.h, mode, cap, C.byref(b)), "csp_workspace_bytes")
        return b.value

    def bind(self, mode: int, cap: int, stream=None):
        need = self.workspace_bytes(mode, cap)
        if self.ws is None or self.ws.numel() < need:
            self.ws = _workspace(need)
        self.stream = stream
        _check(lib().csp_bind(self.h, C.c_void_p(self.ws.data_ptr()), self.ws.numel(),
                              _stream_handle(stream)), "csp_bind")

    def solve(self, mode: int = CSP_ALL, cap: int = 0, lim: csp_limits | None = None,
              raise_on_error: bool = True):
        """csp_solve: returns (status, stats dict, solutions array (stored, n))."""
        self.bind(mode, cap, self.stream)
        n = self.model.n
        sols = np.zeros((max(cap if mode == CSP_ALL else 1, 1), n), dtype=np.int32)
        rc = lib().csp_solve(self.h, mode, cap if mode == CSP_ALL else 1, _ptr(sols, _I32P),
                             C.byref(lim) if lim is not None else None)
        if raise_on_error and rc < 0 and rc not in (CSP_ELIMIT, CSP_ETIMEOUT):
            _check(rc, "csp_solve")
        st = self.stats()
        return rc, st, sols[:st["stored"]].copy()

    def upload(self, mode: int, cap: int):
        _check(lib().csp_upload(self.h, mode, cap), "csp_upload")

    def launch(self, lim: csp_limits | None = None):
        _check(lib().csp_launch(self.h, C.byref(lim) if lim is not None else None), "csp_launch")

    def collect(self, sol_out=None) -> int:
        p = _ptr(sol_out, _I32P) if sol_out is not None else None
        return lib().csp_collect(self.h, p)

    def stats(self) -> dict:
        s = csp_stats_t()
        _check(lib().csp_stats(self.h, C.byref(s)), "csp_stats")
        return _stats_dict(s)

    def set_brancher(self, kind: int, params_bf16=None):
        """csp_set_brancher: first-fail, or learned with bf16 weights (uint16 array)."""
        p = None
        if params_bf16 is not None:
            self._mlp = np.ascontiguousarray(params_bf16, dtype=np.uint16)
            p = self._mlp.ctypes.data_as(_U16P)
        _check(lib().csp_set_brancher(self.h, kind, p), "csp_set_brancher")

    def propagate(self, dom_in: np.ndarray):
        """csp_propagate on `count` states of n*W words: returns (dom_out, failed)."""
        n, W, _ = self.layout()
        d = np.ascontiguousarray(dom_in, dtype=np.uint32).reshape(-1, n * W)
        count = d.shape[0]
        self.bind(CSP_PROPAGATE, count, self.stream)
        out = np.zeros_like(d)
        failed = np.zeros(count, dtype=np.int32)
        _check(lib().csp_propagate(self.h, count, _ptr(d, _U32P), _ptr(out, _U32P),
                                   _ptr(failed, _I32P)), "csp_propagate")
        return out, failed.astype(bool)


# ----------------------------------------------------------------------------- batches

def probe_smem_bandwidth(stream=None, reps: int = 10) -> float:
    """Measured shared-memory read bandwidth of the current device in GB/s."""
    import torch
    out = torch.zeros(16, dtype=torch.uint8, device="cuda")
    g = C.c_double()
    _check(lib().csp_probe_smem_bandwidth(C.c_void_p(out.data_ptr()), _stream_handle(stream),
                                          reps, C.byref(g)), "csp_probe_smem_bandwidth")
    return g.value


MLP_PARAMS, MLP_PACKED_WORDS = 5313, 2948


def _dp(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def mlp_pack(params_bf16, stream=None):
    """csp_mlp_pack: uint16 CUDA tensor of MLP_PARAMS -> int32 tensor of packed words."""
    import torch
    out = torch.empty(MLP_PACKED_WORDS, dtype=torch.int32, device=params_bf16.device)
    _check(lib().csp_mlp_pack(_dp(params_bf16), _dp(out), _stream_handle(stream)), "csp_mlp_pack")
    return out


def mlp_forward(packed, X, stream=None):
    """csp_mlp_forward: scores (float32 CUDA tensor) of the rows of X (rows x 16 float32)."""
    import torch
    rows = X.shape[0]
    out = torch.empty(rows, dtype=torch.float32, device=X.device)
    _check(lib().csp_mlp_forward(_dp(packed), _dp(X), rows, _dp(out), _stream_handle(stream)),
           "csp_mlp_forward")
    return out


def mlp_grad(master, X, y, stream=None):
    """csp_mlp_grad: (gradient tensor, loss tensor) of the mean squared error."""
    import torch
    g = torch.empty(MLP_PARAMS, dtype=torch.float32, device=X.device)
    loss = torch.empty(1, dtype=torch.float32, device=X.device)
    _check(lib().csp_mlp_grad(_dp(master), _dp(X), _dp(y), X.shape[0], _dp(g), _dp(loss),
                              _stream_handle(stream)), "csp_mlp_grad")
    return g, loss


def mlp_adam(master, m, v, grad, step, lr, params_bf16=None, stream=None):
    """csp_mlp_adam: in-place Adam step on master (and m, v); refreshes params_bf16."""
    _check(lib().csp_mlp_adam(_dp(master), _dp(m), _dp(v), _dp(grad), step, lr, _dp(params_bf16),
                              _stream_handle(stream)), "csp_mlp_adam")


class Batch:
    """Many CSPs solved by one persistent launch (csp_batch_*)."""

    def __init__(self, problems):
        L = lib()
        self.problems = list(problems)
        arr = (_VP * len(self.problems))(*[p.h for p in self.problems])
        b = _VP()
        _check(L.csp_batch_create(C.byref(b), arr, len(self.problems)), "csp_batch_create")
        self.b = b
        self.ws = None
        self.stream = None

    @classmethod
    def from_roots(cls, base: "Csp", roots) -> "Batch":
        """csp_batch_create_roots: copies of `base` with root domains roots[i] & base's
        (roots: (count, n, W) uint32)."""
        n, W, _ = base.layout()
        r = np.ascontiguousarray(np.asarray(roots, dtype=np.uint32).reshape(-1, n * W))
        bt = object.__new__(cls)
        bt.problems = [base] * r.shape[0]
        b = _VP()
        _check(lib().csp_batch_create_roots(C.byref(b), base.h, r.shape[0], _ptr(r, _U32P)),
               "csp_batch_create_roots")
        bt.b, bt.ws, bt.stream, bt._roots = b, None, None, r
        return bt

    def __del__(self):
        b = getattr(self, "b", None)
        if b is not None and _lib is not None:
            _lib.csp_batch_destroy(b)
            self.b = None

    def set_tiling(self, t: csp_tiling | None):
        _check(lib().csp_batch_set_tiling(self.b, C.byref(t) if t is not None else None),
               "csp_batch_set_tiling")

    def workspace_bytes(self, mode: int) -> int:
        v = C.c_size_t()
        _check(lib().csp_batch_workspace_bytes(self.b, mode, C.byref(v)), "csp_batch_workspace_bytes")
        return v.value

    def bind(self, mode: int, stream=None):
        need = self.workspace_bytes(mode)
        if self.ws is None or self.ws.numel() < need:
            self.ws = _workspace(need)
        self.stream = stream
        _check(lib().csp_batch_bind(self.b, C.c_void_p(self.ws.data_ptr()), self.ws.numel(),
                                    _stream_handle(stream)), "csp_batch_bind")

    def solve(self, mode: int = CSP_FIRST, lim: csp_limits | None = None, use_graph: bool = False,
              bind: bool = True):
        if use_graph and self.stream is None:
            import torch
            self.stream = torch.cuda.Stream()      # graphs cannot capture the legacy stream
        if bind:
            self.bind(mode, self.stream)
        res = (csp_result * len(self.problems))()
        words = lib().csp_batch_solution_words(self.b)
        sol = np.zeros(max(words, 1), dtype=np.int32)
        rc = lib().csp_batch_solve(self.b, mode, C.byref(lim) if lim is not None else None,
                                   int(use_graph), res, _ptr(sol, _I32P))
        if rc < 0 and rc not in (CSP_ELIMIT, CSP_ETIMEOUT):
            _check(rc, "csp_batch_solve")
        out = [{f: getattr(r, f) for f, _ in csp_result._fields_} for r in res]
        for r in out:
            r["solution"] = sol[r["sol_offset"]:r["sol_offset"] + r["n"]].copy() if r["status"] == 1 else None
        return rc, out

    def stats(self) -> dict:
        s = csp_stats_t()
        _check(lib().csp_batch_stats(self.b, C.byref(s)), "csp_batch_stats")
        return _stats_dict(s)
