"""csp_solve_noalloc: the search without any device allocation by the caller or the library.

Some callers cannot call cudaMalloc (code inside a stream capture that must not allocate, a
plug-in whose host owns every allocation, a real-time loop).  For them the library solves
out of a scratch array that is part of its own device image.  These tests call that entry
point through the C ABI and check it against csp_solve, the entry point that uses a
caller-bound workspace, on two calls in a row.  The file sorts last so that a run stopping at
the first failure has run every other test first.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1909_09213_gb300 import cubics as K
from paper_1909_09213_gb300 import instances as I

pytestmark = pytest.mark.gpu

SCRATCH_BYTES = 16 << 20          # CSP_NOALLOC_SCRATCH_BYTES in include/cubics.h


@pytest.fixture(autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _noalloc(p, mode, cap):
    n = p.model.n
    sols = np.zeros((max(cap, 1), n), dtype=np.int32)
    rc = K.lib().csp_solve_noalloc(p.h, mode, cap, sols.ctypes.data_as(K._I32P), None, None)
    st = p.stats()
    return rc, st, sols[:st["stored"]]


def _rows(a):
    return sorted(map(tuple, np.asarray(a).tolist()))


@pytest.mark.parametrize("N,cap", [(10, 1000), (12, 20000)])
def test_noalloc_matches_bound_workspace_twice(N, cap):
    ref = K.Csp(I.queens(N))
    rc, st_ref, sols_ref = ref.solve(K.CSP_ALL, cap)
    assert rc == 0
    p = K.Csp(I.queens(N))
    for call in range(2):               # the array keeps the previous call's contents
        rc, st, sols = _noalloc(p, K.CSP_ALL, cap)
        assert rc == 0, call
        for k in ("solutions", "sol_hash_sum", "sol_hash_xor", "nodes", "fails", "stored"):
            assert st[k] == st_ref[k], (call, k)
        assert _rows(sols) == _rows(sols_ref)


def test_noalloc_first_mode_and_other_problem_between():
    m = I.model_rb(I.seed_for(I.CFG_RB, 3), 25, 10)
    ref = K.Csp(m)
    rc, st_ref, _ = ref.solve(K.CSP_FIRST)
    assert rc == 0
    p = K.Csp(m)
    q = K.Csp(I.queens(9))
    for call in range(2):
        rc, st, sols = _noalloc(p, K.CSP_FIRST, 1)
        assert rc == 0 and st["solutions"] == st_ref["solutions"]
        if st["solutions"]:
            from oracle import oracle as O
            assert O.check_solution(O.OracleModel(m), sols[0])
        rc, st_q, _ = _noalloc(q, K.CSP_ALL, 0)       # a different problem in between
        assert rc == 0 and st_q["solutions"] == 352


def test_noalloc_rejects_what_does_not_fit():
    p = K.Csp(I.queens(16))
    cap = SCRATCH_BYTES // (16 * 4) + 1                  # the solution buffer alone overflows
    sols = np.zeros((1, 16), dtype=np.int32)
    rc = K.lib().csp_solve_noalloc(p.h, K.CSP_ALL, cap, sols.ctypes.data_as(K._I32P), None, None)
    assert rc == K.CSP_ENOMEM
