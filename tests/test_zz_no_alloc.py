"""csp_solve_noalloc: the search without any device allocation by the caller or the library.

Some callers may not call cudaMalloc: a plug-in whose host application owns every device
allocation, or a latency-bound loop in which an allocation may block.  For them the library
solves out of a scratch array that is part of its own device image.  These tests call that
entry point through the C ABI and check it against csp_solve (the entry point that uses a
caller-bound workspace) and against the oracle's or the published counts, on two calls in a
row; they also check that a failed call leaves a handle's own upload usable.  The file sorts
last so that a run stopping at the first failure has run every other test first.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mlp_ref as M
from oracle import oracle as O
from paper_1909_09213_gb300 import cubics as K
from paper_1909_09213_gb300 import instances as I

pytestmark = pytest.mark.gpu

SCRATCH_BYTES = 16 << 20          # CSP_NOALLOC_SCRATCH_BYTES in include/cubics.h
QUEENS = {9: 352, 10: 724, 12: 14200}   # published N-queens counts (tests/golden/queens_counts.txt)


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
def test_noalloc_matches_bound_workspace_and_oracle_twice(N, cap):
    ref = K.Csp(I.queens(N))
    rc, st_ref, sols_ref = ref.solve(K.CSP_ALL, cap)
    assert rc == 0
    orc = O.solve(O.OracleModel(I.queens(N)), cap=0, variant=1) if N <= 10 else None
    p = K.Csp(I.queens(N))
    for call in range(2):               # the array keeps the previous call's contents
        rc, st, sols = _noalloc(p, K.CSP_ALL, cap)
        assert rc == 0, call
        assert st["solutions"] == QUEENS[N]
        for k in ("solutions", "sol_hash_sum", "sol_hash_xor", "nodes", "fails", "stored"):
            assert st[k] == st_ref[k], (call, k)
        if orc is not None:
            assert (st["nodes"], st["fails"], st["sol_hash_sum"], st["sol_hash_xor"]) == (
                orc.nodes, orc.fails, orc.hash_sum, orc.hash_xor)
        assert _rows(sols) == _rows(sols_ref)
        assert all(O.check_solution(O.OracleModel(p.model), s) for s in sols[:50])


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
            assert O.check_solution(O.OracleModel(m), sols[0])
        rc, st_q, _ = _noalloc(q, K.CSP_ALL, 0)       # a different problem in between
        assert rc == 0 and st_q["solutions"] == QUEENS[9]


def test_noalloc_learned_brancher_twice():
    m = I.queens(9)
    w = M.to_bf16_bits(M.init_params(5))
    ref = K.Csp(m)
    ref.set_brancher(K.CSP_BR_LEARNED, w)
    rc, st_ref, sols_ref = ref.solve(K.CSP_ALL, 400)
    assert rc == 0
    p = K.Csp(m)
    p.set_brancher(K.CSP_BR_LEARNED, w)
    for call in range(2):
        rc, st, sols = _noalloc(p, K.CSP_ALL, 400)
        assert rc == 0, call
        for k in ("solutions", "sol_hash_sum", "sol_hash_xor"):
            assert st[k] == st_ref[k], (call, k)
        assert st["solutions"] == QUEENS[9]
        assert _rows(sols) == _rows(sols_ref)
        # the brancher's bf16 parameters are part of what the call uploads
        assert st["h2d_bytes"] == st_ref["h2d_bytes"]


def test_noalloc_rejects_what_does_not_fit():
    p = K.Csp(I.queens(16))
    cap = SCRATCH_BYTES // (16 * 4) + 1                  # the solution buffer alone overflows
    sols = np.zeros((1, 16), dtype=np.int32)
    rc = K.lib().csp_solve_noalloc(p.h, K.CSP_ALL, cap, sols.ctypes.data_as(K._I32P), None, None)
    assert rc == K.CSP_ENOMEM


def test_failed_noalloc_call_leaves_the_bound_upload_usable():
    """A handle bound and uploaded for csp_launch, then a no-alloc call that fails for want
    of space: the upload still launches and gives the oracle's results."""
    m = I.queens(10)
    orc = O.solve(O.OracleModel(m), cap=0, variant=1)
    p = K.Csp(m)
    p.bind(K.CSP_ALL, 0)
    p.upload(K.CSP_ALL, 0)
    cap = SCRATCH_BYTES // (10 * 4) + 1
    sols = np.zeros((1, 10), dtype=np.int32)
    rc = K.lib().csp_solve_noalloc(p.h, K.CSP_ALL, cap, sols.ctypes.data_as(K._I32P), None, None)
    assert rc == K.CSP_ENOMEM
    p.launch()
    assert p.collect() == 0
    st = p.stats()
    assert (st["solutions"], st["nodes"], st["fails"], st["sol_hash_sum"], st["sol_hash_xor"]) == (
        orc.solutions, orc.nodes, orc.fails, orc.hash_sum, orc.hash_xor)
    # and a successful no-alloc call in between changes nothing of the upload either
    rc, st2, _ = _noalloc(K.Csp(I.queens(9)), K.CSP_ALL, 0)
    assert rc == 0 and st2["solutions"] == QUEENS[9]
    rc, st3, _ = _noalloc(p, K.CSP_FIRST, 1)
    assert rc == 0 and st3["solutions"] == 1
    p.launch()
    assert p.collect() == 0
    assert p.stats()["nodes"] == orc.nodes


def test_noalloc_refuses_a_capturing_stream():
    """On a stream being captured the call returns CSP_ESTATE at once and does nothing: the
    capture stays valid (the graph replays what else was captured), and the next call outside
    the capture searches as usual."""
    p = K.Csp(I.queens(8))
    s = torch.cuda.Stream()
    x = torch.zeros(1, device="cuda")
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        rc = K.lib().csp_solve_noalloc(p.h, K.CSP_ALL, 0, None, None, C.c_void_p(s.cuda_stream))
        x += 1
    assert rc == K.CSP_ESTATE
    g.replay()
    torch.cuda.synchronize()
    assert x.item() == 1.0
    rc, st, _ = _noalloc(p, K.CSP_ALL, 0)
    assert rc == 0 and st["solutions"] == 92
