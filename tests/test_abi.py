"""CPU checks of the C ABI: the library loads, exports every declared entry point, and its
host-side validation answers with the documented status codes (no device calls)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1909_09213_gb300 import cubics as K
from paper_1909_09213_gb300 import instances as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for fn in os.listdir(inc):
        if fn.endswith(".h"):
            text = open(os.path.join(inc, fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(csp_\w+)\s*\(", text))
    return names


def test_library_exports_every_declared_symbol():
    L = K.lib()
    names = declared_functions()
    assert len(names) >= 29
    for n in names:
        assert hasattr(L, n), n
    assert names == set(K.SIGNATURES), "binding and header must list the same entry points"


def _create(n, lo, hi):
    h = C.c_void_p()
    lo = np.asarray(lo, np.int32)
    hi = np.asarray(hi, np.int32)
    rc = K.lib().csp_create(C.byref(h), n, lo.ctypes.data_as(K._I32P), hi.ctypes.data_as(K._I32P))
    return rc, h


def test_create_validation():
    assert _create(0, [], [])[0] == K.CSP_EINVAL
    assert _create(1, [3], [2])[0] == K.CSP_EINVAL
    assert _create(1025, [0] * 1025, [1] * 1025)[0] == K.CSP_ETOOBIG
    assert _create(2, [0, 200], [10, 300])[0] == K.CSP_ETOOBIG      # window of 301 values
    rc, h = _create(2, [-5, 0], [5, 250])
    assert rc == K.CSP_OK
    n, W, lo0 = C.c_int32(), C.c_int32(), C.c_int32()
    assert K.lib().csp_layout(h, C.byref(n), C.byref(W), C.byref(lo0)) == 0
    assert (n.value, W.value, lo0.value) == (2, 8, -5)
    K.lib().csp_destroy(h)


def test_post_validation():
    L = K.lib()
    rc, h = _create(3, [0, 0, 0], [9, 9, 9])
    assert rc == 0
    assert L.csp_post_int_ne(h, 0, 3, 1) == K.CSP_EINVAL
    assert L.csp_post_int_ne(h, 0, -1, 4) == K.CSP_OK
    v = np.array([0, 0], np.int32)
    assert L.csp_post_alldiff(h, 2, v.ctypes.data_as(K._I32P)) == K.CSP_EINVAL
    a = np.array([1 << 29, 1 << 29], np.int32)
    v = np.array([0, 1], np.int32)
    assert L.csp_post_int_lin_le(h, 2, a.ctypes.data_as(K._I32P), v.ctypes.data_as(K._I32P), 0) == K.CSP_ETOOBIG
    t = np.ones(10, np.uint32)
    assert L.csp_post_table(h, 1, 1, t.ctypes.data_as(K._U32P), 1) == K.CSP_EINVAL
    assert L.csp_post_table(h, 1, 2, t.ctypes.data_as(K._U32P), 0) == K.CSP_EINVAL
    assert L.csp_post_table(h, 1, 2, t.ctypes.data_as(K._U32P), 1) == K.CSP_OK
    assert L.csp_set_tiling(h, C.byref(K.tiling(queue_records=100))) == K.CSP_EINVAL
    assert L.csp_launch(h, None) == K.CSP_ESTATE          # nothing uploaded
    L.csp_destroy(h)


def test_workspace_size_grows_with_cap():
    p = K.Csp(I.queens(6))
    p.set_tiling(K.tiling(blocks=2, warps_per_block=4))
    b0 = p.workspace_bytes(K.CSP_ALL, 0)
    b1 = p.workspace_bytes(K.CSP_ALL, 1000)
    assert b1 >= b0 + 999 * 6 * 4 - 256
    assert p.workspace_bytes(K.CSP_PROPAGATE, 10) > 0


def test_two_nodes_per_warp_planning():
    """threads_per_node = 16 (two sibling nodes per warp) is planned only for all-solution
    search of one-word int_ne problems of at most 16 variables with the first-fail brancher,
    with a stack of 2n levels instead of n + 1; 0 picks it there, 32 never."""
    R = 20                                       # record words of a 16-variable one-word problem
    p = K.Csp(I.queens(16))
    size = {}
    for tpn in (0, 16, 32):
        p.set_tiling(K.tiling(blocks=2, warps_per_block=4, threads_per_node=tpn, split_depth=-1))
        size[tpn] = p.workspace_bytes(K.CSP_ALL, 0)
    assert size[0] == size[16]
    assert abs(size[16] - size[32] - 2 * 4 * (32 - 17) * R * 4) <= 256
    p.set_tiling(K.tiling(blocks=2, threads_per_node=16))
    p.workspace_bytes(K.CSP_ALL, 0)              # split plan too
    with pytest.raises(K.CspError) as e:
        p.workspace_bytes(K.CSP_FIRST, 1)
    assert e.value.code == K.CSP_EINVAL
    L = K.lib()
    one = np.zeros(16, np.uint32)
    failed = np.zeros(1, np.int32)
    assert L.csp_propagate(p.h, 1, one.ctypes.data_as(K._U32P), one.ctypes.data_as(K._U32P),
                           failed.ctypes.data_as(K._I32P)) == K.CSP_EINVAL
    q = K.Csp(I.queens(17))
    q.set_tiling(K.tiling(blocks=2, threads_per_node=16))
    with pytest.raises(K.CspError) as e:
        q.workspace_bytes(K.CSP_ALL, 0)
    assert e.value.code == K.CSP_EINVAL
    q.set_tiling(K.tiling(blocks=2, threads_per_node=0))    # the library's choice: a warp
    q.workspace_bytes(K.CSP_ALL, 0)
    p.set_brancher(K.CSP_BR_LEARNED, np.zeros(K.MLP_PARAMS, np.uint16))
    with pytest.raises(K.CspError) as e:
        p.workspace_bytes(K.CSP_ALL, 0)
    assert e.value.code == K.CSP_EINVAL
    with pytest.raises(K.CspError):
        p.set_tiling(K.tiling(threads_per_node=8))


def test_wider_domain_words_planning():
    """csp_tiling.domain_words: a search planned at a wider bitset has wider records (a larger
    workspace); widths that are not 1, 2, 4 or 8 are refused; two nodes per warp need one-word
    domains; a batch takes only its own width."""
    p = K.Csp(I.queens(8))
    base = None
    for dw in (0, 1, 2, 4, 8):
        p.set_tiling(K.tiling(blocks=2, warps_per_block=4, split_depth=-1, domain_words=dw))
        b = p.workspace_bytes(K.CSP_ALL, 0)
        if dw in (0, 1):
            base = b if base is None else base
            assert b == base
        else:
            assert b > base
    assert p.layout()[1] == 1                    # the problem's own layout is unchanged
    p.set_tiling(K.tiling(blocks=2, threads_per_node=16, domain_words=2))
    with pytest.raises(K.CspError) as e:
        p.workspace_bytes(K.CSP_ALL, 0)
    assert e.value.code == K.CSP_EINVAL
    L = K.lib()
    for bad in (3, 5, 16, -1):
        assert L.csp_set_tiling(p.h, C.byref(K.tiling(domain_words=bad))) == K.CSP_EINVAL
    bt = K.Batch([K.Csp(I.queens(6)), K.Csp(I.queens(7))])
    assert L.csp_batch_set_tiling(bt.b, C.byref(K.tiling(domain_words=2))) == K.CSP_EINVAL
    assert L.csp_batch_set_tiling(bt.b, C.byref(K.tiling(domain_words=1))) == 0


def test_models_build_through_the_abi():
    for m in [I.queens(8), I.worked_example("lin", "table"), I.model_rb(1, 20, 8),
              I.lin_alldiff(3), I.random_tiny(5)]:
        p = K.Csp(m)
        n, W, lo0 = p.layout()
        assert n == m.n and W in (1, 2, 4, 8) and lo0 == min(m.lo)


def test_encoded_root_domains_equal_the_oracle_domains():
    # host-only: the encoder's root bitsets against the oracle's byte flags
    from oracle import oracle as O
    from _util import flags_to_bits
    models = [I.queens(8), I.worked_example("domain", "table"), I.model_rb(3, 25, 20),
              I.lin_alldiff(5, n=30, rows=6, groups=3)]
    models += [I.random_tiny(I.seed_for(I.CFG_TINY, 95000 + k)) for k in range(60)]
    for m in models:
        p = K.Csp(m)
        n, W, lo0 = p.layout()
        om = O.OracleModel(m)
        want = flags_to_bits(om, om.root_flags(), n, W, lo0).reshape(n, W)
        assert np.array_equal(p.root_domains(), want), m.name


def test_tuner_candidates_for_one_problem():
    """The autotuner's search shapes (host side, no device): warps per block x two nodes or
    one per warp x the problem's own bitset width or twice it, the wider width only while it
    is at most 8 words."""
    from paper_1909_09213_gb300 import tune
    one = tune.single_candidates(I.queens(8))                   # one word per domain
    assert len(one) == 3 * 2 * 2
    assert {c["domain_words"] for c in one} == {0, 2}
    assert {c["threads_per_node"] for c in one} == {16, 32}
    assert {c["warps_per_block"] for c in one} == {4, 8, 16}
    m = I.CspModel(n=3, lo=[0, 0, 0], hi=[200, 200, 200], name="wide")   # 201 values: 8 words
    m.ne.append((0, 1, 0))
    assert K.Csp(m).layout()[1] == 8
    wide = tune.single_candidates(m)
    assert {c["domain_words"] for c in wide} == {0} and len(wide) == 6
    for c in one + wide:                                     # every candidate is a valid tiling
        p = K.Csp(I.queens(8))
        p.set_tiling(K.tiling(**c))
