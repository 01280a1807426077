"""Large neighbourhood search, host side (no GPU): the oracle's optimum against closed forms
and enumeration, the neighbourhood construction of the C ABI (csp_clone, csp_fix_values,
csp_root_domains are host-only calls) against the oracle's neighbourhood model, the seeded
reset sets, and the sharing of the incumbent between ranks (gloo, world size 2)."""
import datetime
import json
import os
import socket
import tempfile

import numpy as np
import pytest

from oracle import lns_ref as L
from oracle import oracle as O
from paper_1909_09213_gb300 import instances as I

from _util import flags_to_bits

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _permutation_model(w):
    n = len(w)
    m = I.CspModel(n=n, lo=[0] * n, hi=[n - 1] * n, name=f"perm{n}")
    m.alldiff.append(list(range(n)))
    return m, (list(w), list(range(n)))


@pytest.mark.parametrize("w", [[3, 1, 2], [5, 9, 1, 4], [2, 7, 1, 8, 2, 8], [1, 1, 1, 1, 1]])
def test_optimum_of_a_permutation_is_the_rearrangement_bound(w):
    # min sum w_i x_i over permutations x of 0..n-1: the largest weight takes 0, the next 1, ...
    m, obj = _permutation_model(w)
    closed = sum(k * wk for k, wk in enumerate(sorted(w, reverse=True)))
    best, sol = L.optimum(m, obj)
    assert best == closed
    assert sorted(sol.tolist()) == list(range(len(w))) and L.objective(obj, sol) == closed


@pytest.mark.parametrize("seed", range(4))
def test_optimum_equals_enumeration(seed):
    m, obj = I.small_optimisation(seed, n=6, d=6)
    best, sol = L.optimum(m, obj)
    assert best == L.brute_force_optimum(m, obj)
    if best is not None:
        assert O.check_solution(O.OracleModel(m), sol)


def test_neighbourhood_bound_separates_the_optimum():
    m, obj = I.small_optimisation(1, n=7, d=7)
    best, sol = L.optimum(m, obj)
    assert best is not None
    everything = np.ones(m.n, dtype=bool)
    assert L.verdict(L.neighbourhood_model(m, sol, everything, obj, best)) == 1
    assert L.verdict(L.neighbourhood_model(m, sol, everything, obj, best - 1)) == 0
    # nothing reset: the incumbent itself is the only candidate
    nothing = np.zeros(m.n, dtype=bool)
    assert L.verdict(L.neighbourhood_model(m, sol, nothing, obj, best)) == 1
    assert L.verdict(L.neighbourhood_model(m, sol, nothing, obj, best - 1)) == 0


def test_relax_masks_are_seeded_and_never_empty():
    a = I.relax_masks(30, 64, 0.1, 3, 11)
    b = I.relax_masks(30, 64, 0.1, 3, 11)
    c = I.relax_masks(30, 64, 0.1, 4, 11)
    assert a.shape == (64, 30) and a.dtype == bool
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert a.any(axis=1).all()
    big = I.relax_masks(40, 4000, 0.25, 0, 5)
    assert abs(big.mean() - 0.25) < 0.01
    assert I.relax_masks(10, 3, 1.0, 0, 1).all()


def _lib_available():
    try:
        from paper_1909_09213_gb300 import cubics as K
        K.lib()
        return True
    except Exception:                                            # noqa: BLE001
        return False


@pytest.mark.skipif(not _lib_available(), reason="library not built")
@pytest.mark.parametrize("seed", range(3))
def test_clone_and_fix_match_the_oracle_neighbourhood(seed):
    from paper_1909_09213_gb300 import cubics as K
    m, obj = I.small_optimisation(seed, n=9, d=9)
    m.removed += [(2, 4), (5, 0)]
    best, sol = L.optimum(m, obj)
    base = K.Csp(m)
    n, W, lo0 = base.layout()
    before = base.root_domains().copy()
    for mask in I.relax_masks(m.n, 8, 0.4, seed, 3):
        c = base.clone()
        fixed = np.nonzero(~mask)[0]
        c.fix_values(fixed, sol[fixed])
        om = O.OracleModel(L.neighbourhood_model(m, sol, mask, obj, best))
        want = flags_to_bits(om, om.root_flags(), n, W, lo0).reshape(n, W)
        assert np.array_equal(c.root_domains(), want)
    assert np.array_equal(base.root_domains(), before)          # the source is untouched


@pytest.mark.skipif(not _lib_available(), reason="library not built")
@pytest.mark.parametrize("d", [9, 40, 100])          # one, two and four words per domain
def test_shared_encoding_roots_equal_the_copies(d):
    from paper_1909_09213_gb300 import cubics as K
    from paper_1909_09213_gb300 import lns
    m, obj = I.small_optimisation(4, n=9, d=d)
    m.removed += [(0, 3), (8, 8)]
    sol = np.asarray(O.solve(O.OracleModel(m), mode=1, cap=1, variant=1).sols[0])
    best = L.objective(obj, sol)
    base = K.Csp(m)
    _, _, lo0 = base.layout()
    masks = I.relax_masks(m.n, 16, 0.35, 2, 9)
    roots = lns.neighbourhood_roots(base.root_domains(), lo0, sol, masks)
    for mk, rt in zip(masks, roots):
        assert np.array_equal(lns.neighbourhood(base, sol, mk, obj, best).root_domains(), rt)
    b = K.Batch.from_roots(base, roots)                         # host only: encodes once
    assert len(b.problems) == 16
    with pytest.raises(K.CspError) as e:
        K.Batch.from_roots(base, roots[:0])
    assert e.value.code == K.CSP_EINVAL


@pytest.mark.skipif(not _lib_available(), reason="library not built")
def test_fix_values_validation_and_empty_domain():
    from paper_1909_09213_gb300 import cubics as K
    m = I.CspModel(n=3, lo=[0, 0, 0], hi=[3, 3, 3])
    p = K.Csp(m)
    before = p.root_domains().copy()
    with pytest.raises(K.CspError) as e:
        p.fix_values([0, 7], [1, 1])
    assert e.value.code == K.CSP_EINVAL
    assert np.array_equal(p.root_domains(), before)              # nothing changed
    p.fix_values([1, 2], [2, 9])                                 # 9 is not in D(x2)
    d = p.root_domains()[:, 0]
    assert d[0] == 0b1111 and d[1] == 0b0100 and d[2] == 0


# ---------------------------------------------------------------------------- two ranks

def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _share_worker(rank, world, port, outdir, offers):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=20))
    from paper_1909_09213_gb300 import lns
    v, s = offers[rank]
    bv, bs = lns.share_best(v, None if s is None else np.asarray(s, dtype=np.int32))
    proof = lns._all_ranks(rank == world - 1)
    with open(os.path.join(outdir, f"rank{rank}.json"), "w") as f:
        json.dump({"value": bv, "sol": None if bs is None else bs.tolist(), "proof": proof}, f)
    dist.destroy_process_group()


@pytest.mark.parametrize("offers", [
    [(40, [1, 2, 3]), (35, [3, 2, 1])],
    [(None, None), (12, [0, 0, 1])],
    [(7, [9, 9, 9]), (7, [1, 1, 1])],          # tie: the lower rank's solution
])
def test_two_ranks_agree_on_the_best_incumbent(offers):
    import torch.multiprocessing as mp
    port = _free_port()
    with tempfile.TemporaryDirectory() as d:
        ctx = mp.get_context("spawn")
        procs = [ctx.Process(target=_share_worker, args=(r, 2, port, d, offers)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            if p.is_alive():
                p.kill()
                raise AssertionError("a rank did not finish")
        out = [json.load(open(os.path.join(d, f"rank{r}.json"))) for r in range(2)]
    vals = [v for v, _ in offers if v is not None]
    want_v = min(vals)
    want_s = next(s for v, s in offers if v == want_v)
    for o in out:
        assert o["value"] == want_v and o["sol"] == want_s and o["proof"] is True
