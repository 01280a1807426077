"""GPU: large neighbourhood search rounds against the oracle.

One round's verdicts are exact (each neighbourhood is a plain problem: the oracle decides it),
so the batched launch must give the same SAT/UNSAT status per copy, and every solution must
satisfy the model, the fixings and the bound.  A whole search on small problems must end at
the oracle's optimum with a proof of optimality.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import lns_ref as L
from oracle import oracle as O
from paper_1909_09213_gb300 import cubics as K
from paper_1909_09213_gb300 import instances as I
from paper_1909_09213_gb300 import lns

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("build", ["copies", "shared_encoding"])
@pytest.mark.parametrize("seed", range(3))
def test_round_verdicts_match_the_oracle(seed, build):
    m, obj = I.small_optimisation(seed, n=9, d=9)
    om = O.OracleModel(m)
    r0 = O.solve(om, mode=1, cap=1, variant=1)
    assert r0.status == 1
    inc = r0.sols[0]
    f0 = L.objective(obj, inc)
    base = K.Csp(m)
    for frac in (0.3, 0.6):
        masks = I.relax_masks(m.n, 24, frac, seed, 17)
        if build == "copies":
            batch = K.Batch([lns.neighbourhood(base, inc, mk, obj, f0 - 1) for mk in masks])
        else:
            bounded = base.clone()
            bounded.post_lin(obj[0], obj[1], f0 - 1)
            _, _, lo0 = bounded.layout()
            batch = K.Batch.from_roots(bounded, lns.neighbourhood_roots(bounded.root_domains(), lo0,
                                                                        inc, masks))
        rc, res = batch.solve(K.CSP_FIRST)
        assert rc == 0
        for mk, r in zip(masks, res):
            want = L.verdict(L.neighbourhood_model(m, inc, mk, obj, f0 - 1))
            assert r["status"] == want
            if want == 1:
                s = r["solution"]
                assert O.check_solution(om, s)
                assert L.objective(obj, s) <= f0 - 1
                assert all(s[x] == inc[x] for x in range(m.n) if not mk[x])


@pytest.mark.parametrize("seed", range(4))
def test_search_ends_at_the_oracle_optimum(seed):
    m, obj = I.small_optimisation(seed, n=8, d=8)
    best, _ = L.optimum(m, obj)
    # the rounds stop at the proof; the cap only bounds a long run of small improvements
    res = lns.LNS(m, obj, copies=32, frac=0.25, node_limit=500, seed=seed).run(rounds=400,
                                                                               time_budget_s=60)
    if best is None:
        assert res.best is None
        return
    assert res.optimal and res.best == best
    assert O.check_solution(O.OracleModel(m), res.solution)
    assert L.objective(obj, res.solution) == best
    values = [res.initial] + [r.best for r in res.rounds]
    assert all(b <= a for a, b in zip(values, values[1:]))       # never worse


def test_search_on_a_mixed_instance_improves_and_stays_valid():
    m = I.lin_alldiff(I.seed_for(I.CFG_LINAD, 0))
    obj = I.objective_weights(0, m.n)
    res = lns.LNS(m, obj, copies=64, frac=0.1, node_limit=2000, seed=3).run(rounds=4)
    assert res.initial is not None and res.best <= res.initial
    assert O.check_solution(O.OracleModel(m), res.solution)
    assert L.objective(obj, res.solution) == res.best
