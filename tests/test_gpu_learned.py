"""The learned brancher inside the search: it may change the order of exploration, never the
results.  First-fail is its fallback; its features are node-local, so the learned tree does
not depend on how the workers share it.  Subtree logging yields well-formed training data,
and a short training run lowers the loss on it.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mlp_ref as M
from oracle import oracle as O
from paper_1909_09213_gb300 import cubics as K
from paper_1909_09213_gb300 import instances as I
from paper_1909_09213_gb300 import learn

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _weights(seed):
    return M.to_bf16_bits(M.init_params(seed))


def _solve(m, kind, w=None, tiling=None, mode=K.CSP_ALL, cap=100000):
    p = K.Csp(m)
    if tiling is not None:
        p.set_tiling(tiling)
    if kind == K.CSP_BR_LEARNED:
        p.set_brancher(kind, w)
    rc, st, sols = p.solve(mode, cap)
    assert rc == 0
    return st, sols


def _models():
    # all-solution searches of a few thousand to a hundred thousand nodes (oracle-sized)
    return [I.queens(9), I.model_rb(I.seed_for(I.CFG_RB, 716), 12, 8),
            I.lin_alldiff(31, n=8, dmax=5, rows=3, kmin=2, kmax=4, groups=1, gsize=4, theta=0.5)]


@pytest.mark.parametrize("seed", [0, 1])
def test_learned_order_never_changes_the_solution_set(seed):
    w = _weights(seed)
    for m in _models():
        ff, ff_sols = _solve(m, K.CSP_BR_FIRST_FAIL)
        le, le_sols = _solve(m, K.CSP_BR_LEARNED, w)
        for k in ("solutions", "sol_hash_sum", "sol_hash_xor"):
            assert le[k] == ff[k], (m.name, k)
        assert sorted(map(tuple, le_sols.tolist())) == sorted(map(tuple, ff_sols.tolist()))


def test_learned_tree_does_not_depend_on_work_sharing():
    w = _weights(3)
    m = I.queens(11)
    one, _ = _solve(m, K.CSP_BR_LEARNED, w, K.tiling(blocks=1, warps_per_block=1))
    many, _ = _solve(m, K.CSP_BR_LEARNED, w)
    assert (one["nodes"], one["fails"], one["solutions"]) == (many["nodes"], many["fails"], many["solutions"])
    ff, _ = _solve(m, K.CSP_BR_FIRST_FAIL)
    assert one["solutions"] == ff["solutions"] == 2680


@pytest.mark.parametrize("split", [-1, 3, 8])
def test_learned_order_ignores_the_split_depth(split):
    # the device expansion of a split branches first-fail, so the learned brancher always
    # searches the whole tree through one queue: the tree is the same at every split depth
    w = _weights(6)
    for m in _models():
        ref, ref_sols = _solve(m, K.CSP_BR_LEARNED, w, K.tiling(split_depth=-1))
        st, sols = _solve(m, K.CSP_BR_LEARNED, w, K.tiling(split_depth=split))
        for k in ("nodes", "fails", "solutions", "sol_hash_sum", "sol_hash_xor"):
            assert st[k] == ref[k], (m.name, split, k)
        assert sorted(map(tuple, sols.tolist())) == sorted(map(tuple, ref_sols.tolist()))


def test_nan_network_falls_back_to_first_fail():
    w = _weights(4)
    w[M.N_PARAMS - 1] = 0x7FC0                      # b3 = NaN: every score is NaN
    for m in _models():
        ff, _ = _solve(m, K.CSP_BR_FIRST_FAIL)
        le, _ = _solve(m, K.CSP_BR_LEARNED, w)
        assert (le["nodes"], le["fails"], le["solutions"]) == (ff["nodes"], ff["fails"], ff["solutions"])


def test_learned_first_mode_is_valid():
    w = _weights(5)
    for k in range(20):
        m = I.model_rb(I.seed_for(I.CFG_RB, 300 + k), 18, 8)
        om = O.OracleModel(m)
        r = O.solve(om, mode=1, cap=1)
        st, sols = _solve(m, K.CSP_BR_LEARNED, w, mode=K.CSP_FIRST, cap=1)
        assert st["solutions"] == (1 if r.status == 1 else 0)
        if r.status == 1:
            assert O.check_solution(om, sols[0])


def test_trained_network_gain_over_first_fail():
    """The learning configuration at reduced size (2000 training instances n = 30, d = 16;
    128 held-out instances n = 80, d = 20, first solution): the network trained on the
    solver's own subtree logs must give the same verdict on every instance and explore fewer
    nodes than first-fail.  The gain is an empirical measurement, not a pinned value."""
    r = learn.learning_config(2000, 128, epochs=6)
    assert r["same_status"]
    ff, le = r["first_fail_nodes"], r["learned_nodes"]
    print(f"\nlearned vs first-fail: nodes {le} vs {ff} ({ff / max(le, 1):.1f}x fewer), "
          f"time {r['learned_ms']:.1f} ms vs {r['first_fail_ms']:.1f} ms")
    assert le < ff
    for m, res in zip(r["eval_models"], r["eval"]["learned"]["results"]):
        if res["status"] == 1:
            om = O.OracleModel(m)
            assert O.check_solution(om, res["solution"])


def test_subtree_logging_and_training():
    # the learning configuration's training instances (n = 30, d = 16): UNSAT proofs of
    # tens to hundreds of nodes each
    models = I.rb_batch(64, n_range=(30, 30), d_range=(16, 16), config_id=I.CFG_RB_TRAIN)
    data, info = learn.collect(models, cap=200000, sample=1)
    assert info["entries"] > 1000
    d = data.cpu().numpy()
    assert np.isfinite(d).all()
    assert (d[:, 16] >= 0).all()                     # log2 of at least one node
    assert np.allclose(d[:, 15], 1.0)                # the bias feature
    assert ((d[:, 0] > 0) & (d[:, 0] <= 1)).all()    # relative domain size of an unfixed var
    # the exhaustive searches are unchanged by logging: counts equal plain batches
    b = K.Batch([K.Csp(m) for m in models])
    rc, res = b.solve(K.CSP_ALL)
    assert info["nodes"] == sum(r["nodes"] for r in res)
    params, tinfo = learn.train(data, epochs=10, batch=256, lr=2e-3)
    # better than the constant predictor (the target variance)
    assert tinfo["mse_per_epoch"][-1] < 0.9 * tinfo["target_variance"]
    assert len(params) == K.MLP_PARAMS


@pytest.mark.parametrize("W", [2, 4, 8])
def test_learned_order_at_wider_domains(W):
    """The learned kernels for 2-, 4- and 8-word domains: the solution set, count and hash
    equal first-fail's and the oracle's; only the tree may differ."""
    from test_gpu_parity import mixed_model, pooled_wide_model, strided_queens
    if W == 2:
        models = [mixed_model(100 + k, 40, 5) for k in range(2)]
    else:
        stride, span = (13, 100) if W == 4 else (31, 250)
        models = [strided_queens(9, stride), strided_queens(8, stride, alldiff=True, rows=True),
                  pooled_wide_model(1002, span)]
    w = _weights(11)
    for m in models:
        assert K.Csp(m).layout()[1] == W, m.name
        r = O.solve(O.OracleModel(m), cap=100000, variant=1)
        ff, ff_sols = _solve(m, K.CSP_BR_FIRST_FAIL)
        le, le_sols = _solve(m, K.CSP_BR_LEARNED, w)
        for k in ("solutions", "sol_hash_sum", "sol_hash_xor"):
            assert le[k] == ff[k], (m.name, k)
        assert (le["solutions"], le["sol_hash_sum"], le["sol_hash_xor"]) == (
            r.solutions, r.hash_sum, r.hash_xor), m.name
        if r.solutions <= 100000:              # otherwise each stores an arbitrary 100000
            assert sorted(map(tuple, le_sols.tolist())) == sorted(map(tuple, ff_sols.tolist()))
            assert sorted(map(tuple, le_sols.tolist())) == sorted(map(tuple, r.sols.tolist()))


def test_learned_first_solution_on_mixed_wide_instances():
    """First-solution batches of small mixed linear/alldifferent instances over 0..255 (W = 8)
    with the learned brancher: where both orderings decide an instance they agree on SAT /
    UNSAT, every solution satisfies the model, and the oracle's verdict is met."""
    models = [I.lin_alldiff(I.seed_for(I.CFG_LINAD_TRAIN, 900 + k), n=16, dmax=255, rows=8,
                            kmin=3, kmax=6, groups=2, gsize=8, theta=0.3) for k in range(24)]
    lim = K.limits(node_limit=100_000)
    out = {}
    for kind in (K.CSP_BR_FIRST_FAIL, K.CSP_BR_LEARNED):
        b = K.Batch([K.Csp(m) for m in models])
        if kind == K.CSP_BR_LEARNED:
            w = np.ascontiguousarray(_weights(4), dtype=np.uint16)
            K._check(K.lib().csp_batch_set_brancher(b.b, kind, w.ctypes.data_as(K._U16P)), "brancher")
        rc, out[kind] = b.solve(K.CSP_FIRST, lim=lim)
        assert rc == 0
    decided = 0
    for m, f, l in zip(models, out[K.CSP_BR_FIRST_FAIL], out[K.CSP_BR_LEARNED]):
        assert K.Csp(m).layout()[1] == 8
        om = O.OracleModel(m)
        r = O.solve(om, mode=1, cap=1, node_limit=100_000)
        for res in (f, l):
            if res["status"] == 1:
                assert O.check_solution(om, res["solution"]), m.name
            if res["status"] >= 0 and r.status >= 0:
                assert res["status"] == r.status, m.name
        if f["status"] >= 0 and l["status"] >= 0:
            decided += 1
            assert f["status"] == l["status"], m.name
    assert decided >= 12
