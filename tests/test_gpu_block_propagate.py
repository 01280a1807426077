"""Constraint-parallel propagation of one node by a whole block (csp_tiling.threads_per_node
= 64..1024): every warp of the block takes its share of each round's constraints.  The
fixpoints must equal the oracle's bit for bit, as those of the warp-per-node kernel do, for
every constraint kind and domain width, and for a node too large for the shared memory of
eight warps."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_1909_09213_gb300 import cubics as K
from paper_1909_09213_gb300 import instances as I

from _util import bits_to_flags, flags_to_bits, random_subdomains

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _parity(m, tpn, rng, count, check=None):
    om = O.OracleModel(m)
    p = K.Csp(m)
    p.set_tiling(K.tiling(threads_per_node=tpn))
    n, W, lo0 = p.layout()
    subs = [om.root_flags()] + random_subdomains(om, rng, count)
    din = np.stack([flags_to_bits(om, f, n, W, lo0) for f in subs])
    dout, failed = p.propagate(din)
    fails = 0
    for k, f in enumerate(subs if check is None else subs[:check]):
        of, od = O.propagate(om, f, variant=1)
        assert bool(failed[k]) == of, (m.name, tpn, k)
        if of:
            fails += 1
            continue
        got = bits_to_flags(om, dout[k], n, W, lo0)
        assert np.array_equal(got, od), (m.name, tpn, k)
    # the warp-per-node kernel agrees on every state, checked or not
    q = K.Csp(m)
    d2, f2 = q.propagate(din)
    assert np.array_equal(f2, failed)
    assert np.array_equal(d2[~failed], dout[~failed])
    return fails


@pytest.mark.parametrize("tpn", [64, 128, 256, 1024])
def test_block_fixpoints_every_kind(tpn):
    import sys, os
    sys.path.insert(0, os.path.dirname(__file__))
    from test_gpu_parity import mixed_model, pooled_wide_model
    from test_gpu_alldiff_bc import group_model
    rng = np.random.default_rng(tpn)
    fails = 0
    models = [I.queens(12), I.model_rb(I.seed_for(I.CFG_RB, 5), 30, 16), I.lin_alldiff(13, n=40, rows=12, groups=4)]
    models += [I.random_tiny(I.seed_for(I.CFG_TINY, 61000 + i)) for i in range(40)]
    models += [mixed_model(s, span) for s in range(3) for span in (40, 100, 250)]
    models += [pooled_wide_model(1000 + s, 250) for s in range(3)]
    models += [group_model(3000 + s, 8 + s, 60, extra=True, ve=True) for s in range(4)]
    for m in models:
        fails += _parity(m, tpn, rng, 6)
    assert fails > 10


def test_huge_node():
    """1000 variables over 0..255 (8 words each), 300 rows and 100 groups: a state is 32 KB,
    too large for eight warps' shared memory; the block kernel and the (narrower) warp
    kernel reach the oracle's fixpoints."""
    m = I.lin_alldiff(I.seed_for(I.CFG_LINAD, 77), n=1000, dmax=255, rows=300, groups=100,
                      gsize=10)
    rng = np.random.default_rng(9)
    for tpn in (256, 1024):
        _parity(m, tpn, rng, 24, check=4)


def test_shapes_are_validated():
    p = K.Csp(I.queens(8))
    with pytest.raises(K.CspError):
        p.set_tiling(K.tiling(threads_per_node=48))          # not a multiple of 32
    p.set_tiling(K.tiling(threads_per_node=256))
    with pytest.raises(K.CspError) as e:                      # the search runs a warp per node
        p.workspace_bytes(K.CSP_ALL, 0)
    assert e.value.code == K.CSP_EINVAL


def test_tuner_picks_a_shape():
    from paper_1909_09213_gb300 import tune
    m = I.lin_alldiff(I.seed_for(I.CFG_LINAD, 78), n=600, dmax=255, rows=180, groups=60, gsize=10)
    om = O.OracleModel(m)
    p = K.Csp(m)
    n, W, lo0 = p.layout()
    rng = np.random.default_rng(3)
    states = np.stack([flags_to_bits(om, f, n, W, lo0) for f in random_subdomains(om, rng, 64)])
    t, entry = tune.tune_propagate(m, states, reps=1, use_cache=False)
    assert t.threads_per_node in (32, 64, 128, 256, 512, 1024)
    assert len(entry["candidates"]) >= 5
