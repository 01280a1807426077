"""GPU parity of the brancher network's kernels against the FP64 reference, element by element.

The device takes bf16 weights and inputs, rounds hidden activations to bf16 and accumulates
in fp32; the reference (oracle/mlp_ref.py) takes the same bf16 weights and inputs, computes
in float64 and rounds the activations at the same points (act_round=True).

Exact cases.  With dyadic inputs (small integers times powers of two) every product and
partial sum of the forward pass is a multiple of a known granule g and bounded by the sum of
the absolute terms A; when A / g < 2^24 every partial sum, in any order and on the tensor
cores as on the CUDA cores, is exactly representable in fp32.  The forward pass is then exact
on both sides, the bf16 rounding of each activation is decided on the same value, and the
scores must equal the reference's bit for bit.  The tests check that precondition on the
drawn data before they rely on it.

Bounds.  In the backward pass the sums over the rows of the batch are rounded.  Recursive
summation of n terms in any order errs by at most gamma_n * sum |terms| with
gamma_n = n u / (1 - n u), u = 2^-24 (Higham, Accuracy and Stability of Numerical
Algorithms, section 4.2); a quantity computed from already-rounded sums inherits their bound
through the absolute values.  Each gradient element is checked against that bound.  Adam's
fp32 constants 0.9f and 0.999f differ from 0.9 and 0.999 by at most u/2 each, which is a
relative error of up to 500 u in 1 - beta2; the bounds below add those terms.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mlp_ref as M
from paper_1909_09213_gb300 import cubics as K

pytestmark = pytest.mark.gpu

U = 2.0 ** -24


def gamma(n):
    return n * U / (1 - n * U)


@pytest.fixture(autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _params(seed):
    flat = M.init_params(seed)
    p = M.unflatten(flat)
    rng = np.random.default_rng(seed + 100)
    p["b1"] = rng.normal(0, 0.1, 64)
    p["b2"] = rng.normal(0, 0.1, 64)
    p["b3"] = rng.normal(0, 0.1, 1)
    return M.bf16_round(M.flatten(p).astype(np.float32))


def _features(rows, seed):
    rng = np.random.default_rng(seed)
    return M.bf16_round(rng.uniform(-1, 2, size=(rows, 16)).astype(np.float32))


# granules of the dyadic draws: X 2^-2, W1 2^-5, b1 2^-7 -> Z1, H1 2^-7; W2 2^-5, b2 2^-12 ->
# Z2, H2 2^-12; w3 2^-3, b3 2^-15 -> s 2^-15
G1, G2, G3 = 2.0 ** -7, 2.0 ** -12, 2.0 ** -15


def _dyadic_params(seed):
    rng = np.random.default_rng(seed)
    p = {"W1": rng.integers(-16, 17, (16, 64)) / 32.0, "b1": rng.integers(-16, 17, 64) / 128.0,
         "W2": rng.integers(-8, 9, (64, 64)) / 32.0, "b2": rng.integers(-64, 65, 64) / 4096.0,
         "w3": rng.integers(-2, 3, 64) / 8.0, "b3": rng.integers(-64, 65, 1) / 32768.0}
    flat = M.flatten(p).astype(np.float32)
    assert np.array_equal(M.bf16_round(flat), flat)          # every weight is a bf16 value
    return flat


def _dyadic_features(rows, seed):
    X = (np.random.default_rng(seed).integers(-4, 5, (rows, 16)) / 4.0).astype(np.float32)
    assert np.array_equal(M.bf16_round(X), X)
    return X


def _assert_exact_forward(flat, X):
    """The precondition of exactness: each layer's absolute sum over its granule < 2^24."""
    p = M.unflatten(flat)
    _, (X64, Z1, H1, Z2, H2) = M.forward(flat, X, act_round=True)
    a1 = np.abs(X64) @ np.abs(p["W1"]) + np.abs(p["b1"])
    a2 = np.abs(H1) @ np.abs(p["W2"]) + np.abs(p["b2"])
    a3 = np.abs(H2) @ np.abs(p["w3"]) + abs(p["b3"][0])
    assert a1.max() / G1 < 2 ** 24 and a2.max() / G2 < 2 ** 24 and a3.max() / G3 < 2 ** 24
    # the activations stay on their granules after bf16 rounding
    assert np.all(np.mod(H1 / G1, 1.0) == 0) and np.all(np.mod(H2 / G2, 1.0) == 0)


def _forward(flat, X):
    packed = K.mlp_pack(torch.from_numpy(M.to_bf16_bits(flat).view(np.int16)).cuda())
    return K.mlp_forward(packed, torch.from_numpy(X).cuda()).cpu().numpy()


@pytest.mark.parametrize("rows", [1, 16, 37, 1000])
def test_forward_is_exact_on_dyadic_inputs(rows):
    flat = _dyadic_params(rows)
    X = _dyadic_features(rows, 7 + rows)
    _assert_exact_forward(flat, X)
    s = _forward(flat, X)
    ref, _ = M.forward(flat, X, act_round=True)
    assert np.array_equal(s, ref.astype(np.float32)), np.flatnonzero(s != ref.astype(np.float32))[:8]


@pytest.mark.parametrize("rows", [1, 16, 37, 1000])
def test_forward_within_rounding_bound(rows):
    """Non-dyadic inputs: every score within the first-order effect of one bf16 ulp
    (2^-7 relative) on every activation, plus fp32 accumulation, of the reference's."""
    flat = _params(rows)
    X = _features(rows, 7)
    s = _forward(flat, X)
    p = M.unflatten(flat)
    ref, (X64, Z1, H1, Z2, H2) = M.forward(flat, X, act_round=True)
    aw3, aW2 = np.abs(p["w3"]), np.abs(p["W2"])
    flips = 2.0 ** -7 * (np.abs(H2) @ aw3 + (np.abs(H1) @ aW2) @ aw3)
    acc = gamma(90) * ((np.abs(X64) @ np.abs(p["W1"]) + np.abs(p["b1"])) @ aW2 @ aw3
                       + np.abs(H2) @ aw3 + abs(p["b3"][0]))
    bound = 2 * (flips + acc) + 1e-30
    err = np.abs(s - ref)
    assert np.all(err <= bound), (np.argmax(err / bound), float(np.max(err / bound)))


def _abs_grad(flat, X, y):
    """Per parameter: the sum of the absolute values of the terms whose rounded sums make
    up its gradient (the quantity that bounds the fp32 summation error)."""
    p = M.unflatten(flat)
    s, (X64, Z1, H1, Z2, H2) = M.forward(flat, X, act_round=True)
    B = X.shape[0]
    ads = np.abs(2.0 * (s - y) / B)
    adZ2 = np.outer(ads, np.abs(p["w3"])) * (Z2 > 0)
    adZ1 = (adZ2 @ np.abs(p["W2"]).T) * (Z1 > 0)
    g = {"w3": np.abs(H2).T @ ads, "b3": np.array([ads.sum()]), "W2": np.abs(H1).T @ adZ2,
         "b2": adZ2.sum(axis=0), "W1": np.abs(X64).T @ adZ1, "b1": adZ1.sum(axis=0)}
    return M.flatten(g)


def _grad(flat, X, y):
    g, loss = K.mlp_grad(torch.from_numpy(flat).cuda(), torch.from_numpy(X).cuda(),
                         torch.from_numpy(y.astype(np.float32)).cuda())
    return g.cpu().numpy().astype(np.float64), float(loss.item())


@pytest.mark.parametrize("rows", [4096, 777])
def test_gradient_per_element_on_dyadic_inputs(rows):
    flat = _dyadic_params(50 + rows)
    X = _dyadic_features(rows, 11)
    _assert_exact_forward(flat, X)
    s, _ = M.forward(flat, X, act_round=True)
    # targets on the score's granule, so that the residual s - y is exact too
    y = s + np.random.default_rng(12).integers(-2 ** 15, 2 ** 15, rows) / 2.0 ** 15
    assert np.all(np.mod(y / G3, 1.0) == 0)
    g, loss = _grad(flat, X, y)
    ref_loss, ref_g = M.loss_and_grad(flat, X, y, act_round=True)
    bound = gamma(rows + 70) * _abs_grad(flat, X, y) + 1e-30
    err = np.abs(g - ref_g)
    bad = np.flatnonzero(err > bound)
    assert bad.size == 0, (bad[:8], err[bad[:8]], bound[bad[:8]])
    assert abs(loss - ref_loss) <= gamma(rows + 4) * ref_loss
    # the bound is far below the size of the gradient (a few per cent of it in the median,
    # because the terms of a sum cancel): a dropped or misplaced term shows
    nz = np.abs(ref_g) > 0
    assert np.median(bound[nz] / np.abs(ref_g[nz])) < 5e-2


def test_gradient_matches_reference_on_random_inputs():
    """Non-dyadic inputs: a few activations may round to the other bf16 neighbour, so the
    comparison is by relative norm per tensor (against the same-rounding reference) and by
    the per-layer 2^-7 sqrt(K) bound (against the float64-activation reference)."""
    rows = 4096
    flat = _params(3)
    X = _features(rows, 11)
    y = np.random.default_rng(12).normal(2.0, 1.5, rows).astype(np.float32)
    g, loss = _grad(flat, X, y)
    ref_loss, ref_g = M.loss_and_grad(flat, X, y, act_round=True)
    assert abs(loss - ref_loss) <= 1e-3 * ref_loss
    for name, shape in M.SHAPES:
        a, b = M.unflatten(g)[name], M.unflatten(ref_g)[name]
        err = np.linalg.norm(a - b) / (np.linalg.norm(b) + 1e-12)
        assert err <= 1e-2, (name, err)
    _, ref64 = M.loss_and_grad(flat, X, y)
    for name, shape in M.SHAPES:
        a, b = M.unflatten(g)[name], M.unflatten(ref64)[name]
        err = np.linalg.norm(a - b) / (np.linalg.norm(b) + 1e-12)
        assert err <= 2 ** -7 * np.sqrt(64) * 2, (name, err)


def test_adam_per_element_and_learns():
    """Three Adam steps fed the same gradients on both sides: m, v and the master weights
    element by element against the FP64 update, then a training run that lowers the loss."""
    rows = 2048
    rng = np.random.default_rng(5)
    X = _features(rows, 21)
    w_true = rng.normal(size=16)
    y = (X @ w_true).astype(np.float32)                 # a learnable target
    flat = M.init_params(9)
    master = torch.from_numpy(flat.copy()).cuda()
    m = torch.zeros_like(master)
    v = torch.zeros_like(master)
    params = torch.zeros(M.N_PARAMS, dtype=torch.int16, device="cuda")
    Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    ref, rm, rv = flat.astype(np.float64), np.zeros(M.N_PARAMS), np.zeros(M.N_PARAMS)
    am, av = np.zeros(M.N_PARAMS), np.zeros(M.N_PARAMS)   # the same recurrences on |g|
    lr = 1e-3
    losses = []
    for step in range(1, 201):
        g, loss = K.mlp_grad(master, Xd, yd)
        losses.append(float(loss.item()))
        K.mlp_adam(master, m, v, g, step, lr, params)
        if step <= 3:
            g64 = g.cpu().numpy().astype(np.float64)
            w_prev = ref
            ref, rm, rv = M.adam(ref, g64, rm, rv, step, lr=lr)
            am = 0.9 * am + 0.1 * np.abs(g64)
            av = 0.999 * av + 0.001 * g64 * g64
            got_m, got_v = m.cpu().numpy(), v.cpu().numpy()
            got_w = master.cpu().numpy()
            # m: two rounded products and a sum per step, 0.9f and 1 - 0.9f within 4 u
            assert np.all(np.abs(got_m - rm) <= 16 * step * U * am + 1e-38)
            # v: as m, plus 1 - 0.999f within 500 u of 0.001
            assert np.all(np.abs(got_v - rv) <= (600 + 16 * step) * U * av + 1e-38)
            # the update lr * mh / (sqrt(vh) + eps): bias corrections with powf (within 8 u of
            # beta^t) over 1 - beta^t >= 0.001 give at most 1e-2 relative error in the step at
            # step 1..3 (9000 u in vh, halved by the square root, plus the m and v terms);
            # then one rounding of the new weight
            step_ref = np.abs(ref - w_prev)
            assert np.all(np.abs(got_w - ref) <= 1e-2 * step_ref + U * np.abs(ref) + 1e-12)
            # the step is about lr in size: the check above is far tighter than the step
            assert np.median(step_ref) > 0.5 * lr
            # keep both sides on the same weights for the next step
            ref = got_w.astype(np.float64)
    assert losses[-1] < 0.2 * losses[0]
    bits = params.cpu().numpy().view(np.uint16)
    assert np.array_equal(bits, M.to_bf16_bits(master.cpu().numpy()))
