"""GPU parity of the brancher network's kernels against the FP64 reference.

The device takes bf16 weights and inputs, rounds hidden activations to bf16 and accumulates
in fp32; the reference takes the same bf16-rounded weights and inputs.  Against the
reference with the same activation rounding the only difference is fp32 summation order
(and the rare activation that rounds to the other bf16 neighbour); against the
float64-activation reference the tolerance is 2^-7 sqrt(K) relative per layer.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mlp_ref as M
from paper_1909_09213_gb300 import cubics as K

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("rows", [1, 16, 37, 1000])
def test_forward_tensor_core_tiles_match_reference(rows):
    flat = _params(rows)
    X = _features(rows, 7)
    packed = K.mlp_pack(torch.from_numpy(M.to_bf16_bits(flat).view(np.int16)).cuda())
    s = K.mlp_forward(packed, torch.from_numpy(X).cuda()).cpu().numpy()
    ref_r, _ = M.forward(flat, X, act_round=True)
    ref, _ = M.forward(flat, X)
    scale = np.abs(ref).max() + 1e-3
    assert np.max(np.abs(s - ref_r)) <= 2e-2 * scale
    # float64-activation reference: per-layer bound 2^-7 sqrt(K), K = 16, 64, 64
    tol = 2 ** -7 * (np.sqrt(16) + np.sqrt(64) + np.sqrt(64))
    assert np.max(np.abs(s - ref)) <= tol * scale


def test_gradient_matches_reference():
    rows = 4096
    flat = _params(3)
    X = _features(rows, 11)
    y = np.random.default_rng(12).normal(2.0, 1.5, rows).astype(np.float32)
    g, loss = K.mlp_grad(torch.from_numpy(flat).cuda(), torch.from_numpy(X).cuda(),
                         torch.from_numpy(y).cuda())
    g = g.cpu().numpy().astype(np.float64)
    ref_loss, ref_g = M.loss_and_grad(flat, X, y, act_round=True)
    assert abs(float(loss.item()) - ref_loss) <= 1e-3 * ref_loss
    for name, shape in M.SHAPES:
        a, b = M.unflatten(g)[name], M.unflatten(ref_g)[name]
        err = np.linalg.norm(a - b) / (np.linalg.norm(b) + 1e-12)
        assert err <= 1e-2, (name, err)
    _, ref64 = M.loss_and_grad(flat, X, y)
    for name, shape in M.SHAPES:
        a, b = M.unflatten(g)[name], M.unflatten(ref64)[name]
        err = np.linalg.norm(a - b) / (np.linalg.norm(b) + 1e-12)
        assert err <= 2 ** -7 * np.sqrt(64) * 2, (name, err)


def test_adam_matches_reference_and_learns():
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
    losses = []
    for step in range(1, 201):
        g, loss = K.mlp_grad(master, Xd, yd)
        losses.append(float(loss.item()))
        if step == 1:
            _, rg = M.loss_and_grad(M.bf16_round(flat), X, y, act_round=True)
            K.mlp_adam(master, m, v, g, step, 1e-3, params)
            ref, rm, rv = M.adam(ref, rg, rm, rv, 1, lr=1e-3)
            got = master.cpu().numpy()
            # the first Adam step moves every weight by about lr in the gradient's sign
            moved = np.abs(got - flat) > 5e-4
            assert np.mean(np.sign(got - flat)[moved] == np.sign(ref - flat)[moved]) > 0.97
        else:
            K.mlp_adam(master, m, v, g, step, 1e-3, params)
    assert losses[-1] < 0.2 * losses[0]
    bits = params.cpu().numpy().view(np.uint16)
    assert np.array_equal(bits, M.to_bf16_bits(master.cpu().numpy()))
