"""Pins of the FP64 network reference: gradients against central finite differences, closed
forms, bfloat16 rounding, and Adam's first step."""
import numpy as np

from oracle import mlp_ref as M


def test_parameter_count():
    assert M.N_PARAMS == 5313


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    flat = M.init_params(1).astype(np.float64)
    X = rng.normal(size=(37, 16))
    y = rng.normal(size=37)
    loss, g = M.loss_and_grad(flat, X, y)
    idx = rng.choice(M.N_PARAMS, 300, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(flat)
        e[i] = h
        num = (M.loss_and_grad(flat + e, X, y)[0] - M.loss_and_grad(flat - e, X, y)[0]) / (2 * h)
        assert abs(num - g[i]) <= 1e-6 + 1e-5 * abs(num), (i, num, g[i])


def test_closed_forms():
    # zero weights: every score is b3; the loss gradient of b3 is 2 mean(b3 - y)
    flat = np.zeros(M.N_PARAMS)
    p = M.unflatten(flat)
    p["b3"][0] = 0.75
    flat = M.flatten(p)
    X = np.random.default_rng(1).normal(size=(10, 16))
    y = np.arange(10, dtype=float)
    s, _ = M.forward(flat, X)
    assert np.allclose(s, 0.75)
    loss, g = M.loss_and_grad(flat, X, y)
    assert np.isclose(loss, np.mean((0.75 - y) ** 2))
    assert np.isclose(M.unflatten(g)["b3"][0], 2 * np.mean(0.75 - y))
    # a single active path: s = w3[j] * relu(W2[i, j] * relu(W1[k, i] * x_k))
    p = M.unflatten(np.zeros(M.N_PARAMS))
    p["W1"][3, 5] = 2.0
    p["W2"][5, 7] = -1.5
    p["w3"][7] = 0.5
    x = np.zeros((2, 16))
    x[0, 3] = 1.0
    x[1, 3] = -1.0
    s, _ = M.forward(M.flatten(p), x)
    assert np.allclose(s, [0.0, 0.0])           # the second layer's output is negative: relu
    p["W2"][5, 7] = 1.5
    s, _ = M.forward(M.flatten(p), x)
    assert np.allclose(s, [0.5 * 1.5 * 2.0, 0.0])


def test_bf16_rounding():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7, 1.0 + 3 * 2 ** -8, -2.5, 0.0, 1e-40], np.float32)
    r = M.bf16_round(vals)
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: to even (1); 1 + 3*2^-8 rounds up to 1 + 2^-6
    assert list(r[:4]) == [1.0, 1.0, 1.0 + 2 ** -7, 1.0 + 2 ** -6]
    assert r[4] == -2.5 and r[5] == 0.0
    assert np.array_equal(M.from_bf16_bits(M.to_bf16_bits(vals)), r)


def test_adam_first_step_is_sign_times_lr():
    flat = np.ones(5)
    g = np.array([0.3, -2.0, 1e-3, 0.0, 5.0])
    new, m, v = M.adam(flat, g, np.zeros(5), np.zeros(5), 1, lr=0.01)
    expect = 1 - 0.01 * np.sign(g) * (np.abs(g) / (np.abs(g) + 1e-8))
    assert np.allclose(new, expect)


def test_activation_rounding_closed_form():
    # one active path x3 -> h5 -> h7 -> s with unit weights downstream: the hidden values are
    # rounded to bf16 (8 significant bits) when act_round is on
    p = M.unflatten(np.zeros(M.N_PARAMS))
    p["W2"][5, 7] = 1.0
    p["w3"][7] = 1.0
    x = np.zeros((1, 16))
    x[0, 3] = 1.0
    # 1 + 2^-8 + 2^-10 lies above the midpoint 1 + 2^-8 of 1 and 1 + 2^-7: rounds up
    p["W1"][3, 5] = 1.0 + 2 ** -8 + 2 ** -10
    s, _ = M.forward(M.flatten(p), x, act_round=True)
    assert s[0] == 1.0 + 2 ** -7
    s, _ = M.forward(M.flatten(p), x)
    assert s[0] == 1.0 + 2 ** -8 + 2 ** -10
    # exactly the midpoint: a tie, to the even neighbour 1
    p["W1"][3, 5] = 1.0 + 2 ** -8
    s, _ = M.forward(M.flatten(p), x, act_round=True)
    assert s[0] == 1.0
    # the second layer rounds too: H2 = bf16(3 * (1 + 2^-7)) = bf16(3 + 3 * 2^-7); the bf16
    # spacing in [2, 4) is 2^-6, and 3 + 3 * 2^-7 = 3 + 1.5 * 2^-6 rounds to 3 + 2 * 2^-6
    p["W1"][3, 5] = 1.0 + 2 ** -7
    p["W2"][5, 7] = 3.0
    s, (_, _, H1, Z2, H2) = M.forward(M.flatten(p), x, act_round=True)
    assert H1[0, 5] == 1.0 + 2 ** -7 and Z2[0, 7] == 3.0 + 3 * 2 ** -7
    assert s[0] == H2[0, 7] == 3.0 + 2 ** -5
    # negative pre-activations are cut by the ReLU before rounding
    p["W2"][5, 7] = -3.0
    s, _ = M.forward(M.flatten(p), x, act_round=True)
    assert s[0] == 0.0
