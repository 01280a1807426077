"""FP64 reference of the learned brancher's network (test infrastructure only).

The network scores a variable from its 16 features: s = w3 . relu(W2^T relu(W1^T x + b1) + b2)
+ b3 (16 -> 64 -> 64 -> 1).  The GPU computes with bfloat16 weights and activations and fp32
accumulation; this reference takes the same bfloat16-rounded weights and inputs and works
in float64, so the two differ only by the GPU's rounding of activations and sums.

Loss: mean squared error between s and the target (log2 of the subtree size).  Update: Adam
on fp32 master weights (Kingma and Ba 2015).

Shared with nothing on the CUDA side; only tests/ and bench.py may import it.
"""
from __future__ import annotations

import numpy as np

SHAPES = [("W1", (16, 64)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)), ("w3", (64,)), ("b3", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)          # 5313


def bf16_round(a) -> np.ndarray:
    """Round float32 values to bfloat16 (round to nearest even), returned as float32."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    rounded = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    out = (rounded & 0xFFFFFFFF).astype(np.uint32).view(np.float32)
    return np.where(np.isnan(a), a, out)


def to_bf16_bits(a) -> np.ndarray:
    return (bf16_round(a).view(np.uint32) >> 16).astype(np.uint16)


def from_bf16_bits(b) -> np.ndarray:
    return (np.asarray(b, dtype=np.uint32) << 16).view(np.float32)


def unflatten(flat):
    flat = np.asarray(flat, dtype=np.float64).reshape(-1)
    assert flat.size == N_PARAMS
    out, o = {}, 0
    for name, shape in SHAPES:
        k = int(np.prod(shape))
        out[name] = flat[o:o + k].reshape(shape)
        o += k
    return out


def flatten(p) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).reshape(-1) for name, _ in SHAPES])


def init_params(seed: int = 0) -> np.ndarray:
    """He-style initialisation from a numpy Generator (host side only)."""
    rng = np.random.default_rng(seed)
    p = {"W1": rng.normal(0, np.sqrt(2 / 16), (16, 64)), "b1": np.zeros(64),
         "W2": rng.normal(0, np.sqrt(2 / 64), (64, 64)), "b2": np.zeros(64),
         "w3": rng.normal(0, np.sqrt(1 / 64), (64,)), "b3": np.zeros(1)}
    return flatten(p).astype(np.float32)


def _act(a, act_round):
    return bf16_round(a.astype(np.float32)).astype(np.float64) if act_round else a


def forward(flat, X, act_round=False):
    """Scores of the rows of X (B x 16): returns s (B,) and the activations.  With
    act_round the hidden activations are rounded to bfloat16, as the device stores them."""
    p = unflatten(flat)
    X = np.asarray(X, dtype=np.float64)
    Z1 = X @ p["W1"] + p["b1"]
    H1 = _act(np.maximum(Z1, 0.0), act_round)
    Z2 = H1 @ p["W2"] + p["b2"]
    H2 = _act(np.maximum(Z2, 0.0), act_round)
    s = H2 @ p["w3"] + p["b3"][0]
    return s, (X, Z1, H1, Z2, H2)


def loss_and_grad(flat, X, y, act_round=False):
    """Mean squared error and its gradient with respect to the flat parameters (the
    activation rounding, when on, is treated as the identity in the backward pass)."""
    p = unflatten(flat)
    s, (X, Z1, H1, Z2, H2) = forward(flat, X, act_round)
    B = X.shape[0]
    r = s - np.asarray(y, dtype=np.float64)
    loss = float(np.mean(r * r))
    ds = 2.0 * r / B
    g = {"w3": H2.T @ ds, "b3": np.array([ds.sum()])}
    dZ2 = np.outer(ds, p["w3"]) * (Z2 > 0)
    g["W2"] = H1.T @ dZ2
    g["b2"] = dZ2.sum(axis=0)
    dZ1 = (dZ2 @ p["W2"].T) * (Z1 > 0)
    g["W1"] = X.T @ dZ1
    g["b1"] = dZ1.sum(axis=0)
    return loss, flatten(g)


def adam(flat, grad, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (t counts from 1); returns new (flat, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return flat - lr * mh / (np.sqrt(vh) + eps), m, v
