"""Training and evaluation of the learned brancher.

1. collect: exhaustive searches of a batch of instances with subtree logging on — every
   sampled completed search level gives (features of its branching variable, log2 of the
   nodes in its subtree);
2. train: mean squared error with Adam, mini-batches of 4096, using the library's own
   gradient and update kernels (csp_mlp_grad, csp_mlp_adam); fp32 master weights, bf16
   weights for inference;
3. evaluate: the same batch solved with first-fail and with the learned brancher.

Torch only holds buffers and shuffles indices; the arithmetic runs in libcubics.so.
"""
from __future__ import annotations

import time

import numpy as np

from . import cubics as K

N_FEAT = 16


def collect(models, cap=4_000_000, sample=8, mode=K.CSP_ALL, stream=None, lim=None):
    """Subtree logs of the searches of `models` (exhaustive in CSP_ALL mode; in CSP_FIRST
    mode the levels refuted before the first solution): a (rows, 17) float32 CUDA tensor.
    `lim`: csp_limits (a node limit per instance; instances that reach it still log the
    levels they completed)."""
    import torch
    probs = [K.Csp(m) for m in models]
    b = K.Batch(probs)
    b.set_tiling(K.tiling(warps_per_block=1, smem_levels=8))
    log = torch.zeros((cap, N_FEAT + 1), dtype=torch.float32, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    K._check(K.lib().csp_batch_set_log(b.b, K._dp(log), K._dp(count), cap, sample), "csp_batch_set_log")
    t0 = time.time()
    rc, res = b.solve(mode, lim=lim)
    if rc != 0:
        raise RuntimeError(f"logging search failed: {rc}")
    n = min(int(count.item()), cap)
    st = b.stats()
    info = {"entries": n, "logged": int(count.item()), "nodes": sum(r["nodes"] for r in res),
            "ms": st["ms"], "wall_s": time.time() - t0}
    return log[:n].clone(), info


def init_params(seed: int = 0, out_bias: float = 0.0) -> np.ndarray:
    """He-style initial weights in the flat layout of csp_set_brancher (float32), output bias
    set to `out_bias` (the mean target, so training starts from the constant predictor)."""
    rng = np.random.default_rng(seed)
    parts = [rng.normal(0, np.sqrt(2 / 16), 16 * 64), np.zeros(64),
             rng.normal(0, np.sqrt(2 / 64), 64 * 64), np.zeros(64),
             rng.normal(0, np.sqrt(1 / 64), 64), np.array([out_bias])]
    return np.concatenate(parts).astype(np.float32)


def train(data, epochs=8, batch=4096, lr=1e-3, seed=0, verbose=False):
    """Adam on the logged data; returns (bf16 params as uint16 numpy, info)."""
    import torch
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    X = data[:, :N_FEAT].contiguous()
    y = data[:, N_FEAT].contiguous()
    master = torch.from_numpy(init_params(seed, float(y.mean().item()))).cuda()
    m = torch.zeros_like(master)
    v = torch.zeros_like(master)
    params = torch.zeros(K.MLP_PARAMS, dtype=torch.int16, device="cuda")
    rows = X.shape[0]
    steps, losses = 0, []
    t0 = time.time()
    for ep in range(epochs):
        perm = torch.randperm(rows, device="cuda", generator=g)
        ep_loss, nb = 0.0, 0
        for s in range(0, rows - batch + 1 if rows >= batch else 1, batch):
            idx = perm[s:s + batch]
            xb, yb = X[idx].contiguous(), y[idx].contiguous()
            grad, loss = K.mlp_grad(master, xb, yb)
            steps += 1
            K.mlp_adam(master, m, v, grad, steps, lr, params)
            ep_loss += float(loss.item()) if nb % 50 == 0 else 0.0
            nb += 1
        # full-data loss at the end of the epoch (sampled mini-batch of up to 65536 rows)
        sel = perm[: min(rows, 65536)]
        _, l_all = K.mlp_grad(master, X[sel].contiguous(), y[sel].contiguous())
        losses.append(float(l_all.item()))
        if verbose:
            print(f"epoch {ep}: mse {losses[-1]:.4f}", flush=True)
    torch.cuda.synchronize()
    var = float(y.var().item()) if rows > 1 else 0.0
    info = {"steps": steps, "mse_per_epoch": losses, "target_variance": var,
            "train_s": time.time() - t0, "rows": rows}
    return params.cpu().numpy().view(np.uint16).copy(), info


def learning_config(train_count=20000, eval_count=1024, epochs=8, sample=1, cap=8_000_000,
                    eval_tiling=None, verbose=False):
    """The learning configuration end to end: exhaustive, logged searches of `train_count`
    model-RB instances (n = 30, d = 16), training, then first-solution searches of
    `eval_count` held-out instances (n = 80, d = 20) with first-fail and with the network."""
    from . import instances as I
    t0 = time.time()
    train_models = I.rb_batch(train_count, n_range=(30, 30), d_range=(16, 16), config_id=I.CFG_RB_TRAIN)
    eval_models = I.rb_batch(eval_count, n_range=(80, 80), d_range=(20, 20), config_id=I.CFG_RB_EVAL)
    gen_s = time.time() - t0
    data, cinfo = collect(train_models, cap=cap, sample=sample)
    if verbose:
        print("collected", cinfo, flush=True)
    params, tinfo = train(data, epochs=epochs, verbose=verbose)
    ev = evaluate(eval_models, params, tiling=eval_tiling, reps=2)
    same = ev["first_fail"]["status"] == ev["learned"]["status"]
    return {"generate_s": gen_s, "collect": cinfo, "train": tinfo, "same_status": same,
            "first_fail_ms": ev["first_fail"]["ms"], "learned_ms": ev["learned"]["ms"],
            "first_fail_nodes": ev["first_fail"]["nodes"], "learned_nodes": ev["learned"]["nodes"],
            "sat": sum(s == 1 for s in ev["learned"]["status"]), "eval": ev, "params": params,
            "eval_models": eval_models}


def linad_training(train_count=2048, node_limit=40_000, epochs=16):
    """The brancher of the mixed linear/alldifferent workload: first-solution searches of
    `train_count` training-seed instances of the same generator (200 vars on 0..255, 8-word
    domains), at most `node_limit` nodes each, log the sizes of the levels they refute before
    a solution (every completed level is a subtree without solution); the network is trained
    on those logs.  Returns (bf16 params, info)."""
    from . import instances as I
    t0 = time.time()
    models = I.linad_batch(train_count, config_id=I.CFG_LINAD_TRAIN)
    gen_s = time.time() - t0
    data, cinfo = collect(models, cap=8_000_000, sample=1, mode=K.CSP_FIRST,
                          lim=K.limits(node_limit=node_limit))
    params, tinfo = train(data, epochs=epochs)
    return params, {"generate_s": gen_s, "collect": cinfo, "train": tinfo,
                    "train_instances": train_count, "node_limit": node_limit}


def evaluate(models, params_bf16, mode=K.CSP_FIRST, tiling=None, reps=1, stream=None):
    """Solve `models` as one batch with first-fail and with the learned brancher."""
    out = {}
    for name in ("first_fail", "learned"):
        probs = [K.Csp(m) for m in models]
        b = K.Batch(probs)
        if tiling is not None:
            b.set_tiling(tiling)
        if name == "learned":
            w = np.ascontiguousarray(params_bf16, dtype=np.uint16)
            K._check(K.lib().csp_batch_set_brancher(b.b, K.CSP_BR_LEARNED, w.ctypes.data_as(K._U16P)),
                     "csp_batch_set_brancher")
        best, res = None, None
        for _ in range(reps):
            rc, res = b.solve(mode)
            if rc != 0:
                raise RuntimeError(f"{name} batch failed: {rc}")
            ms = b.stats()["ms"]
            best = ms if best is None else min(best, ms)
        out[name] = {"ms": best, "nodes": sum(r["nodes"] for r in res),
                     "status": [r["status"] for r in res], "results": res}
    return out
