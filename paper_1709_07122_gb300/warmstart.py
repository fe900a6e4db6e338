"""Learned warm start: training and use of the per-node network.

Orchestration only: every arithmetic step runs in the pcpm_ws_* kernels
(features, targets, forward/backward, Adam, initial ranks). The network
predicts log(n * PR*(v)); the solve then starts from the softmax of the
prediction and runs to the same residual as the uniform start.
"""
from __future__ import annotations

import numpy as np

from . import (PNG, WS_FEATURES, WS_HIDDEN, WS_PARAMS, WS_TRAINABLE, to_device_csr, ws_adam, ws_feature_moments,
               ws_features, ws_init_ranks, ws_loss_grad, ws_predict, ws_standardisation, ws_targets)


def rmat_params(a: float):
    """RMAT quadrant probabilities (a, b, c) for a given a: b = c =
    min(0.19, (0.95 - a) / 2); d = 1 - a - b - c is implied."""
    b = min(0.19, (0.95 - a) / 2)
    return a, b, b


class Sample:
    """Features and targets of one graph, resident on the device."""

    def __init__(self, row_ptr, col, part_size: int, d: float = 0.85, tol: float = 1e-9, max_iters: int = 300):
        drp, dcol = to_device_csr(row_ptr, col)
        self.n = row_ptr.size - 1
        with PNG(drp, dcol, part_size) as g:
            self.features = ws_features(g, drp, dcol)
            pr, self.iters, self.residual = g.pagerank(d, max_iters=max_iters, tol=tol)
        self.target = ws_targets(pr)


def init_params(samples, seed: int = 0):
    """Standardisation from all training features (FP64 moments summed on the
    device) and He-normal initial weights, which are seeded random inputs
    drawn on the host; returns a CUDA float32 tensor [WS_PARAMS]."""
    import torch
    rng = np.random.default_rng(seed)
    F, H = WS_FEATURES, WS_HIDDEN
    p = np.zeros(WS_PARAMS, np.float32)
    o = WS_TRAINABLE
    p[o:o + H * F] = rng.standard_normal(H * F) * np.sqrt(2.0 / F)
    o += H * F + H
    p[o:o + H * H] = rng.standard_normal(H * H) * np.sqrt(2.0 / H)
    o += H * H + H
    p[o:o + H] = rng.standard_normal(H) * np.sqrt(1.0 / H)
    params = torch.from_numpy(p).cuda()
    moments = torch.zeros(11, dtype=torch.float64, device="cuda")
    for s in samples:
        ws_feature_moments(s.features, moments)
    ws_standardisation(moments, params)
    return params


def train(params, samples, steps: int = 600, batch: int = 65536, lr: float = 3e-3, seed: int = 1,
          log_every: int = 100, schedule: str = "constant"):
    """Adam on batches of consecutive rows of a random sample (node labels are
    random, so consecutive rows are a random draw of that graph's nodes).
    schedule "cosine" lowers the step size from lr towards 0 along half a
    cosine over the steps. Returns the loss log [(step, loss)]."""
    import torch
    rng = np.random.default_rng(seed)
    grad = torch.zeros(WS_PARAMS, dtype=torch.float32, device="cuda")
    m = torch.zeros_like(grad)
    v = torch.zeros_like(grad)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    log = []
    for step in range(1, steps + 1):
        s = samples[rng.integers(len(samples))]
        b = min(batch, s.n)
        i0 = int(rng.integers(0, s.n - b + 1))
        ws_loss_grad(params, s.features[i0:i0 + b], s.target[i0:i0 + b], grad, loss)
        step_lr = lr if schedule == "constant" else max(lr * 0.5 * (1.0 + np.cos(np.pi * step / steps)), lr * 1e-3)
        ws_adam(params, grad, m, v, step, step_lr)
        if step % log_every == 0 or step == steps:
            log.append((step, float(loss.item())))
    return log


def warm_start_ranks(params, features):
    """Initial ranks from the network: softmax of its prediction."""
    return ws_init_ranks(ws_predict(params, features))


def evaluate(params, row_ptr, col, part_size: int, d: float = 0.85, tol: float = 1e-7, max_iters: int = 300):
    """Iterations and device time to reach the residual `tol` from the uniform
    start and from the warm start (its features, one PCPM iteration among
    them, and inference counted in its time); both final rank vectors."""
    import torch
    drp, dcol = to_device_csr(row_ptr, col)
    out = {}
    with PNG(drp, dcol, part_size) as g:
        g.pagerank(d, max_iters=3)  # warm-up
        for name in ("uniform", "warm"):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            x0 = None
            if name == "warm":
                x0 = warm_start_ranks(params, ws_features(g, drp, dcol))
            pr, iters, res = g.pagerank(d, max_iters=max_iters, tol=tol, pr_init=x0)
            e1.record()
            torch.cuda.synchronize()
            out[name] = {"iters": iters, "ms": e0.elapsed_time(e1), "residual": res, "ranks": pr.clone()}
    return out
