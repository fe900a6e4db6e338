"""FP64 reference of the learned warm start (test infrastructure only).

Not in the paper. A per-node MLP predicts log(n * PR*(v)) from degree features
and one PageRank iteration, so that power iteration (Eq. 1) can start from
softmax(prediction) instead of 1/n. This module restates, in plain numpy FP64,
what the CUDA kernels compute: the features, the network's forward pass, the
mean-squared-error loss with its gradient, and the Adam update. Only the
tests and the benchmark may import it.

Features of node v (F = 5):
  0  log1p(indeg(v))
  1  log1p(outdeg(v))
  2  log1p(sum over in-neighbours u of indeg(u))
  3  log1p(sum over in-neighbours u of outdeg(u))
  4  log(n * PR_1(v)), PR_1 = one Eq. 1 step from the uniform start
     (d = 0.85, dangling mass spread uniformly)

Parameters, one flat float array (P = 4619 entries), in this order:
  mu[5], inv_sigma[5]          input standardisation (not trained)
  W1[64][5], b1[64]            layer 1, ReLU
  W2[64][64], b2[64]           layer 2, ReLU
  w3[64], b3                   output
"""
from __future__ import annotations

import numpy as np

from . import pagerank as _pagerank

F, H = 5, 64
OFF_MU, OFF_IS = 0, F
OFF_W1 = 2 * F
OFF_B1 = OFF_W1 + H * F
OFF_W2 = OFF_B1 + H
OFF_B2 = OFF_W2 + H * H
OFF_W3 = OFF_B2 + H
OFF_B3 = OFF_W3 + H
P = OFF_B3 + 1
TRAINABLE = slice(OFF_W1, P)


def unpack(params):
    p = np.asarray(params, dtype=np.float64)
    assert p.size == P
    return dict(mu=p[OFF_MU:OFF_MU + F], inv_sigma=p[OFF_IS:OFF_IS + F],
                W1=p[OFF_W1:OFF_B1].reshape(H, F), b1=p[OFF_B1:OFF_W2],
                W2=p[OFF_W2:OFF_B2].reshape(H, H), b2=p[OFF_B2:OFF_W3],
                w3=p[OFF_W3:OFF_B3], b3=p[OFF_B3])


def features(row_ptr, col, d: float = 0.85):
    """The five features above, FP64, shape (n, 5)."""
    rp = np.asarray(row_ptr, dtype=np.int64)
    c = np.asarray(col, dtype=np.int64)
    n = rp.size - 1
    outdeg = np.diff(rp)
    src = np.repeat(np.arange(n), outdeg)
    indeg = np.bincount(c, minlength=n).astype(np.int64)
    s_in = np.zeros(n, dtype=np.int64)
    s_out = np.zeros(n, dtype=np.int64)
    np.add.at(s_in, c, indeg[src])
    np.add.at(s_out, c, outdeg[src])
    pr1 = _pagerank(rp.astype(np.uint32), c.astype(np.uint32), d, iters=1)["x"]
    return np.stack([np.log1p(indeg), np.log1p(outdeg), np.log1p(s_in.astype(np.float64)),
                     np.log1p(s_out.astype(np.float64)), np.log(n * pr1)], axis=1)


def forward(params, x, cache: bool = False):
    """Network output for feature rows x (n, 5); with cache, also the
    intermediate values the backward pass needs."""
    q = unpack(params)
    xh = (np.asarray(x, np.float64) - q["mu"]) * q["inv_sigma"]
    z1 = xh @ q["W1"].T + q["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ q["W2"].T + q["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ q["w3"] + q["b3"]
    if cache:
        return y, dict(xh=xh, z1=z1, h1=h1, z2=z2, h2=h2)
    return y


def loss_and_grad(params, x, target):
    """L = sum_v (y(v) - t(v))^2 / n and dL/dparams (zero for mu, inv_sigma)."""
    q = unpack(params)
    y, c = forward(params, x, cache=True)
    n = y.size
    r = y - np.asarray(target, np.float64)
    loss = float((r * r).sum() / n)
    dy = 2.0 * r / n
    g = np.zeros(P)
    g[OFF_W3:OFF_B3] = c["h2"].T @ dy
    g[OFF_B3] = dy.sum()
    dz2 = np.outer(dy, q["w3"]) * (c["z2"] > 0)
    g[OFF_W2:OFF_B2] = (dz2.T @ c["h1"]).ravel()
    g[OFF_B2:OFF_W3] = dz2.sum(axis=0)
    dz1 = (dz2 @ q["W2"]) * (c["z1"] > 0)
    g[OFF_W1:OFF_B1] = (dz1.T @ c["xh"]).ravel()
    g[OFF_B1:OFF_W2] = dz1.sum(axis=0)
    return loss, g


def adam(params, grad, m, v, step: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
         eps: float = 1e-8):
    """One Adam step (Kingma and Ba, 2015, Algorithm 1) on the trainable
    entries; returns new (params, m, v)."""
    p = np.array(params, np.float64)
    m = np.array(m, np.float64)
    v = np.array(v, np.float64)
    g = np.asarray(grad, np.float64)
    s = TRAINABLE
    m[s] = beta1 * m[s] + (1 - beta1) * g[s]
    v[s] = beta2 * v[s] + (1 - beta2) * g[s] * g[s]
    mhat = m[s] / (1 - beta1 ** step)
    vhat = v[s] / (1 - beta2 ** step)
    p[s] -= lr * mhat / (np.sqrt(vhat) + eps)
    return p, m, v


def warm_start(pred):
    """Initial ranks from predicted log(n * PR): softmax, summing to 1."""
    e = np.exp(np.asarray(pred, np.float64) - np.max(pred))
    return e / e.sum()
