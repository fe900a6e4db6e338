"""The warm-start gradient bound (tests/ws_bounds.py) on the CPU: it holds
for the network evaluated in FP32 arithmetic (numpy float32, the same steps
as the FP64 reference), and plausible mistakes in a gradient exceed it."""
import numpy as np

from oracle import warmstart as ows
from ws_bounds import gradient_bound


def fp32_loss_grad(p, x, t):
    """The FP64 reference's steps in float32 arithmetic (test-only emulation
    of the kernels' precision; the order of the sums differs)."""
    f32 = np.float32
    q = {k: np.asarray(v, f32) for k, v in ows.unpack(p).items()}
    xh = ((x.astype(f32) - q["mu"]) * q["inv_sigma"]).astype(f32)
    z1 = xh @ q["W1"].T + q["b1"]
    h1 = np.maximum(z1, f32(0))
    z2 = h1 @ q["W2"].T + q["b2"]
    h2 = np.maximum(z2, f32(0))
    y = h2 @ q["w3"] + q["b3"]
    dy = (f32(2) * (y - t.astype(f32)) / f32(y.size)).astype(f32)
    g = np.zeros(ows.P, f32)
    g[ows.OFF_W3:ows.OFF_B3] = h2.T @ dy
    g[ows.OFF_B3] = dy.sum(dtype=f32)
    dz2 = (np.outer(dy, q["w3"]) * (z2 > 0)).astype(f32)
    g[ows.OFF_W2:ows.OFF_B2] = (dz2.T @ h1).ravel()
    g[ows.OFF_B2:ows.OFF_W3] = dz2.sum(axis=0, dtype=f32)
    dz1 = ((dz2 @ q["W2"]) * (z1 > 0)).astype(f32)
    g[ows.OFF_W1:ows.OFF_B1] = (dz1.T @ xh).ravel()
    g[ows.OFF_B1:ows.OFF_W2] = dz1.sum(axis=0, dtype=f32)
    return g.astype(np.float64)


def case(seed, rows=2000):
    rng = np.random.default_rng(seed)
    p = rng.standard_normal(ows.P) * 0.2
    p[:5] = rng.standard_normal(5)
    p[5:10] = 0.5 + rng.random(5)
    p = p.astype(np.float32).astype(np.float64)
    x = (rng.standard_normal((rows, 5)) * 2).astype(np.float32).astype(np.float64)
    t = rng.standard_normal(rows).astype(np.float32).astype(np.float64)
    return p, x, t


def test_bound_holds_for_fp32_arithmetic():
    for seed in range(4):
        p, x, t = case(seed)
        _, g = ows.loss_and_grad(p, x, t)
        assert np.all(np.abs(fp32_loss_grad(p, x, t) - g) <= gradient_bound(p, x, t))


def test_bound_catches_plausible_mistakes():
    p, x, t = case(7)
    _, g = ows.loss_and_grad(p, x, t)
    B = gradient_bound(p, x, t)
    H = ows.H
    mistakes = {}
    w = g.copy()
    w[ows.OFF_W2:ows.OFF_B2] = g[ows.OFF_W2:ows.OFF_B2].reshape(H, H).T.ravel()
    mistakes["W2 transposed"] = w
    w = g.copy()
    w[ows.OFF_B1:ows.OFF_W2] *= -1
    mistakes["b1 sign"] = w
    w = g.copy()
    w[ows.TRAINABLE] *= 0.5
    mistakes["factor 2 of the squared error dropped"] = w
    w = g.copy()
    w[ows.OFF_B2:ows.OFF_W3] = 0.0
    mistakes["b2 block missing"] = w
    for name, wrong in mistakes.items():
        assert np.any(np.abs(wrong - g) > B), name
