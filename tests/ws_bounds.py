"""Per-entry rounding bounds for the learned warm start's FP32 kernels.

The bound follows each value of the network's forward and backward pass
through FP32 arithmetic as a magnitude and an absolute error bound (running
error analysis, u = 2^-24 per rounding): a k-term dot product or sum in FP32
adds at most (k + 1) u times the sum of its terms' magnitudes, and the error
of each input is carried through the products. A ReLU whose input lies
within its own error bound of zero may switch either way; the whole
contribution of such units is added to the bound. The batch sum of a
gradient entry (per-tile FP32 sums, then FP32 atomics over the tiles) adds
(tile + tiles) u times the sum of the per-node magnitudes.

Used only by the tests: it turns "the GPU gradient matches the FP64 oracle"
into a check of every entry against its own bound, so a wrong small block
cannot hide under large entries.
"""
import numpy as np

from oracle import warmstart as ows

U = 2.0 ** -24


def gradient_bound(params, x, target, tile: int = 256):
    p = np.asarray(params, np.float64)
    q = ows.unpack(p)
    x = np.asarray(x, np.float64)
    t = np.asarray(target, np.float64)
    n = x.shape[0]
    y, c = ows.forward(p, x, cache=True)
    aW1, aW2, aw3 = np.abs(q["W1"]), np.abs(q["W2"]), np.abs(q["w3"])
    # standardisation: (x - mu) * inv_sigma, two roundings
    xa = np.abs(c["xh"])
    ex = 2 * U * xa
    # layer 1: 5-term FMA chain plus the bias
    s1 = xa @ aW1.T + np.abs(q["b1"])
    ez1 = (6 + 1) * U * s1 + ex @ aW1.T
    amb1 = np.abs(c["z1"]) <= ez1
    on1 = (c["z1"] > 0) | amb1
    h1a = np.abs(c["h1"]) + ez1 * amb1
    eh1 = ez1 * on1
    # layer 2: 64-term FMA chain plus the bias
    s2 = h1a @ aW2.T + np.abs(q["b2"])
    ez2 = 66 * U * s2 + eh1 @ aW2.T
    amb2 = np.abs(c["z2"]) <= ez2
    on2 = (c["z2"] > 0) | amb2
    h2a = np.abs(c["h2"]) + ez2 * amb2
    eh2 = ez2 * on2
    # output and residual
    ey = 66 * U * (h2a @ aw3 + abs(q["b3"])) + eh2 @ aw3
    r = y - t
    dya = 2 * (np.abs(r) + ey) / n
    edy = 2 * (ey + 2 * U * (np.abs(r) + np.abs(t))) / n + 3 * U * dya
    # backward: dz2 = dy w3 on units that may be on
    dz2a = np.outer(dya, aw3) * on2
    edz2 = (np.outer(edy, aw3) + U * dz2a) * on2 + np.outer(dya, aw3) * amb2
    dz1a = (dz2a @ aW2) * on1
    edz1 = (66 * U * (dz2a @ aW2) + edz2 @ aW2) * on1 + (dz2a @ aW2) * amb1
    k_sum = (tile + -(-n // tile)) * U
    B = np.zeros(ows.P)
    # each block: propagated per-node errors plus the batch sum's rounding
    B[ows.OFF_W3:ows.OFF_B3] = edy @ h2a + dya @ eh2 + k_sum * (dya @ h2a)
    B[ows.OFF_B3] = edy.sum() + k_sum * dya.sum()
    B[ows.OFF_W2:ows.OFF_B2] = (edz2.T @ h1a + dz2a.T @ eh1 + k_sum * (dz2a.T @ h1a)).ravel()
    B[ows.OFF_B2:ows.OFF_W3] = edz2.sum(0) + k_sum * dz2a.sum(0)
    B[ows.OFF_W1:ows.OFF_B1] = (edz1.T @ xa + dz1a.T @ ex + k_sum * (dz1a.T @ xa)).ravel()
    B[ows.OFF_B1:ows.OFF_W2] = edz1.sum(0) + k_sum * dz1a.sum(0)
    return B
