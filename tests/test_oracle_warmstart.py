"""Pins of the FP64 warm-start reference (oracle/warmstart.py)."""
import math

import numpy as np

import graphgen
from oracle import warmstart as ws


def csr(n, edges):
    src = np.array([e[0] for e in edges])
    dst = np.array([e[1] for e in edges])
    return graphgen.csr_from_edges(n, src, dst)


def test_features_directed_cycle():
    # every node: in = out = 1, 2-hop sums 1, PR_1 = 1/n exactly
    n = 7
    rp, col = csr(n, [(i, (i + 1) % n) for i in range(n)])
    f = ws.features(rp, col)
    np.testing.assert_allclose(f[:, :4], math.log(2.0), rtol=0, atol=1e-15)
    np.testing.assert_allclose(f[:, 4], 0.0, atol=1e-12)


def test_features_bidirectional_star():
    # centre 0 <-> leaves 1..n-1: centre in = out = n-1, leaf in = out = 1;
    # centre's in-neighbours (leaves) have in = out = 1, so both sums are n-1;
    # a leaf's only in-neighbour is the centre: sums n-1.
    # PR_1 from 1/n: centre (1-d)/n + d(n-1)/n; leaf (1-d)/n + d/(n(n-1)).
    n, d = 9, 0.85
    rp, col = csr(n, [(0, i) for i in range(1, n)] + [(i, 0) for i in range(1, n)])
    f = ws.features(rp, col, d)
    L = math.log1p(n - 1)
    np.testing.assert_allclose(f[0, :4], [L, L, L, L], rtol=1e-15)
    np.testing.assert_allclose(f[1:, :4], np.tile([math.log(2), math.log(2), L, L], (n - 1, 1)), rtol=1e-15)
    assert abs(f[0, 4] - math.log((1 - d) + d * (n - 1))) < 1e-12
    assert abs(f[1, 4] - math.log((1 - d) + d / (n - 1))) < 1e-12


def test_two_hop_sums_by_explicit_loops():
    rp, col = graphgen.random_graph(60, 400, seed=5)
    n = rp.size - 1
    indeg = [0] * n
    for v in col:
        indeg[int(v)] += 1
    s_in, s_out = [0] * n, [0] * n
    for u in range(n):
        for e in range(int(rp[u]), int(rp[u + 1])):
            v = int(col[e])
            s_in[v] += indeg[u]
            s_out[v] += int(rp[u + 1] - rp[u])
    f = ws.features(rp, col)
    np.testing.assert_allclose(f[:, 2], np.log1p(s_in), rtol=1e-15)
    np.testing.assert_allclose(f[:, 3], np.log1p(s_out), rtol=1e-15)


def random_params(rng, scale=0.3):
    p = rng.standard_normal(ws.P) * scale
    p[ws.OFF_MU:ws.OFF_MU + ws.F] = rng.standard_normal(ws.F)
    p[ws.OFF_IS:ws.OFF_IS + ws.F] = 0.5 + rng.random(ws.F)
    return p


def test_forward_closed_form_with_zero_weights():
    rng = np.random.default_rng(1)
    p = random_params(rng)
    p[ws.OFF_W1:ws.OFF_B1] = 0.0
    p[ws.OFF_W2:ws.OFF_B2] = 0.0
    x = rng.standard_normal((11, ws.F))
    q = ws.unpack(p)
    want = np.maximum(q["b2"], 0.0) @ q["w3"] + q["b3"]
    np.testing.assert_allclose(ws.forward(p, x), want, rtol=1e-14)


def test_forward_by_explicit_loops():
    # The parameter layout read entry by entry: W1[j][f] multiplies input f
    # into hidden unit j (row j of the flat W1 block), W2[j][i] multiplies h1[i]
    # into h2[j]. A transposed block or a dropped bias changes the output.
    rng = np.random.default_rng(4)
    p = random_params(rng, scale=0.5)
    x = rng.standard_normal((6, ws.F)) * 2
    F, H = ws.F, ws.H
    for r in range(x.shape[0]):
        xh = [(x[r][f] - p[ws.OFF_MU + f]) * p[ws.OFF_IS + f] for f in range(F)]
        h1 = []
        for j in range(H):
            z = p[ws.OFF_B1 + j]
            for f in range(F):
                z += p[ws.OFF_W1 + j * F + f] * xh[f]
            h1.append(max(z, 0.0))
        h2 = []
        for j in range(H):
            z = p[ws.OFF_B2 + j]
            for i in range(H):
                z += p[ws.OFF_W2 + j * H + i] * h1[i]
            h2.append(max(z, 0.0))
        y = p[ws.OFF_B3] + sum(p[ws.OFF_W3 + j] * h2[j] for j in range(H))
        assert abs(ws.forward(p, x[r:r + 1])[0] - y) <= 1e-12 * max(1.0, abs(y))
    # the hidden layers are not symmetric in their indices: a transposed W2
    # gives another network
    q = p.copy()
    q[ws.OFF_W2:ws.OFF_B2] = p[ws.OFF_W2:ws.OFF_B2].reshape(H, H).T.ravel()
    assert np.abs(ws.forward(q, x) - ws.forward(p, x)).max() > 1e-3


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(2)
    p = random_params(rng)
    x = rng.standard_normal((23, ws.F)) * 2
    t = rng.standard_normal(23)
    _, g = ws.loss_and_grad(p, x, t)
    assert np.all(g[:ws.OFF_W1] == 0.0)
    idx = np.concatenate([rng.choice(np.arange(ws.OFF_W1, ws.P), 60, replace=False), [ws.P - 1]])
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        num = (ws.loss_and_grad(pp, x, t)[0] - ws.loss_and_grad(pm, x, t)[0]) / (2 * h)
        assert abs(num - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, num, g[i])


def test_adam_first_step_closed_form():
    # step 1: mhat = g and vhat = g^2, so every trainable entry moves by
    # -lr * g / (|g| + eps)
    rng = np.random.default_rng(3)
    p = random_params(rng)
    g = rng.standard_normal(ws.P)
    lr, eps = 1e-2, 1e-8
    p1, m1, v1 = ws.adam(p, g, np.zeros(ws.P), np.zeros(ws.P), 1, lr, eps=eps)
    s = ws.TRAINABLE
    np.testing.assert_allclose(p1[s], p[s] - lr * g[s] / (np.abs(g[s]) + eps), rtol=1e-12)
    np.testing.assert_array_equal(p1[:ws.OFF_W1], p[:ws.OFF_W1])
    np.testing.assert_allclose(m1[s], 0.1 * g[s], rtol=1e-15)
    np.testing.assert_allclose(v1[s], 0.001 * g[s] ** 2, rtol=1e-14)  # 1 - 0.999 rounds in FP64


def test_warm_start_is_a_distribution_proportional_to_exp():
    pred = np.array([0.0, 1.0, -2.0, 3.5])
    x = ws.warm_start(pred)
    assert abs(x.sum() - 1.0) < 1e-15
    np.testing.assert_allclose(x / x[0], np.exp(pred), rtol=1e-14)
