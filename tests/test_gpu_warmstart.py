"""Learned warm start on the GPU against the FP64 reference (oracle/warmstart.py).

Features: the three integer in-edge sums bit-exact against numpy's integer
sums, their FP32 logarithms within a few units in the last place, and the
one-iteration feature within the FP32 path's 1e-6 bar. Inference (tensor
cores, BF16 weights and activations) against the FP64 network on the same
rounded weights within a running-error bound. The loss gradient against the FP64 gradient
entry by entry, each within its own rounding bound (tests/ws_bounds.py);
Adam per entry; the initial ranks against the FP64 softmax. End to end, a
network trained on small RMAT graphs starts an unseen graph's solve, which
needs strictly fewer iterations to the same residual and reaches the same
ranks as the uniform start.
"""
import numpy as np
import pytest

import graphgen
import oracle
from oracle import warmstart as ows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1709_07122_gb300 as pcpm  # noqa: E402
from paper_1709_07122_gb300 import warmstart as ws  # noqa: E402

FP32 = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pcpm.build()
    pcpm.lib()


def gpu_features(rp, col, q):
    drp, dcol = pcpm.to_device_csr(rp, col)
    with pcpm.PNG(drp, dcol, q) as g:
        sums = pcpm.ws_degree_sums(g, drp).cpu().numpy().view(np.uint32)
        return pcpm.ws_features(g, drp, dcol).cpu().numpy(), sums


def exact_sums(rp, col):
    rp = rp.astype(np.int64)
    c = col.astype(np.int64)
    n = rp.size - 1
    outdeg = np.diff(rp)
    src = np.repeat(np.arange(n), outdeg)
    indeg = np.bincount(c, minlength=n).astype(np.int64)
    s_in = np.zeros(n, np.int64)
    s_out = np.zeros(n, np.int64)
    np.add.at(s_in, c, indeg[src])
    np.add.at(s_out, c, outdeg[src])
    return np.stack([indeg, s_in, s_out])


@pytest.mark.parametrize("name,gen,q", [
    ("rmat12", lambda: graphgen.rmat(12, 16, seed=61), 512),
    ("random2000", lambda: graphgen.random_graph(2000, 9000, seed=62), 300),
    ("rmat10_bfs", lambda: graphgen.rmat(10, 8, seed=63, relabel="bfs"), 100),
    ("rmat14_q32768", lambda: graphgen.rmat(14, 16, seed=64), 32768),
    ("ragged_q7", lambda: graphgen.random_graph(1000, 4000, seed=65), 7),
])
def test_features_match_reference(name, gen, q):
    rp, col = gen()
    got, sums = gpu_features(rp, col, q)
    want = ows.features(rp, col)
    # the integer sums are exact
    np.testing.assert_array_equal(sums.astype(np.int64), exact_sums(rp, col))
    # their logarithms: log1pf of the count (exact in float below 2^24) within
    # a few FP32 units in the last place of the FP64 value
    got = got.astype(np.float64)
    ulp = np.spacing(np.abs(want[:, :4]).astype(np.float32)).astype(np.float64)
    assert np.all(np.abs(got[:, :4] - want[:, :4]) <= 4 * ulp)
    # log(n * PR_1): PR_1 from the FP32 path (L1 <= 1e-6 against FP64), so
    # |d log| <= |d PR| / PR per node; the sum of |n PR1 - n PR1*| is what the
    # 1e-6 bar controls
    n = rp.size - 1
    x_got, x_want = np.exp(got[:, 4]) / n, np.exp(want[:, 4]) / n
    assert np.abs(x_got - x_want).sum() <= 1e-6 + 64 * FP32 * x_want.sum()


@pytest.mark.parametrize("opts", [{}, {"update_dtype": "f16"}, {"gather_windows": 2},
                                  {"canonical_gather": 1, "gather_windows": 2}])
def test_degree_sums_exact_on_every_build_path(opts):
    # window layout (in-degrees kept by the build, sums scattered into FP32
    # bins), 16-bit bins (sources' degrees read at random), chunk layouts (an
    # in-degree pass)
    rp, col = graphgen.rmat(13, 16, seed=66)
    drp, dcol = pcpm.to_device_csr(rp, col)
    with pcpm.PNG(drp, dcol, 1000, **opts) as g:
        sums = pcpm.ws_degree_sums(g, drp).cpu().numpy().view(np.uint32)
        np.testing.assert_array_equal(sums.astype(np.int64), exact_sums(rp, col))
        # the handle solves normally afterwards (FP32 bins: the 1e-6 bar)
        if "update_dtype" not in opts:
            pr, _, _ = g.pagerank(0.85, max_iters=5)
            ref = oracle.pagerank(rp, col, 0.85, iters=5)["x"]
            assert float(np.abs(pr.cpu().numpy().astype(np.float64) - ref).sum()) <= 1e-6


def test_degree_sums_exact_past_fp32_integers():
    # 4099 sources, each pointing to the same 4099 targets: every target's sum
    # of in-neighbours' out-degrees is 4099^2 = 16,801,801, odd and above
    # 2^24, which FP32 cannot hold; the exact passes must take over
    k = 4099
    src = np.repeat(np.arange(k), k)
    dst = k + np.tile(np.arange(k), k)
    rp, col = graphgen.csr_from_edges(2 * k, src, dst)
    drp, dcol = pcpm.to_device_csr(rp, col)
    with pcpm.PNG(drp, dcol, 1024) as g:
        sums = pcpm.ws_degree_sums(g, drp).cpu().numpy().view(np.uint32)
    want = exact_sums(rp, col)
    assert want[2].max() == k * k
    np.testing.assert_array_equal(sums.astype(np.int64), want)


def rand_params(rng):
    p = rng.standard_normal(ows.P).astype(np.float32) * 0.2
    p[:5] = rng.standard_normal(5).astype(np.float32)
    p[5:10] = (0.5 + rng.random(5)).astype(np.float32)
    return p


def bf16_weights(p):
    q = p.astype(np.float64).copy()
    q[ows.TRAINABLE] = oracle.load_updates(oracle.store_updates(p[ows.TRAINABLE], "bf16"), "bf16")
    return q


def test_predict_matches_reference_with_bf16_weights():
    rng = np.random.default_rng(64)
    p = rand_params(rng)
    for rows in (3000, 16, 17, 1):  # whole and ragged 16-node tiles
        x = (rng.standard_normal((rows, 5)) * 2 + 3).astype(np.float32)
        got = pcpm.ws_predict(torch.from_numpy(p).cuda(), torch.from_numpy(x).cuda()).cpu().numpy()
        want = ows.forward(bf16_weights(p), x.astype(np.float64))
        # Running error: the standardised inputs and h1 are rounded to BF16
        # for the tensor-core products (relative 2^-9 = 2^15 u each), the
        # products are exact and summed in FP32 (<= 66 u of the sum of their
        # sizes per layer); bias, ReLU (which does not increase an error) and
        # the FP32 dot product with w3 (<= 66 u). Each rounding's effect on the
        # output is bounded by the fully absolute-valued network's output, so
        # the output is within about (2 * 2^15 + 2 * 66 + 66) u of it.
        q = ows.unpack(bf16_weights(p))
        xa = np.abs((x.astype(np.float64) - q["mu"]) * q["inv_sigma"])
        s1 = xa @ np.abs(q["W1"]).T + np.abs(q["b1"])
        s2 = s1 @ np.abs(q["W2"]).T + np.abs(q["b2"])
        scale = s2 @ np.abs(q["w3"]) + abs(q["b3"])
        assert np.all(np.abs(got - want) <= (2.0 ** 16 + 512) * FP32 * scale), rows


def test_loss_and_gradient_match_reference():
    from ws_bounds import gradient_bound
    rng = np.random.default_rng(65)
    p = rand_params(rng)
    for rows in (5000, 300, 1):
        x = (rng.standard_normal((rows, 5)) * 2).astype(np.float32)
        t = rng.standard_normal(rows).astype(np.float32)
        grad = torch.zeros(ows.P, dtype=torch.float32, device="cuda")
        loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        pcpm.ws_loss_grad(torch.from_numpy(p).cuda(), torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda(), grad,
                          loss)
        L, g = ows.loss_and_grad(p.astype(np.float64), x.astype(np.float64), t.astype(np.float64))
        assert abs(loss.item() - L) <= 1e-5 * L
        gg = grad.cpu().numpy().astype(np.float64)
        assert np.all(gg[:ows.OFF_W1] == 0.0)
        # every entry within its own running-error bound
        bound = gradient_bound(p, x, t)
        bad = np.nonzero(np.abs(gg - g) > bound)[0]
        assert bad.size == 0, (rows, bad[:10], (gg - g)[bad[:10]], bound[bad[:10]])


def test_adam_step_matches_reference():
    rng = np.random.default_rng(66)
    p = rand_params(rng)
    g = rng.standard_normal(ows.P).astype(np.float32)
    m = (rng.standard_normal(ows.P) * 0.1).astype(np.float32)
    v = (rng.random(ows.P) * 0.01).astype(np.float32)
    tp, tm, tv = (torch.from_numpy(a.copy()).cuda() for a in (p, m, v))
    lr = 1e-3
    pcpm.ws_adam(tp, torch.from_numpy(g).cuda(), tm, tv, 7, lr)
    # the reference with the kernel's FP32 constants (0.9f, 0.999f, 1e-8f)
    b1, b2, eps = (float(np.float32(c)) for c in (0.9, 0.999, 1e-8))
    wp, wm, wv = ows.adam(p, g, m, v, 7, lr, b1, b2, eps)
    g64, m64, v64 = (a.astype(np.float64) for a in (g, m, v))
    # each moment is two FP32 products and a sum: within 4u of its terms
    tol_m = 4 * FP32 * (b1 * np.abs(m64) + (1 - b1) * np.abs(g64))
    tol_v = 4 * FP32 * (b2 * v64 + (1 - b2) * g64 * g64)
    s = ows.TRAINABLE
    assert np.all(np.abs(tm.cpu().numpy()[s] - wm[s]) <= tol_m[s])
    assert np.all(np.abs(tv.cpu().numpy()[s] - wv[s]) <= tol_v[s])
    # the step lr * mhat / (sqrt(vhat) + eps) to within a few FP32 roundings
    # of its size, plus the moments' own error carried through it
    step = np.abs(wp[s] - p[s].astype(np.float64))
    carried = lr * (tol_m[s] / (1 - b1 ** 7)) / (np.sqrt(wv[s] / (1 - b2 ** 7)) + eps)
    assert np.all(np.abs(tp.cpu().numpy()[s] - wp[s]) <= 16 * FP32 * (np.abs(wp[s]) + step) + 2 * carried)


def test_initial_ranks_are_the_softmax():
    rng = np.random.default_rng(67)
    pred = (rng.standard_normal(100000) * 3).astype(np.float32)
    x = pcpm.ws_init_ranks(torch.from_numpy(pred).cuda()).cpu().numpy().astype(np.float64)
    want = ows.warm_start(pred.astype(np.float64))
    assert abs(x.sum() - 1.0) <= 1e-6
    # expf within 2 ulp (4 u), the FP32 reciprocal of the FP64 sum and the
    # product one rounding each: 6 u
    np.testing.assert_allclose(x, want, rtol=8 * FP32, atol=0)


def test_targets_are_log_n_pr():
    rng = np.random.default_rng(68)
    pr = (rng.random(50000) + 0.01).astype(np.float32)
    pr /= pr.sum()
    got = pcpm.ws_targets(torch.from_numpy(pr).cuda()).cpu().numpy()
    np.testing.assert_allclose(got, np.log(pr.size * pr.astype(np.float64)), rtol=0, atol=4 * FP32 * 10)


def test_trained_network_starts_an_unseen_graph_to_the_same_fixed_point():
    train_graphs = [graphgen.rmat(s, 16, *ws.rmat_params(a), seed=70 + i)
                    for i, (s, a) in enumerate([(12, 0.5), (13, 0.57), (12, 0.62), (13, 0.45)])]
    samples = [ws.Sample(rp, col, 1024) for rp, col in train_graphs]
    params = ws.init_params(samples, seed=3)
    log = ws.train(params, samples, steps=300, batch=4096, lr=3e-3, log_every=50)
    assert log[-1][1] < log[0][1]  # the loss goes down
    rp, col = graphgen.rmat(14, 16, 0.57, 0.19, 0.19, seed=99)
    res = ws.evaluate(params, rp, col, 2048, tol=1e-7)
    for name in ("uniform", "warm"):
        assert res[name]["residual"] < 1e-7, name
    # both stop within d/(1-d) * 1e-7 of the fixed point
    diff = float((res["warm"]["ranks"] - res["uniform"]["ranks"]).abs().sum())
    assert diff <= 2 * 0.85 / 0.15 * 1e-7 + 1e-6
    # what the trained network gains: strictly fewer iterations to 1e-7
    assert res["warm"]["iters"] < res["uniform"]["iters"], (res["warm"]["iters"], res["uniform"]["iters"])
