"""GPU parity at full size: the benchmark's own workload and launch setup.

RMAT scale 24 (16,777,216 nodes; a, b, c = 0.57, 0.19, 0.19; edge factor 16;
random labels; duplicates and self-loops removed, 263M edges), q = 32768
(k = 512), automatic build options, both iteration forms. The whole PNG is
compared bit for bit with the oracle's and every rank of the first iterations
within L1 1e-6 of the FP64 oracle, with the L1 change per iteration matched
too. About a minute on the host for the oracle and the generator.
"""
import numpy as np
import pytest

import graphgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1709_07122_gb300 as pcpm  # noqa: E402

SCALE, Q, D, ITERS = 24, 32768, 0.85, 3
L1_TOL = 1e-6


@pytest.fixture(scope="module")
def graph():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pcpm.build()
    pcpm.lib()
    return graphgen.rmat(SCALE, 16, 0.57, 0.19, 0.19, seed=1710, relabel="random")


@pytest.fixture(scope="module")
def reference(graph):
    rp, col = graph
    return oracle.pagerank(rp, col, D, iters=ITERS, history=True)


def l1(a, b):
    return float(np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64)).sum())


def test_fullsize_png_bit_exact(graph):
    rp, col = graph
    ref = oracle.png(rp, col, Q)
    with pcpm.PNG.from_host(rp, col, Q) as g:
        info = g.info
        assert (info["num_partitions"], info["num_edges"], info["num_updates"]) == (ref["k"], ref["m"], ref["ne"])
        out = g.export()
    for key in ("cnt_u", "cnt_e", "off_u", "off_e", "bin_u", "bin_e", "src_idx", "dest_ids"):
        np.testing.assert_array_equal(out[key], np.asarray(ref[key], dtype=np.uint32), err_msg=key)


@pytest.mark.parametrize("mode", ["two_phase", "fused"])
def test_fullsize_ranks_follow_oracle(graph, reference, mode):
    rp, col = graph
    hist, resid = reference["hist"], reference["resid"]
    with pcpm.PNG.from_host(rp, col, Q) as g:
        g.reset()
        for i in range(1, ITERS + 1):
            _, res = g.iterate(D, 1, mode=mode)
            x = g.ranks().cpu().numpy()
            assert l1(x, hist[i]) <= L1_TOL, (mode, i, l1(x, hist[i]))
            assert abs(res - resid[i - 1]) <= 2 * L1_TOL, (mode, i, res, resid[i - 1])
            assert abs(float(np.sum(x, dtype=np.float64)) - 1.0) <= L1_TOL
