"""GPU parity at full size: the benchmark's own workload and launch setup.

The scale-24 graphs of the plain-PCPM configuration: RMAT scale 24 (16,777,216
nodes; a, b, c = 0.57, 0.19, 0.19; edge factor 16; duplicates and self-loops
removed, 263M edges) under random labels and under the BFS relabel, and an
Erdos-Renyi graph of 2^24 nodes with mean out-degree 16; q = 32768 (k = 512),
automatic build options. The whole PNG of the benchmark graph is compared bit
for bit with the oracle's; every rank of all 20 iterations of each graph,
both iteration forms, within L1 1e-6 of the FP64 oracle (iterated from the
same uniform start on all host threads), with the L1 change per iteration
matched too. A few minutes on the host for the generators and the oracle.
"""
import numpy as np
import pytest

import graphgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1709_07122_gb300 as pcpm  # noqa: E402

Q, D, ITERS = 32768, 0.85, 20
L1_TOL = 1e-6

GRAPHS = {
    "rmat24_random": lambda: graphgen.rmat(24, 16, 0.57, 0.19, 0.19, seed=1710, relabel="random"),
    "rmat24_bfs": lambda: graphgen.rmat(24, 16, 0.57, 0.19, 0.19, seed=1710, relabel="bfs"),
    "er24_random": lambda: graphgen.erdos_renyi(1 << 24, 16, seed=1710, relabel="random"),
}


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pcpm.build()
    pcpm.lib()


_cache = {}


def graph(name):
    if name not in _cache:
        _cache.clear()  # one scale-24 graph in host memory at a time
        _cache[name] = GRAPHS[name]()
    return _cache[name]


def l1(a, b):
    return float(np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64)).sum())


def test_fullsize_png_bit_exact():
    rp, col = graph("rmat24_random")
    ref = oracle.png(rp, col, Q)
    with pcpm.PNG.from_host(rp, col, Q) as g:
        info = g.info
        assert (info["num_partitions"], info["num_edges"], info["num_updates"]) == (ref["k"], ref["m"], ref["ne"])
        out = g.export()
    for key in ("cnt_u", "cnt_e", "off_u", "off_e", "bin_u", "bin_e", "src_idx", "dest_ids"):
        np.testing.assert_array_equal(out[key], np.asarray(ref[key], dtype=np.uint32), err_msg=key)


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_fullsize_ranks_follow_oracle_for_20_iterations(name):
    rp, col = graph(name)
    n = rp.size - 1
    pull = oracle.Pull(rp, col)
    threads = oracle.host_threads()
    with pcpm.PNG.from_host(rp, col, Q) as g:
        for mode in ("two_phase", "fused"):
            x = np.full(n, 1.0 / n)
            y = np.empty(n)
            g.reset()
            for i in range(1, ITERS + 1):
                want_res = pull.step_all(x, y, D, "uniform", threads)
                x, y = y, x
                _, res = g.iterate(D, 1, mode=mode)
                got = g.ranks().cpu().numpy()
                assert l1(got, x) <= L1_TOL, (name, mode, i, l1(got, x))
                assert abs(res - want_res) <= 2 * L1_TOL, (name, mode, i, res, want_res)
                assert abs(float(np.sum(got, dtype=np.float64)) - 1.0) <= L1_TOL
