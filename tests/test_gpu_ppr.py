"""GPU parity of batched personalized PageRank (pcpm_ppr_*) against the FP64
oracle (oracle/ppr.py), through the C ABI.

Bar: after every tested number of iterations, each column of the FP32 ranks
within L1 1e-6 of the oracle's (as for PageRank: FP32 rows and sums, FP64
reductions); the per-iteration L1 changes within 1e-6 absolute."""
import numpy as np
import pytest

import graphgen
import oracle
from oracle import ppr as oppr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1709_07122_gb300 as pcpm  # noqa: E402

C = pcpm.PPR_COLS
L1_TOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pcpm.build()
    pcpm.lib()


def seeds(n, rng, max_seeds=1000):
    """Column j uniform over 1 .. max_seeds distinct random nodes (the batched
    workload's teleport vectors)."""
    ptr, idx = [0], []
    for _ in range(C):
        s = int(rng.integers(1, min(max_seeds, n) + 1))
        idx.extend(rng.choice(n, size=s, replace=False).tolist())
        ptr.append(len(idx))
    return np.array(ptr, np.uint32), np.array(idx, np.uint32)


def hub_graph():
    # node 0 has in-degree 3000 (> 1024: summed in pieces), plus an RMAT part
    n = 5000
    rp, col = graphgen.rmat(12, 8, seed=31)
    src = np.repeat(np.arange(rp.size - 1), np.diff(rp))
    src = np.concatenate([src, np.arange(1, 3001)])
    dst = np.concatenate([col.astype(np.int64), np.zeros(3000, np.int64)])
    return graphgen.csr_from_edges(n, src, dst)


GRAPHS = {
    "rmat12_q512": lambda: (graphgen.rmat(12, 16, seed=21), 512),
    "rmat12_bfs_q4096": lambda: (graphgen.rmat(12, 16, seed=22, relabel="bfs"), 4096),
    "er13_q1000": lambda: (graphgen.erdos_renyi(1 << 13, 8, seed=23), 1000),
    "random3000_dangling_q7": lambda: (graphgen.random_graph(3000, 6000, seed=24), 7),
    "hub_q2048": lambda: (hub_graph(), 2048),
}


def run_case(rp, col, q, ptr, idx, d, iters):
    with pcpm.PNG.from_host(rp, col, q) as g, pcpm.PPR(g, ptr, idx) as p:
        p.run(d, iters)
        r = p.ranks().cpu().numpy().astype(np.float64)
        return r, p.residuals(), p.info


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_matches_oracle(name):
    (rp, col), q = GRAPHS[name]()
    ptr, idx = seeds(rp.size - 1, np.random.default_rng(len(name)))
    ref = oppr.ppr(rp, col, ptr, idx, 0.85, iters=12, history=True)
    for iters in (0, 1, 2, 12):
        r, res, info = run_case(rp, col, q, ptr, idx, 0.85, iters)
        l1 = np.abs(r - ref["hist"][iters]).sum(axis=0)
        assert l1.max() <= L1_TOL, (iters, l1.max())
        if iters:
            np.testing.assert_allclose(res, ref["resid"][:iters], rtol=0, atol=1e-6)
    if name == "hub_q2048":
        assert info["split_destinations"] >= 1


def test_uniform_teleport_matches_the_pagerank_path():
    rp, col = graphgen.rmat(12, 16, seed=25)
    n = rp.size - 1
    ptr = np.arange(C + 1, dtype=np.uint32) * n
    idx = np.tile(np.arange(n, dtype=np.uint32), C)
    r, _, _ = run_case(rp, col, 512, ptr, idx, 0.85, 10)
    with pcpm.PNG.from_host(rp, col, 512) as g:
        x, _, _ = g.pagerank(0.85, max_iters=10, tol=0.0)
        x = x.cpu().numpy() if hasattr(x, "cpu") else np.asarray(x)
    assert np.abs(r - x.astype(np.float64)[:, None]).sum(axis=0).max() <= 2 * L1_TOL


def test_columns_keep_unit_mass_and_d0_is_the_teleport():
    rp, col = graphgen.rmat(12, 16, seed=26, relabel="bfs")
    n = rp.size - 1
    ptr, idx = seeds(n, np.random.default_rng(5))
    r, _, _ = run_case(rp, col, 512, ptr, idx, 0.85, 15)
    np.testing.assert_allclose(r.sum(axis=0), 1.0, atol=1e-5)
    r0, _, _ = run_case(rp, col, 512, ptr, idx, 0.0, 3)
    np.testing.assert_allclose(r0, oppr.teleport(n, ptr, idx), atol=1e-7)


def test_rerun_restarts_from_the_teleport():
    (rp, col), q = GRAPHS["rmat12_q512"]()
    ptr, idx = seeds(rp.size - 1, np.random.default_rng(6))
    ref = oppr.ppr(rp, col, ptr, idx, 0.85, iters=3)["r"]
    with pcpm.PNG.from_host(rp, col, q) as g, pcpm.PPR(g, ptr, idx) as p:
        p.run(0.85, 7)
        p.run(0.85, 3)
        r = p.ranks().cpu().numpy().astype(np.float64)
    assert np.abs(r - ref).sum(axis=0).max() <= L1_TOL


def test_bad_seeds_rejected():
    rp, col = graphgen.rmat(10, 8, seed=27)
    n = rp.size - 1
    ok_ptr = np.arange(C + 1, dtype=np.uint32)
    ok_idx = np.arange(C, dtype=np.uint32) % n
    with pcpm.PNG.from_host(rp, col, 256) as g:
        with pcpm.PPR(g, ok_ptr, ok_idx):
            pass
        bad = [
            (np.concatenate([[0, 0], ok_ptr[2:]]), ok_idx),     # an empty column
            (ok_ptr, np.where(np.arange(C) == 3, n, ok_idx)),   # a seed >= n
            (np.concatenate([[0], ok_ptr[1:] + 1]), np.concatenate([[5, 5], ok_idx[1:]])),  # repeated seed
        ]
        for ptr, idx in bad:
            with pytest.raises(pcpm.PcpmError):
                pcpm.PPR(g, np.asarray(ptr, np.uint32), np.asarray(idx, np.uint32))
        with pcpm.PPR(g, ok_ptr, ok_idx) as p:
            with pytest.raises(pcpm.PcpmError):
                p.run(1.0, 3)


def test_edgeless_graph_keeps_the_teleport():
    n = 10  # every node dangling, fewer nodes than gather lanes; seeds shared across columns
    rp = np.zeros(n + 1, np.uint32)
    ptr = np.arange(C + 1, dtype=np.uint32)
    idx = (np.arange(C) % n).astype(np.uint32)
    r, res, _ = run_case(rp, np.zeros(0, np.uint32), 4, ptr, idx, 0.85, 3)
    np.testing.assert_allclose(r, oppr.teleport(n, ptr, idx), atol=1e-7)
    assert np.abs(res).max() <= 1e-6


def test_full_size_rmat22_two_iterations():
    """The batched workload's graph (RMAT s22, q = 32768) and seed mix, two
    iterations against the FP64 oracle."""
    rp, col = graphgen.rmat(22, 16, 0.57, 0.19, 0.19, seed=1711, relabel="random")
    n = rp.size - 1
    ptr, idx = seeds(n, np.random.default_rng(22))
    t = oppr.teleport(n, ptr, idx)
    r1 = oppr.step(rp, col, t, t, 0.85)
    r2 = oppr.step(rp, col, r1, t, 0.85)
    r, res, info = run_case(rp, col, 32768, ptr, idx, 0.85, 2)
    l1 = np.abs(r - r2).sum(axis=0)
    assert l1.max() <= L1_TOL, l1.max()
    np.testing.assert_allclose(res[1], np.abs(r2 - r1).sum(axis=0), rtol=0, atol=L1_TOL)
    assert info["split_destinations"] > 0  # RMAT hubs are summed in pieces
