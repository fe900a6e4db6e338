"""Pins for the oracle's Partition-Node Graph (Sec. 3.1-3.3) and for its
Algorithm 3 + Algorithm 4 simulation.

The brute-force reference below derives every PNG array from a different
definition than the oracle's run-scanning loops: the canonical content of bin
p' is the set of edges (u, v) with v in partition p', sorted by (u, v); an
update is one distinct source u in that list; the first destination of each u
carries the MSB. Offsets follow from counting, per bin, the entries whose
source lies in a lower partition.
"""
import os

import numpy as np
import pytest

import graphgen
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def brute_png(rp, col, q):
    n = rp.size - 1
    k = (n + q - 1) // q
    edges = sorted((u, int(col[e])) for u in range(n) for e in range(rp[u], rp[u + 1]))
    cnt_u = np.zeros((k, k), np.int64)
    cnt_e = np.zeros((k, k), np.int64)
    pairs = {(u, v // q) for u, v in edges}
    for u, pd in pairs:
        cnt_u[u // q, pd] += 1
    for u, v in edges:
        cnt_e[u // q, v // q] += 1
    src_idx, dest_ids, bin_u, bin_e = [], [], [0], [0]
    off_u = np.zeros((k, k), np.int64)
    off_e = np.zeros((k, k), np.int64)
    for pd in range(k):
        into = [(u, v) for u, v in edges if v // q == pd]  # sorted by (u, v)
        for p in range(k):
            off_u[p, pd] = len({u for u, _ in into if u // q < p})
            off_e[p, pd] = sum(1 for u, _ in into if u // q < p)
        prev = None
        for u, v in into:
            if u != prev:
                src_idx.append(u)
                dest_ids.append(v | 0x80000000)
                prev = u
            else:
                dest_ids.append(v)
        bin_u.append(len(src_idx))
        bin_e.append(len(dest_ids))
    return dict(k=k, cnt_u=cnt_u, cnt_e=cnt_e, off_u=off_u, off_e=off_e, bin_u=np.array(bin_u),
                bin_e=np.array(bin_e), src_idx=np.array(src_idx, np.int64), dest_ids=np.array(dest_ids, np.int64))


def assert_png_equal(g, b):
    assert g["k"] == b["k"]
    for key in ("cnt_u", "cnt_e", "off_u", "off_e", "bin_u", "bin_e", "src_idx", "dest_ids"):
        np.testing.assert_array_equal(np.asarray(g[key], np.int64), b[key], err_msg=key)


CASES = [(n, q, seed) for seed in range(4) for n, q in [(1, 1), (2, 1), (9, 3), (10, 3), (23, 4), (40, 7), (40, 40),
                                                         (40, 64), (64, 5), (50, 1)]]


@pytest.mark.parametrize("n,q,seed", CASES)
def test_png_brute_force(n, q, seed):
    rp, col = graphgen.random_graph(n, m_draws=3 * n + seed, seed=1000 + seed + n * 7 + q)
    assert_png_equal(oracle.png(rp, col, q), brute_png(rp, col, q))


def test_png_brute_force_with_hubs_and_isolated():
    # Node 0 points at everything, node 1 at nothing, node 2 receives from all.
    n, q = 30, 4
    src = list(np.zeros(n - 1, int)) + [u for u in range(3, n)]
    dst = list(range(1, n)) + [2] * (n - 3)
    rp, col = graphgen.csr_from_edges(n, np.array(src), np.array(dst))
    assert_png_equal(oracle.png(rp, col, q), brute_png(rp, col, q))


def read_example():
    vals = {}
    with open(os.path.join(GOLDEN, "offsets_example.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                key, *rest = line.split()
                vals[key] = rest
    n, q = int(vals["n"][0]), int(vals["q"][0])
    edges = [tuple(map(int, e.split(">"))) for e in vals["edges"]]
    expect = [int(x) for x in vals["offsets_p2"]]
    return n, q, edges, expect


def test_paper_offsets_example():
    # Sec. 3.1: P_2's offsets into update_bins[0..2] are 0, 1, 1.
    n, q, edges, expect = read_example()
    rp, col = graphgen.csr_from_edges(n, np.array([e[0] for e in edges]), np.array([e[1] for e in edges]))
    g = oracle.png(rp, col, q)
    assert list(g["off_u"][2]) == expect
    # and the facts the paper states about the lower partitions
    assert g["cnt_u"][0, 0] == 0 and g["cnt_u"][1, 0] == 0
    assert g["cnt_u"][1, 1] == 1 and g["cnt_u"][0, 2] == 1
    # node 0 has two neighbours in P_2 but sends one update (Sec. 3.2)
    assert g["cnt_e"][0, 2] == 2


@pytest.mark.parametrize("scale,q", [(10, 64), (12, 1000), (12, 4096), (14, 16384)])
def test_png_structural_invariants(scale, q):
    rp, col = graphgen.rmat(scale, 16, seed=scale)
    g = oracle.png(rp, col, q)
    n, m = rp.size - 1, int(rp[-1])
    k = g["k"]
    assert k == -(-n // q)
    # |E'| = number of distinct (u, partition of v) pairs; sum of E counts = m
    u = np.repeat(np.arange(n, dtype=np.int64), np.diff(rp.astype(np.int64)))
    pairs = np.unique(u * k + col.astype(np.int64) // q)
    assert g["ne"] == pairs.size
    assert int(g["cnt_e"].sum()) == m and g["bin_e"][-1] == m
    flags = (g["dest_ids"] >> 31).astype(np.int64)
    assert flags.sum() == g["ne"]
    # every non-empty bin starts with a flagged ID; bins hold their own partition only
    for pd in range(k):
        lo, hi = g["bin_e"][pd], g["bin_e"][pd + 1]
        if hi > lo:
            assert g["dest_ids"][lo] >> 31 == 1
            ids = g["dest_ids"][lo:hi] & 0x7FFFFFFF
            assert ((ids // q) == pd).all()
    # compression ratio r = m/|E'| lies in [1, m/n'] (Sec. 4 states [1, m/n] for
    # graphs without dangling nodes; each of the n' nodes with out-edges sends at
    # least one update, so the upper end is m/n')
    r = m / g["ne"]
    n_out = int((np.diff(rp.astype(np.int64)) > 0).sum())
    assert 1.0 <= r <= m / n_out + 1e-12
    # offsets are monotone and disjoint per bin
    assert (np.diff(g["off_u"].astype(np.int64), axis=0) == g["cnt_u"][:-1].astype(np.int64)).all()
    assert (np.diff(g["off_e"].astype(np.int64), axis=0) == g["cnt_e"][:-1].astype(np.int64)).all()


def test_compression_grows_with_partition_size():
    # Sec. 5.3.2: larger partitions compress more (r grows with q).
    rp, col = graphgen.rmat(14, 16, seed=5)
    rs = []
    for q in (16, 256, 4096, 16384):
        g = oracle.png(rp, col, q)
        rs.append(g["m"] / g["ne"])
    assert all(b >= a for a, b in zip(rs, rs[1:]))


def test_bfs_labels_raise_compression():
    # Locality-improving relabeling raises r (Table compRatio's trend).
    r = {}
    for lab in ("random", "bfs"):
        rp, col = graphgen.rmat(14, 16, seed=6, relabel=lab)
        g = oracle.png(rp, col, 1024)
        r[lab] = g["m"] / g["ne"]
    assert r["bfs"] > r["random"]


@pytest.mark.parametrize("n,q,seed", [(9, 3, 0), (40, 7, 1), (64, 5, 2), (300, 17, 3), (300, 300, 4), (1, 1, 5)])
def test_scatter_gather_equals_dense_product(n, q, seed):
    # Algorithm 3 + Algorithm 4 over the bins equals A^T spr (dense numpy product).
    rp, col = graphgen.random_graph(n, m_draws=4 * n, seed=seed)
    spr = graphgen.uniform(n, seed=50 + seed)
    A = np.zeros((n, n))
    for u in range(n):
        A[u, col[rp[u]:rp[u + 1]]] = 1.0
    y = oracle.scatter_gather(oracle.png(rp, col, q), spr)
    np.testing.assert_allclose(y, A.T @ spr, rtol=1e-14, atol=1e-15)


def test_scatter_gather_reproduces_pagerank_step():
    # One Eq. 1 step assembled from the PNG gather equals the pull oracle's step.
    rp, col = graphgen.rmat(12, 16, seed=11)
    n = rp.size - 1
    x0 = graphgen.random_rank_vector(n, seed=12)
    outdeg = np.diff(rp.astype(np.int64))
    spr = np.where(outdeg > 0, x0 / np.maximum(outdeg, 1), 0.0)
    dang = x0[outdeg == 0].sum()
    y = oracle.scatter_gather(oracle.png(rp, col, 512), spr)
    step = (1 - 0.85) / n + 0.85 * (y + dang / n)
    ref = oracle.pagerank(rp, col, 0.85, iters=1, x0=x0)["x"]
    np.testing.assert_allclose(step, ref, rtol=1e-13)
