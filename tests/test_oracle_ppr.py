"""Pins of the FP64 personalized-PageRank oracle (oracle/ppr.py) against facts
that do not come from it: the C PageRank oracle (a uniform teleport column is
plain PageRank with dangling mass spread uniformly, Eq. 1), the closed form on
a directed cycle, a dense linear solve, and invariants."""
import numpy as np
import pytest

import graphgen
import oracle
from oracle import ppr as P


def _seeds(n, sizes, rng):
    ptr = [0]
    idx = []
    for s in sizes:
        idx.extend(rng.choice(n, size=s, replace=False).tolist())
        ptr.append(len(idx))
    return np.array(ptr), np.array(idx)


def test_teleport_block():
    t = P.teleport(6, [0, 1, 4], [2, 0, 5, 3])
    np.testing.assert_array_equal(t[:, 0], [0, 0, 1, 0, 0, 0])
    np.testing.assert_allclose(t[:, 1], [1 / 3, 0, 0, 1 / 3, 0, 1 / 3])
    with pytest.raises(ValueError):
        P.teleport(6, [0, 2], [1, 1])
    with pytest.raises(ValueError):
        P.teleport(6, [0, 0], [])


@pytest.mark.parametrize("seed", [1, 2])
def test_uniform_teleport_is_pagerank(seed):
    rp, col = graphgen.rmat(10, 8, seed=seed)
    n = rp.size - 1
    ptr = np.array([0, n, 2 * n])
    idx = np.concatenate([np.arange(n), np.arange(n)[::-1]])
    got = P.ppr(rp, col, ptr, idx, 0.85, iters=15)
    ref = oracle.pagerank(rp, col, 0.85, iters=15, dangling="uniform")
    for j in range(2):
        np.testing.assert_allclose(got["r"][:, j], ref["x"], rtol=0, atol=1e-14)
        np.testing.assert_allclose(got["resid"][:, j], ref["resid"], rtol=1e-9, atol=1e-15)


def test_directed_cycle_closed_form():
    # u -> u+1 (mod L), one seed s: r(v) = (1-d) d^((v-s) mod L) / (1 - d^L)
    L, d = 9, 0.85
    rp, col = graphgen.csr_from_edges(L, np.arange(L), (np.arange(L) + 1) % L)
    for s in (0, 4):
        want = (1 - d) * d ** ((np.arange(L) - s) % L) / (1 - d ** L)
        np.testing.assert_allclose(P.fixed_point(rp, col, [0, 1], [s], d)[:, 0], want, rtol=1e-13)
        np.testing.assert_allclose(P.ppr(rp, col, [0, 1], [s], d, iters=400)["r"][:, 0], want, rtol=1e-10)


def test_iteration_converges_to_dense_solve():
    rng = np.random.default_rng(7)
    for trial in range(4):
        n = 40
        rp, col = graphgen.random_graph(n, 90, seed=100 + trial)  # has dangling nodes
        assert (np.diff(rp) == 0).any()
        ptr, idx = _seeds(n, [1, 3, 7, n], rng)
        want = P.fixed_point(rp, col, ptr, idx, 0.85)
        got = P.ppr(rp, col, ptr, idx, 0.85, iters=300)["r"]
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)


def test_no_edges_keeps_the_teleport():
    n = 12
    rp = np.zeros(n + 1, np.uint32)
    ptr, idx = _seeds(n, [1, 5], np.random.default_rng(3))
    out = P.ppr(rp, np.zeros(0, np.uint32), ptr, idx, 0.85, iters=5)
    np.testing.assert_allclose(out["r"], P.teleport(n, ptr, idx), rtol=0, atol=1e-16)
    assert np.all(out["resid"] < 1e-16)


def test_columns_keep_unit_mass():
    rp, col = graphgen.rmat(11, 16, seed=5, relabel="bfs")
    n = rp.size - 1
    ptr, idx = _seeds(n, [1, 10, 1000], np.random.default_rng(4))
    out = P.ppr(rp, col, ptr, idx, 0.85, iters=12, history=True)
    np.testing.assert_allclose(out["hist"].sum(axis=1), 1.0, rtol=0, atol=1e-12)
    assert np.all(out["hist"] >= 0)
