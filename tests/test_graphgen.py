"""Properties of the seeded synthetic inputs (no method arithmetic here)."""
import numpy as np
import pytest

import graphgen


def check_csr(rp, col):
    n = rp.size - 1
    assert rp[0] == 0 and (np.diff(rp.astype(np.int64)) >= 0).all() and rp[-1] == col.size
    u = np.repeat(np.arange(n), np.diff(rp.astype(np.int64)))
    assert (col < n).all()
    assert (col != u).all()  # no self-loops
    same = u[1:] == u[:-1]
    assert (np.diff(col.astype(np.int64))[same] > 0).all()  # sorted, no duplicates


@pytest.mark.parametrize("relabel", ["none", "random", "bfs"])
def test_rmat_csr_valid_and_thread_independent(relabel):
    a = graphgen.rmat(12, 16, seed=1709, relabel=relabel, threads=1)
    b = graphgen.rmat(12, 16, seed=1709, relabel=relabel, threads=5)
    check_csr(*a)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


def test_relabelings_are_isomorphic():
    # Random and BFS labels permute nodes: the sorted degree sequences agree.
    degs = []
    for relabel in ("random", "bfs"):
        rp, col = graphgen.rmat(12, 16, seed=3, relabel=relabel)
        degs.append((np.sort(np.diff(rp.astype(np.int64))), np.sort(np.bincount(col, minlength=rp.size - 1))))
    np.testing.assert_array_equal(degs[0][0], degs[1][0])
    np.testing.assert_array_equal(degs[0][1], degs[1][1])


def test_rmat_skew_and_er_uniformity():
    rp, col = graphgen.rmat(14, 16, seed=1)
    indeg = np.bincount(col, minlength=rp.size - 1)
    assert indeg.max() > 50 * indeg.mean()  # power-law hubs
    rp, col = graphgen.erdos_renyi(1 << 14, 16, seed=1)
    check_csr(rp, col)
    assert abs(col.size / (1 << 14) - 16) < 0.1
    assert np.bincount(col).max() < 50


def test_seed_changes_graph():
    a = graphgen.rmat(10, 8, seed=1)[1]
    b = graphgen.rmat(10, 8, seed=2)[1]
    assert a.size != b.size or not np.array_equal(a, b)
