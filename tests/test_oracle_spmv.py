"""Pins of the oracle's weighted-graph functions (Sec. 3.5).

spmv is checked against a dense matrix product written independently, and the
bins-based weighted gather against spmv; bin_weights against a brute-force
reconstruction of the bin order from the edge list."""
import numpy as np

import graphgen
import oracle


def dense_product(rp, col, w, x):
    n = rp.size - 1
    A = np.zeros((n, n))
    for u in range(n):
        for e in range(int(rp[u]), int(rp[u + 1])):
            A[u, int(col[e])] += w[e]
    return A.T @ x


def graphs():
    yield graphgen.random_graph(40, 200, seed=1), 6
    yield graphgen.random_graph(300, 2000, seed=2), 64
    yield graphgen.rmat(9, 8, seed=3), 100
    yield graphgen.csr_from_edges(5, np.array([0, 0, 1, 3, 3, 3]), np.array([1, 4, 4, 0, 2, 4])) , 2


def test_spmv_equals_dense_product():
    rng = np.random.default_rng(7)
    for (rp, col), _ in graphs():
        w = rng.standard_normal(int(rp[-1]))
        x = rng.standard_normal(rp.size - 1)
        np.testing.assert_allclose(oracle.spmv(rp, col, w, x), dense_product(rp, col, w, x), rtol=1e-12, atol=1e-12)


def test_weighted_gather_over_bins_equals_spmv():
    rng = np.random.default_rng(8)
    for (rp, col), q in graphs():
        w = rng.standard_normal(int(rp[-1]))
        x = rng.standard_normal(rp.size - 1)
        g = oracle.png(rp, col, q)
        y = oracle.weighted_scatter_gather(g, oracle.bin_weights(rp, col, q, w, g), x)
        np.testing.assert_allclose(y, oracle.spmv(rp, col, w, x), rtol=1e-12, atol=1e-12)


def test_bin_weights_follow_the_destination_ids():
    # brute force: edges sorted by (destination partition, source, position
    # in the row) are the bins' order; the weight of each edge lands there
    rng = np.random.default_rng(9)
    for (rp, col), q in graphs():
        m = int(rp[-1])
        w = rng.standard_normal(m)
        src = np.repeat(np.arange(rp.size - 1), np.diff(rp.astype(np.int64)))
        order = np.lexsort((np.arange(m), src, col // q))
        g = oracle.png(rp, col, q)
        np.testing.assert_array_equal(g["dest_ids"] & 0x7FFFFFFF, col[order])
        np.testing.assert_array_equal(oracle.bin_weights(rp, col, q, w, g), w[order])


def rect(rows, cols, nnz, seed):
    rng = np.random.default_rng(seed)
    r = rng.integers(0, rows, nnz)
    c = rng.integers(0, cols, nnz)
    key = np.unique(r.astype(np.int64) * cols + c)
    r, c = key // cols, key % cols
    rp = np.zeros(rows + 1, np.uint32)
    np.add.at(rp, r + 1, 1)
    return np.cumsum(rp).astype(np.uint32), c.astype(np.uint32)


def test_rect_spmv_equals_dense_product():
    # a rows x cols matrix written out entry by entry: y = A^T x
    rng = np.random.default_rng(10)
    for rows, cols, nnz in ((7, 3, 12), (3, 11, 20), (50, 200, 900), (300, 40, 2000), (1, 5, 3)):
        rp, col = rect(rows, cols, nnz, rows * 31 + cols)
        w = rng.standard_normal(int(rp[-1]))
        x = rng.standard_normal(rows)
        A = np.zeros((rows, cols))
        for r in range(rows):
            for e in range(int(rp[r]), int(rp[r + 1])):
                A[r, int(col[e])] += w[e]
        np.testing.assert_allclose(oracle.spmv_rect(rp, col, w, x, cols), A.T @ x, rtol=1e-12, atol=1e-12)


def test_rect_spmv_of_a_square_matrix_is_spmv():
    rng = np.random.default_rng(11)
    (rp, col), _ = next(graphs())
    w = rng.standard_normal(int(rp[-1]))
    x = rng.standard_normal(rp.size - 1)
    np.testing.assert_array_equal(oracle.spmv_rect(rp, col, w, x, rp.size - 1), oracle.spmv(rp, col, w, x))
