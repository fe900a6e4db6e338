"""Weighted graphs and SpMV over the PNG (Sec. 3.5) on the GPU.

The weights sit beside the destination IDs in bin order: compared bit for
bit with the oracle's placement (the same float32 values, permuted). The
product y = A^T_w x (FP32 accumulation) is compared per node with the FP64
oracle within the FP32 summation bound: a node with k in-edges sums k
products in some order, so |y - y*| <= (k + 4) * 2^-24 * sum |w x|.
"""
import numpy as np
import pytest

import graphgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1709_07122_gb300 as pcpm  # noqa: E402

U = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pcpm.build()
    pcpm.lib()


GRAPHS = {
    "rmat14_q2048": lambda: (graphgen.rmat(14, 16, seed=81), 2048),
    "rmat12_bfs_q512": lambda: (graphgen.rmat(12, 16, seed=82, relabel="bfs"), 512),
    "random1000_q7": lambda: (graphgen.random_graph(1000, 5000, seed=83), 7),
    "single_partition": lambda: (graphgen.random_graph(700, 4000, seed=84), 16384),
}


def weighted(rp, col, w, q, **opts):
    drp, dcol = pcpm.to_device_csr(rp, col)
    return pcpm.PNG.weighted(drp, dcol, torch.from_numpy(w).cuda(), q, **opts)


def bound(rp, col, w, x):
    k = np.bincount(col, minlength=rp.size - 1)
    mag = oracle.spmv(rp, col, np.abs(w.astype(np.float64)), np.abs(x.astype(np.float64)))
    return (k + 4) * U * mag + 1e-30


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_weighted_bins_bit_exact(name):
    (rp, col), q = GRAPHS[name]()
    rng = np.random.default_rng(85)
    w = rng.standard_normal(int(rp[-1])).astype(np.float32)
    ref = oracle.png(rp, col, q)
    with weighted(rp, col, w, q) as g:
        ex = g.export()
        wb = g.export_weights()
    for key in ("cnt_u", "cnt_e", "off_u", "off_e", "bin_u", "bin_e", "src_idx", "dest_ids"):
        np.testing.assert_array_equal(ex[key], np.asarray(ref[key], np.uint32), err_msg=key)
    want = oracle.bin_weights(rp, col, q, w.astype(np.float64), ref).astype(np.float32)
    np.testing.assert_array_equal(wb.view(np.uint32), want.view(np.uint32))


DECOMP = [dict(), dict(gather_unit_chunks=1, gather_cluster=1), dict(gather_unit_chunks=3, gather_cluster=4),
          dict(gather_unit_chunks=1 << 30, gather_cluster=8), dict(gather_windows=2),
          dict(gather_windows=2, gather_runs=1), dict(gather_windows=2, gather_runs=2),
          dict(gather_windows=2, gather_unit_chunks=1, gather_cluster=1)]


@pytest.mark.parametrize("opts", DECOMP, ids=lambda o: ",".join(f"{k}={v}" for k, v in o.items()) or "auto")
@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_spmv_matches_oracle(name, opts):
    (rp, col), q = GRAPHS[name]()
    rng = np.random.default_rng(86)
    w = rng.standard_normal(int(rp[-1])).astype(np.float32)
    x = rng.standard_normal(rp.size - 1).astype(np.float32)
    want = oracle.spmv(rp, col, w.astype(np.float64), x.astype(np.float64))
    with weighted(rp, col, w, q, **opts) as g:
        for _ in range(2):  # the handle is reusable
            y = g.spmv(torch.from_numpy(x).cuda()).cpu().numpy().astype(np.float64)
            assert np.all(np.abs(y - want) <= bound(rp, col, w, x))


def test_spmv_on_an_unweighted_handle_uses_unit_weights():
    (rp, col), q = GRAPHS["rmat14_q2048"]()
    x = np.random.default_rng(87).standard_normal(rp.size - 1).astype(np.float32)
    ones = np.ones(int(rp[-1]))
    with pcpm.PNG.from_host(rp, col, q) as g:
        y = g.spmv(torch.from_numpy(x).cuda()).cpu().numpy().astype(np.float64)
    assert np.all(np.abs(y - oracle.spmv(rp, col, ones, x)) <= bound(rp, col, ones.astype(np.float32), x))


def test_pagerank_on_a_weighted_handle_ignores_the_weights():
    (rp, col), q = GRAPHS["rmat12_bfs_q512"]()
    w = np.random.default_rng(88).random(int(rp[-1])).astype(np.float32)
    ref = oracle.pagerank(rp, col, 0.85, iters=5)["x"]
    with weighted(rp, col, w, q) as g:
        pr, _, _ = g.pagerank(0.85, max_iters=5)
    assert float(np.abs(pr.cpu().numpy().astype(np.float64) - ref).sum()) <= 1e-6


def test_bad_weighted_options_rejected():
    rp, col = graphgen.random_graph(300, 900, seed=7)
    w = np.ones(int(rp[-1]), np.float32)
    for q, opts in ((32768, {}), (64, dict(canonical_gather=1)), (64, dict(update_dtype="f16"))):
        with pytest.raises(pcpm.PcpmError) as e:
            weighted(rp, col, w, q, **opts)
        assert e.value.code == -1


def rect_matrix(rows, cols, nnz, seed):
    """A rows x cols CSR with sorted, distinct columns per row."""
    rng = np.random.default_rng(seed)
    r = rng.integers(0, rows, nnz)
    c = rng.integers(0, cols, nnz)
    key = np.unique(r.astype(np.int64) * cols + c)
    r, c = key // cols, key % cols
    rp = np.zeros(rows + 1, np.int64)
    np.add.at(rp, r + 1, 1)
    return np.cumsum(rp).astype(np.uint32), c.astype(np.uint32)


RECT = {
    "tall_5000x700_q256": (5000, 700, 40000, 256),
    "wide_600x9000_q1000": (600, 9000, 30000, 1000),
    "wide_ragged_1000x33001_q4096": (1000, 33001, 50000, 4096),
    "tall_one_col_partition_40000x300_q16384": (40000, 300, 200000, 16384),
    "single_row_1x5000_q7": (1, 5000, 3000, 7),
}


@pytest.mark.parametrize("opts", [{}, {"gather_windows": 2}, {"gather_unit_chunks": 1, "gather_cluster": 1}],
                         ids=["windows", "chunks", "cut_bins"])
@pytest.mark.parametrize("weights", [True, False], ids=["weighted", "unit"])
@pytest.mark.parametrize("name", sorted(RECT))
def test_rect_spmv_matches_oracle(name, weights, opts):
    rows, cols, nnz, q = RECT[name]
    rp, col = rect_matrix(rows, cols, nnz, seed=rows + cols)
    m = int(rp[-1])
    rng = np.random.default_rng(89)
    w = rng.standard_normal(m).astype(np.float32) if weights else np.ones(m, np.float32)
    x = rng.standard_normal(rows).astype(np.float32)
    want = oracle.spmv_rect(rp, col, w.astype(np.float64), x.astype(np.float64), cols)
    k = np.bincount(col, minlength=cols)
    mag = oracle.spmv_rect(rp, col, np.abs(w.astype(np.float64)), np.abs(x.astype(np.float64)), cols)
    drp, dcol = pcpm.to_device_csr(rp, col)
    wq = min(q, 16384) if weights else q
    g = pcpm.PNG.rect(drp, dcol, cols, wq, torch.from_numpy(w).cuda() if weights else None, **opts)
    with g:
        assert g.info["shard_part_hi"] == -(-cols // wq)  # only the column partitions are gathered
        for _ in range(2):  # the handle is reusable
            y = g.spmv_rect(torch.from_numpy(x).cuda()).cpu().numpy().astype(np.float64)
            assert y.shape == (cols,)
            assert np.all(np.abs(y - want) <= (k + 4) * U * mag + 1e-30)


def test_rect_rejects_pagerank_and_columns_out_of_range():
    rp, col = rect_matrix(300, 100, 1000, seed=5)
    drp, dcol = pcpm.to_device_csr(rp, col)
    with pcpm.PNG.rect(drp, dcol, 100, 64) as g:
        for call in (lambda: g.pagerank(0.85, 2), lambda: g.reset(), lambda: g.spmv(torch.ones(g.n, device="cuda"))):
            with pytest.raises(pcpm.PcpmError) as e:
                call()
            assert e.value.code == -1
    with pytest.raises(pcpm.PcpmError) as e:
        pcpm.PNG.rect(drp, dcol, 50, 64)  # columns up to 99 but only 50 declared
    assert e.value.code == -6
