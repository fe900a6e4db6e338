"""Reduced-precision update bins (FP16 of SPR * 2^15, BF16 of SPR) on the GPU.

Not in the paper, which stores 4-byte updates (Sec. 3.2). The stored update
bins are compared bit for bit with the oracle's formats applied to SPR
computed on the host. Each PageRank step is compared with the FP64 oracle's
step from the same ranks, within the bound the rounding allows: every stored
update carries a relative error of at most u (2^-11 for FP16 in its normal
range, 2^-8 for BF16) plus, for FP16, an absolute floor of 2^-25 * 2^-15 per
value below the normal range; summed over a node's out-edges this gives

    L1(step) <= d * (u * sum_{u not dangling} x(u) + m * 2^-40) + 1e-6,

the last term being the FP32 path's own bar.
"""
import numpy as np
import pytest

import graphgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1709_07122_gb300 as pcpm  # noqa: E402

UNIT = {"f16": 2.0 ** -11, "bf16": 2.0 ** -8}
FP32_BAR = 1e-6
D = 0.85


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pcpm.build()
    pcpm.lib()


GRAPHS = {
    "rmat14_q2048": lambda: (graphgen.rmat(14, 16, seed=41), 2048),
    "rmat12_bfs_q512": lambda: (graphgen.rmat(12, 16, seed=42, relabel="bfs"), 512),
    "random1000_q7": lambda: (graphgen.random_graph(1000, 5000, seed=43), 7),
    "er13_q1000": lambda: (graphgen.erdos_renyi(1 << 13, 8, seed=44), 1000),
}


def host_spr(x, rp):
    deg = np.diff(rp.astype(np.int64))
    inv = np.where(deg > 0, np.float32(1) / np.maximum(deg, 1).astype(np.float32), np.float32(0))
    return (np.asarray(x, np.float32) * inv.astype(np.float32)).astype(np.float32), deg


def step_bound(x, deg, m, dtype):
    live = float(np.asarray(x, np.float64)[deg > 0].sum())
    return D * (UNIT[dtype] * live + m * 2.0 ** -40) + FP32_BAR


@pytest.mark.parametrize("dtype", ["f16", "bf16"])
@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_stored_updates_bit_exact(name, dtype):
    (rp, col), q = GRAPHS[name]()
    n = rp.size - 1
    x0 = graphgen.random_rank_vector(n, seed=45).astype(np.float32)
    ref = oracle.png(rp, col, q)
    with pcpm.PNG.from_host(rp, col, q, update_dtype=dtype) as g:
        info = g.info
        assert info["update_bytes"] == 2 and info["update_dtype"] == pcpm.UPDATE_DTYPES[dtype]
        g.reset(torch.from_numpy(x0).cuda())
        g.scatter_only()
        st = g.export_state()
    spr, _ = host_spr(x0, rp)
    want = oracle.store_updates(spr[ref["src_idx"]], dtype)
    np.testing.assert_array_equal(st["updates"].view(np.uint16), want.view(np.uint16))


DECOMP = [dict(), dict(gather_unit_chunks=1 << 30), dict(gather_unit_chunks=1, gather_cluster=1),
          dict(gather_unit_chunks=3, gather_cluster=4), dict(gather_windows=2),
          dict(gather_windows=2, gather_runs=1), dict(gather_windows=2, gather_runs=2),
          dict(gather_windows=2, gather_unit_chunks=1, gather_cluster=1)]


@pytest.mark.parametrize("opts", DECOMP, ids=lambda o: ",".join(f"{k}={v}" for k, v in o.items()) or "auto")
@pytest.mark.parametrize("mode", ["two_phase", "fused"])
@pytest.mark.parametrize("dtype", ["f16", "bf16"])
@pytest.mark.parametrize("name", ["rmat14_q2048", "rmat12_bfs_q512"])
def test_each_step_within_rounding_bound(name, dtype, mode, opts):
    (rp, col), q = GRAPHS[name]()
    m = int(rp[-1])
    _, deg = host_spr(np.zeros(rp.size - 1, np.float32), rp)
    with pcpm.PNG.from_host(rp, col, q, update_dtype=dtype, **opts) as g:
        g.reset()
        x = g.ranks().cpu().numpy()
        for i in range(5):
            g.iterate(D, 1, mode=mode)
            y = g.ranks().cpu().numpy()
            want = oracle.pagerank(rp, col, D, iters=1, x0=x.astype(np.float64))["x"]
            err = float(np.abs(y.astype(np.float64) - want).sum())
            assert err <= step_bound(x, deg, m, dtype), (i, err, step_bound(x, deg, m, dtype))
            x = y


@pytest.mark.parametrize("dtype", ["f16", "bf16"])
def test_fused_iteration_leaves_next_updates_in_the_format(dtype):
    # A fused iteration scatters SPR' of the new ranks into the other update
    # buffer from shared memory: those bins equal the format of the host's
    # SPR' of the exported ranks.
    (rp, col), q = GRAPHS["rmat14_q2048"]()
    ref = oracle.png(rp, col, q)
    with pcpm.PNG.from_host(rp, col, q, update_dtype=dtype, gather_unit_chunks=1 << 30) as g:
        assert g.info["fused_ok"] == 1
        g.reset()
        g.iterate(D, 2, mode="fused")
        st = g.export_state()
    spr, _ = host_spr(st["pr"], rp)
    want = oracle.store_updates(spr[ref["src_idx"]], dtype)
    np.testing.assert_array_equal(st["updates"].view(np.uint16), want.view(np.uint16))


def test_bad_update_options_rejected():
    rp, col = graphgen.random_graph(300, 900, seed=7)
    for opts in (dict(update_dtype=3), dict(update_dtype="f16", canonical_gather=1)):
        with pytest.raises(pcpm.PcpmError) as e:
            pcpm.PNG.from_host(rp, col, 16, **opts)
        assert e.value.code == -1


def test_sixteen_bit_bins_halve_the_update_bytes():
    (rp, col), q = GRAPHS["rmat14_q2048"]()
    sizes = {}
    for dtype in ("f32", "f16", "bf16"):
        with pcpm.PNG.from_host(rp, col, q, update_dtype=dtype) as g:
            sizes[dtype] = (g.info["update_bytes"], g.info["device_bytes"], g.info["num_updates"])
    ne = sizes["f32"][2]
    assert sizes["f32"][0] == 4 and sizes["f16"][0] == 2 and sizes["bf16"][0] == 2
    # two update buffers of |E'| + 16 entries each; 16-bit handles keep two
    # FP32 rounding left-overs per node for delta iterations
    n = rp.size - 1
    assert sizes["f32"][1] - sizes["f16"][1] == 2 * (ne + 16) * 2 - 8 * n
    assert sizes["f16"][1] == sizes["bf16"][1]
