"""GPU parity of the CUDA path against the FP64 oracle, through the C ABI.

Bar: PNG counts, offsets, bin starts and bins bit-exact; the scatter's update
bins bit-exact (a float copy); ranks within L1 1e-6 of the oracle on every
iteration (FP32 ranks, FP32 shared-memory accumulation, FP64 reductions).
"""
import ctypes

import numpy as np
import pytest

import graphgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1709_07122_gb300 as pcpm  # noqa: E402

L1_TOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pcpm.build()
    pcpm.lib()


def assert_png_matches(g: dict, ref: dict):
    assert g["k"] == ref["k"] and g["ne"] == ref["ne"] and g["m"] == ref["m"]
    for key in ("cnt_u", "cnt_e", "off_u", "off_e", "bin_u", "bin_e", "src_idx", "dest_ids"):
        np.testing.assert_array_equal(g[key], np.asarray(ref[key], dtype=np.uint32), err_msg=key)


def l1(a, b):
    return float(np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64)).sum())


GRAPHS = {
    "rmat16_q16384": lambda: (graphgen.rmat(16, 16, seed=1709), 16384),
    "rmat12_q100_ragged": lambda: (graphgen.rmat(12, 16, seed=3), 100),
    "rmat12_bfs_q512": lambda: (graphgen.rmat(12, 16, seed=4, relabel="bfs"), 512),
    "er14_q512": lambda: (graphgen.erdos_renyi(1 << 14, 16, seed=5), 512),
    "random1000_q7": lambda: (graphgen.random_graph(1000, 5000, seed=6), 7),
    "random300_q1": lambda: (graphgen.random_graph(300, 900, seed=7), 1),
    "single_partition": lambda: (graphgen.random_graph(500, 3000, seed=8), 32768),
    "rmat10_q32768_k1": lambda: (graphgen.rmat(10, 8, seed=9), 32768),
    "rmat14_q_not_multiple": lambda: (graphgen.rmat(14, 16, seed=10), 3000),
    # the staged fill's largest partition count, and one past it (direct fill)
    "rmat12_q4_k1024": lambda: (graphgen.rmat(12, 16, seed=12), 4),
    "random5000_q3_k1667": lambda: (graphgen.random_graph(5000, 40000, seed=11), 3),
    # mostly empty rows: a tile's rows span thousands of zero-degree nodes
    "sparse200000_q32768": lambda: (graphgen.random_graph(200000, 30000, seed=13), 32768),
}


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_png_bit_exact(name):
    (rp, col), q = GRAPHS[name]()
    with pcpm.PNG.from_host(rp, col, q) as g:
        assert_png_matches(g.export(), oracle.png(rp, col, q))


def test_png_edge_cases_bit_exact():
    cases = []
    # one node, no edges
    cases.append((np.array([0, 0], np.uint32), np.array([], np.uint32), 1))
    # no edges at all
    cases.append((np.zeros(11, np.uint32), np.array([], np.uint32), 3))
    # hub pointing everywhere, isolated and dangling nodes, empty bins
    n = 70
    src = [0] * (n - 1) + list(range(5, n, 3))
    dst = list(range(1, n)) + [2] * len(range(5, n, 3))
    cases.append(graphgen.csr_from_edges(n, np.array(src), np.array(dst)) + (8,))
    # duplicates and self-loops kept as ordinary edges
    rp, col = graphgen.csr_from_edges(20, np.array([1, 1, 1, 2, 2, 5]), np.array([3, 3, 1, 2, 19, 0]),
                                      dedupe=False, drop_self_loops=False)
    cases.append((rp, col, 4))
    # a tile boundary inside one long row (> 8192 edges from one node)
    n = 20000
    rp, col = graphgen.csr_from_edges(n, np.zeros(n - 1, int), np.arange(1, n))
    cases.append((rp, col, 1024))
    for rp, col, q in cases:
        with pcpm.PNG.from_host(rp, col, q) as g:
            assert_png_matches(g.export(), oracle.png(rp, col, q))


def test_paper_offsets_example_on_gpu():
    rp, col = graphgen.csr_from_edges(9, np.array([0, 0, 3, 6, 7, 8]), np.array([6, 8, 4, 0, 3, 2]))
    with pcpm.PNG.from_host(rp, col, 3) as g:
        assert list(g.export()["off_u"][2]) == [0, 1, 1]


@pytest.mark.parametrize("name", ["rmat16_q16384", "rmat12_q100_ragged", "random1000_q7", "er14_q512"])
def test_scatter_bit_exact(name):
    (rp, col), q = GRAPHS[name]()
    n = rp.size - 1
    x0 = torch.from_numpy(graphgen.random_rank_vector(n, seed=21).astype(np.float32)).cuda()
    ref = oracle.png(rp, col, q)
    with pcpm.PNG.from_host(rp, col, q) as g:
        g.reset(x0)
        g.scatter_only()
        st = g.export_state()
        # scatter: update[t] = SPR[src[t]] exactly (Algorithm 3)
        np.testing.assert_array_equal(st["updates"], st["spr"][ref["src_idx"]])
        # SPR_0 = PR_0 / outdeg in FP32 (1/outdeg rounded once, then one product)
        deg = np.diff(rp.astype(np.int64))
        inv = np.where(deg > 0, np.float32(1) / np.maximum(deg, 1).astype(np.float32), np.float32(0))
        np.testing.assert_array_equal(st["spr"], (x0.cpu().numpy() * inv.astype(np.float32)).astype(np.float32))
        np.testing.assert_allclose(st["dangling"], x0.cpu().numpy().astype(np.float64)[deg == 0].sum(), rtol=1e-12)


@pytest.mark.parametrize("canonical", [0, 1])
@pytest.mark.parametrize("mode", ["fused", "two_phase"])
@pytest.mark.parametrize("dangling", ["uniform", "leak"])
@pytest.mark.parametrize("start", ["uniform", "random"])
def test_iterations_rmat16_l1_every_iteration(dangling, start, mode, canonical):
    # RMAT scale 16, edge factor 16, q = 16384, d = 0.85, 20 iterations.
    (rp, col), q = GRAPHS["rmat16_q16384"]()
    n = rp.size - 1
    x0 = None if start == "uniform" else graphgen.random_rank_vector(n, seed=33)
    ref = oracle.pagerank(rp, col, 0.85, iters=20, x0=x0, dangling=dangling, history=True)
    x0_t = None if x0 is None else torch.from_numpy(x0.astype(np.float32)).cuda()
    with pcpm.PNG.from_host(rp, col, q, canonical_gather=canonical) as g:
        g.reset(x0_t)
        errs = []
        for i in range(1, 21):
            g.iterate(0.85, 1, dangling=dangling, mode=mode)
            errs.append(l1(g.ranks().cpu().numpy(), ref["hist"][i]))
        assert max(errs) <= L1_TOL, errs
        hist = g.residual_history()
        assert hist.size == 20
        np.testing.assert_allclose(hist, ref["resid"], rtol=1e-3, atol=2e-7)


@pytest.mark.parametrize("mode", ["fused", "two_phase"])
@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_pagerank_matches_oracle(name, mode):
    (rp, col), q = GRAPHS[name]()
    ref = oracle.pagerank(rp, col, 0.85, iters=20)["x"]
    with pcpm.PNG.from_host(rp, col, q) as g:
        pr, iters, res = g.pagerank(0.85, max_iters=20, mode=mode)
        assert iters == 20
        assert l1(pr.cpu().numpy(), ref) <= L1_TOL


def test_modes_interleave():
    # Fused and two-phase iterations share one state: any mix of them follows
    # the oracle, and a fused step after a two-phase one rescatters first.
    (rp, col), q = GRAPHS["rmat12_q100_ragged"]()
    ref = oracle.pagerank(rp, col, 0.85, iters=9, history=True)["hist"]
    with pcpm.PNG.from_host(rp, col, q) as g:
        g.reset()
        done = 0
        for mode, k in [("fused", 2), ("two_phase", 1), ("fused", 3), ("two_phase", 2), ("fused", 1)]:
            g.iterate(0.85, k, mode=mode)
            done += k
            assert l1(g.ranks().cpu().numpy(), ref[done]) <= L1_TOL, (mode, done)


def test_fused_scatter_writes_next_bins_bit_exact():
    # After a fused iteration the current update bins hold SPR of the new ranks
    # at every PNG position (the fused kernel's scatter half).
    (rp, col), q = GRAPHS["rmat14_q_not_multiple"]()
    ref = oracle.png(rp, col, q)
    with pcpm.PNG.from_host(rp, col, q, gather_unit_chunks=1 << 30) as g:
        assert g.info["fused_ok"] == 1
        g.reset()
        g.iterate(0.85, 3)
        st = g.export_state()
        np.testing.assert_array_equal(st["updates"], st["spr"][ref["src_idx"]])


def test_tolerance_stops_at_first_iteration_below():
    (rp, col), q = GRAPHS["rmat12_q100_ragged"]()
    ref = oracle.pagerank(rp, col, 0.85, iters=200)
    first = int(np.argmax(ref["resid"] < 1e-6)) + 1
    with pcpm.PNG.from_host(rp, col, q) as g:
        pr, iters, res = g.pagerank(0.85, max_iters=200, tol=1e-6)
        assert res < 1e-6
        assert abs(iters - first) <= 1
        hist = g.residual_history()
        assert hist.size == iters and hist[-1] == res and (hist[:-1] >= 1e-6).all()
        # too few iterations: NOT_CONVERGED is reported, ranks still returned
        pr, iters, res = g.pagerank(0.85, max_iters=3, tol=1e-12)
        assert iters == 3 and res > 1e-12


def test_state_continues_across_calls_and_reset():
    (rp, col), q = GRAPHS["er14_q512"]()
    ref = oracle.pagerank(rp, col, 0.9, iters=7, history=True)["hist"]
    with pcpm.PNG.from_host(rp, col, q) as g:
        g.reset()
        g.iterate(0.9, 3)
        g.iterate(0.9, 4, sync=False)
        assert l1(g.ranks().cpu().numpy(), ref[7]) <= L1_TOL
        assert g.info["iterations_done"] == 7
        g.reset()
        assert l1(g.ranks().cpu().numpy(), ref[0]) <= 1e-6
        g.iterate(0.9, 2)
        assert l1(g.ranks().cpu().numpy(), ref[2]) <= L1_TOL


def test_closed_forms_on_gpu():
    # Directed cycle: 1/n stays fixed; in-star with a dangling centre.
    n = 5000
    rp, col = graphgen.csr_from_edges(n, np.arange(n), (np.arange(n) + 1) % n)
    with pcpm.PNG.from_host(rp, col, 512) as g:
        pr, _, _ = g.pagerank(0.85, 20)
        np.testing.assert_allclose(pr.cpu().numpy(), 1.0 / n, rtol=1e-5)
    rp, col = graphgen.csr_from_edges(n, np.arange(1, n), np.zeros(n - 1, int))
    d = 0.85
    with pcpm.PNG.from_host(rp, col, 777) as g:
        pr, _, _ = g.pagerank(d, 200)
        x = pr.cpu().numpy()
        den = n + d * (n - 1)
        # The centre sums n-1 equal FP32 terms in shared memory every iteration:
        # a sequential FP32 sum of N terms is within gamma_N = N*2^-24 (relative)
        # of the exact sum, about 3e-4 here; the leaves inherit it through D/n.
        gamma = (n - 1) * 2.0 ** -24
        np.testing.assert_allclose(x[1:], 1 / den, rtol=gamma)
        np.testing.assert_allclose(x[0], (1 + d * (n - 1)) / den, rtol=gamma)
        assert abs(x.astype(np.float64).sum() - 1) < 2 * gamma


def test_pagerank_host_end_to_end():
    (rp, col), q = GRAPHS["rmat12_q100_ragged"]()
    ref = oracle.pagerank(rp, col, 0.85, iters=20)["x"]
    pr, iters, res = pcpm.pagerank_host(rp, col, q, 0.85, 20)
    assert iters == 20 and l1(pr, ref) <= L1_TOL


def test_pool_reuse_across_builds_and_trim():
    """Freed handles return their memory to the library's pool; later builds
    reuse it (different sizes, interleaved lifetimes) and stay bit-exact."""
    a_rp, a_col = graphgen.rmat(14, 16, seed=21)
    b_rp, b_col = graphgen.erdos_renyi(1 << 13, 8, seed=22)
    ref_a, ref_b = oracle.png(a_rp, a_col, 1000), oracle.png(b_rp, b_col, 512)
    for _ in range(3):
        ga = pcpm.PNG.from_host(a_rp, a_col, 1000)
        with pcpm.PNG.from_host(b_rp, b_col, 512) as gb:
            ga.close()
            assert_png_matches(gb.export(), ref_b)
        with pcpm.PNG.from_host(a_rp, a_col, 1000) as ga2:
            assert_png_matches(ga2.export(), ref_a)
    ref = oracle.pagerank(a_rp, a_col, 0.85, iters=10)["x"]
    for _ in range(3):  # shared-memory atomics: equal within the tolerance, not bitwise
        assert l1(pcpm.pagerank_host(a_rp, a_col, 1000, 0.85, 10)[0], ref) <= L1_TOL
    pcpm.release_cached_memory()
    with pcpm.PNG.from_host(b_rp, b_col, 512) as gb:
        assert_png_matches(gb.export(), ref_b)
    pcpm.release_cached_memory()


def test_autotune_picks_the_fastest_valid_part_size():
    rp, col = graphgen.rmat(14, 16, seed=40)
    d_rp, d_col = pcpm.to_device_csr(rp, col)
    best, ms = pcpm.autotune(d_rp, d_col, (1024, 4096, 16384, 40000), iters=3)
    assert ms[40000] is None  # above the largest partition size: rejected, not fatal
    valid = {q: t for q, t in ms.items() if t is not None}
    assert set(valid) == {1024, 4096, 16384} and all(t > 0 for t in valid.values())
    assert best == min(valid, key=valid.get)
    with pytest.raises(pcpm.PcpmError):
        pcpm.autotune(d_rp, d_col, (40000, 0))


def test_autotune_over_tile_shapes_picks_the_fastest_valid_pair():
    rp, col = graphgen.rmat(14, 16, seed=40)
    d_rp, d_col = pcpm.to_device_csr(rp, col)
    shapes = ({}, {"gather_cluster": 1}, {"gather_unit_chunks": 64}, {"gather_windows": 2},
              {"gather_cluster": 3})  # 3 is not a cluster size: rejected
    best_q, best_opts, table = pcpm.autotune_tiles(d_rp, d_col, (2048, 8192), shapes, iters=3)
    assert all(table[(q, 4)] is None for q in (2048, 8192))
    valid = {k: t for k, t in table.items() if t is not None}
    assert len(valid) == 8 and all(t > 0 for t in valid.values())
    q, j = min(valid, key=valid.get)
    assert (best_q, best_opts) == (q, shapes[j])
    # the chosen pair solves like any other
    ref = oracle.pagerank(rp, col, 0.85, iters=5)["x"]
    with pcpm.PNG(d_rp, d_col, best_q, **best_opts) as g:
        x, _, _ = g.pagerank(0.85, max_iters=5)
    assert l1(x.cpu().numpy(), ref) <= L1_TOL


def test_errors_from_bad_inputs():
    rp = np.array([0, 2, 3, 3], np.uint32)
    unsorted = np.array([2, 1, 0], np.uint32)
    with pytest.raises(pcpm.PcpmError) as e:
        pcpm.PNG.from_host(rp, unsorted, 2)
    assert e.value.code == -6
    out_of_range = np.array([1, 7, 0], np.uint32)
    with pytest.raises(pcpm.PcpmError) as e:
        pcpm.PNG.from_host(rp, out_of_range, 2)
    assert e.value.code == -6
    decreasing = np.array([0, 2, 1, 3], np.uint32)
    with pytest.raises(pcpm.PcpmError) as e:
        pcpm.PNG.from_host(decreasing, np.array([1, 2, 0], np.uint32), 2)
    assert e.value.code == -6
    # host pointers where device pointers are required
    h = ctypes.c_void_p()
    host_rp = rp.ctypes.data_as(ctypes.c_void_p)
    assert pcpm.lib().pcpm_build(host_rp, host_rp, 3, 3, 2, None, ctypes.byref(h)) == -1
    (rp2, col2), q = GRAPHS["random300_q1"]()
    with pcpm.PNG.from_host(rp2, col2, q) as g:
        with pytest.raises(pcpm.PcpmError):
            g.iterate(1.0, 1)
        with pytest.raises(ValueError):
            g.iterate(0.85, 1, dangling="bogus")


DECOMPOSITIONS = [
    dict(),                                             # automatic: window layout
    dict(gather_unit_chunks=1 << 30),                   # one unit per bin: fused path
    dict(gather_unit_chunks=1, gather_cluster=1),       # every window its own unit
    dict(gather_unit_chunks=3, gather_cluster=4),       # CTAs of a cluster without windows
    dict(gather_unit_chunks=1 << 30, gather_cluster=8),
    dict(scatter_unit_groups=1),                        # every 4-update group its own unit
    dict(scatter_unit_groups=7, gather_unit_chunks=5, gather_cluster=2),
    dict(canonical_gather=1),                           # decode the canonical bins' flags
    dict(canonical_gather=1, gather_unit_chunks=1 << 30),
    dict(canonical_gather=1, gather_unit_chunks=2, gather_cluster=1),
    dict(gather_windows=2),                             # bank-spread 256-ID chunks, atomics
    dict(gather_windows=2, gather_runs=1),              # ... with register runs
    dict(gather_windows=2, gather_runs=1, gather_unit_chunks=1 << 30),
    dict(gather_windows=2, gather_runs=1, gather_unit_chunks=1, gather_cluster=1),
    dict(gather_windows=2, gather_runs=2),              # ... one shared-memory add per ID
]


@pytest.mark.parametrize("opts", DECOMPOSITIONS, ids=lambda o: ",".join(f"{k}={v}" for k, v in o.items()) or "auto")
@pytest.mark.parametrize("name", ["rmat12_bfs_q512", "rmat14_q_not_multiple", "random1000_q7", "single_partition"])
@pytest.mark.parametrize("mode", ["fused", "two_phase"])
def test_work_decompositions_match_oracle(name, opts, mode):
    # How bins and source partitions are cut into work units, and how many
    # CTAs share a unit, changes scheduling only: the bins stay bit-exact and
    # the ranks follow the oracle on every iteration.
    (rp, col), q = GRAPHS[name]()
    ref = oracle.pagerank(rp, col, 0.85, iters=6, history=True)["hist"]
    with pcpm.PNG.from_host(rp, col, q, **opts) as g:
        info = g.info
        k = info["num_partitions"]
        assert info["gather_units"] >= k and info["scatter_units"] >= k
        assert info["fused_ok"] == (info["gather_units"] == k)
        assert info["canonical_gather"] == opts.get("canonical_gather", 0)
        assert info["gather_windows"] == (not opts.get("canonical_gather") and opts.get("gather_windows", 0) != 2)
        assert info["merged_adds"] <= int(rp[-1])
        if info["canonical_gather"]:
            assert info["gather_runs"] == 0 and info["merged_adds"] == 0
        elif info["gather_windows"]:
            assert info["gather_runs"] == 1 and info["num_windows"] >= 1
        elif opts.get("gather_runs"):
            assert info["gather_runs"] == (opts["gather_runs"] == 1)
        else:
            assert info["gather_runs"] == (info["merged_adds"] * 16 >= info["num_edges"])
        if opts.get("gather_unit_chunks") == 1 << 30:
            assert info["gather_units"] == k
        g.reset()
        for i in range(1, 7):
            g.iterate(0.85, 1, mode=mode)
            assert l1(g.ranks().cpu().numpy(), ref[i]) <= L1_TOL, i
    if opts in (DECOMPOSITIONS[2], DECOMPOSITIONS[7]):
        with pcpm.PNG.from_host(rp, col, q, **opts) as g:
            assert_png_matches(g.export(), oracle.png(rp, col, q))


def test_skewed_bins_are_cut_into_units():
    # BFS labels put most in-edges into the first partitions (a few bins hold
    # most of the graph): the automatic decomposition cuts them into several
    # gather units, and the result still follows the oracle.
    rp, col = graphgen.rmat(16, 16, seed=1710, relabel="bfs")
    q = 4096
    ref = oracle.pagerank(rp, col, 0.85, iters=5)["x"]
    with pcpm.PNG.from_host(rp, col, q) as g:
        info = g.info
        assert info["gather_units"] > info["num_partitions"]
        pr, iters, _ = g.pagerank(0.85, max_iters=5)
        assert l1(pr.cpu().numpy(), ref) <= L1_TOL


def test_bad_cluster_option_rejected():
    (rp, col), q = GRAPHS["random300_q1"]()
    with pytest.raises(pcpm.PcpmError) as e:
        pcpm.PNG.from_host(rp, col, q, gather_cluster=3)
    assert e.value.code == -1
    with pytest.raises(pcpm.PcpmError) as e:
        pcpm.PNG.from_host(rp, col, q, gather_runs=3)
    assert e.value.code == -1
    for bad in (dict(gather_windows=3), dict(gather_windows=1, canonical_gather=1)):
        with pytest.raises(pcpm.PcpmError) as e:
            pcpm.PNG.from_host(rp, col, q, **bad)
        assert e.value.code == -1


def test_hot_destinations_take_register_runs():
    # Every source points at the same 40 nodes: inside a bank each of them
    # repeats, so most IDs join a run and the automatic choice sums runs in
    # registers; a uniform random graph with large partitions has few repeats
    # per chunk and keeps one add per ID. Both follow the oracle.
    rng = np.random.default_rng(77)
    n = 6000
    src = np.repeat(np.arange(n), 12)
    dst = rng.integers(0, 40, size=src.size) * 7 % 97
    rp, col = graphgen.csr_from_edges(n, src, dst)
    ref = oracle.pagerank(rp, col, 0.85, iters=5)["x"]
    with pcpm.PNG.from_host(rp, col, 1024) as g:
        info = g.info
        assert info["merged_adds"] * 4 >= int(rp[-1]), info
        assert info["gather_runs"] == 1
        pr, _, _ = g.pagerank(0.85, max_iters=5)
        assert l1(pr.cpu().numpy(), ref) <= L1_TOL
    rp, col = graphgen.random_graph(1 << 15, 1 << 18, seed=5)
    with pcpm.PNG.from_host(rp, col, 1 << 15, gather_windows=2) as g:
        assert g.info["gather_runs"] == 0, g.info
    for layout in (0, 2):  # both gather layouts with the hot destinations
        rp, col = graphgen.csr_from_edges(n, src, dst)
        with pcpm.PNG.from_host(rp, col, 1024, gather_windows=layout) as g:
            assert g.info["gather_windows"] == (layout == 0)
            pr, _, _ = g.pagerank(0.85, max_iters=5)
            assert l1(pr.cpu().numpy(), ref) <= L1_TOL


def test_handles_with_different_partition_sizes_coexist():
    # Kernel limits (such as the dynamic shared memory a launch may use) are
    # shared by all handles: building a small-q handle must not break a
    # large-q handle built before it, and the other way round.
    graphs = [(graphgen.rmat(10, 8, seed=91), 32768), (graphgen.rmat(11, 8, seed=92), 64),
              (graphgen.rmat(9, 8, seed=93), 4096)]
    handles = [pcpm.PNG.from_host(rp, col, q) for (rp, col), q in graphs]
    refs = [oracle.pagerank(rp, col, 0.85, iters=4)["x"] for (rp, col), _ in graphs]
    for order in ([0, 1, 2], [2, 0, 1]):
        for i in order:
            handles[i].reset()
            handles[i].iterate(0.85, 4, mode="two_phase")
            assert l1(handles[i].ranks().cpu().numpy(), refs[i]) <= L1_TOL
    for h in handles:
        h.close()
