"""Destination shards on the GPU, through the C ABI, against the FP64 oracle.

* Bins: each shard's bins of its own destination partitions equal the whole
  graph's bins of the oracle bit for bit (counts, offsets, sources, IDs), its
  other bins are empty, and the shards' bins together make up the whole PNG.
* Ranks: the shards of one graph, each driven by pcpm_shard_init and
  pcpm_shard_step, with their sums added and their slices copied between
  iterations as the exchange does, follow the oracle within L1 1e-6 on each of
  20 iterations under both dangling readings, and their summed L1 changes
  follow the oracle's.
* Two processes, one shard each, exchanging over gloo (host-staged), run the
  product's sharded solve (sharded.ShardedPageRank). The two processes share
  this GPU; their kernels never wait on each other (the exchange is on the
  host between iterations).
"""
import json
import os
import socket

import numpy as np
import pytest

import graphgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1709_07122_gb300 as pcpm  # noqa: E402
from paper_1709_07122_gb300.sharded import node_bounds  # noqa: E402

L1_TOL = 1e-6
D = 0.85


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pcpm.build()
    pcpm.lib()


def l1(a, b):
    return float(np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64)).sum())


GRAPHS = {
    "rmat16_q16384": lambda: (graphgen.rmat(16, 16, seed=1709), 16384),  # the C1 configuration
    "rmat13_q300_ragged": lambda: (graphgen.rmat(13, 12, seed=21), 300),
    "er13_q512": lambda: (graphgen.erdos_renyi(1 << 13, 16, seed=22), 512),
    "rmat12_bfs_q100": lambda: (graphgen.rmat(12, 16, seed=23, relabel="bfs"), 100),
    "random2000_q7": lambda: (graphgen.random_graph(2000, 9000, seed=24), 7),
}


def split(rp, col, q, nranks):
    n = rp.size - 1
    d_rp, d_col = pcpm.to_device_csr(rp, col)
    counts = pcpm.dest_partition_counts(d_col, n, q, m=col.size)
    k = (n + q - 1) // q
    np.testing.assert_array_equal(counts, np.bincount(col // q, minlength=k).astype(np.uint64))
    return d_rp, d_col, pcpm.shard_split(counts, n, q, nranks)


@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("nranks", [2, 3])
def test_shard_bins_bit_exact(name, nranks):
    (rp, col), q = GRAPHS[name]()
    ref = oracle.png(rp, col, q)
    d_rp, d_col, cuts = split(rp, col, q, nranks)
    k = ref["k"]
    seen_u = np.zeros(k, int)
    for r in range(nranks):
        lo, hi = int(cuts[r]), int(cuts[r + 1])
        g = pcpm.PNG.shard(d_rp, d_col, q, lo, hi)
        info = g.info
        assert (info["shard_part_lo"], info["shard_part_hi"]) == (lo, hi)
        out = g.export()
        g.close()
        own = np.zeros(k, bool)
        own[lo:hi] = True
        for key in ("cnt_u", "cnt_e", "off_u", "off_e"):
            refk = np.asarray(ref[key], np.uint32).reshape(k, k)
            np.testing.assert_array_equal(out[key][:, own], refk[:, own], err_msg=key)
        assert not out["cnt_u"][:, ~own].any() and not out["cnt_e"][:, ~own].any()
        for p in range(lo, hi):
            a, b = int(out["bin_u"][p]), int(out["bin_u"][p + 1])
            ra, rb = int(ref["bin_u"][p]), int(ref["bin_u"][p + 1])
            np.testing.assert_array_equal(out["src_idx"][a:b], ref["src_idx"][ra:rb])
            a, b = int(out["bin_e"][p]), int(out["bin_e"][p + 1])
            ra, rb = int(ref["bin_e"][p]), int(ref["bin_e"][p + 1])
            np.testing.assert_array_equal(out["dest_ids"][a:b], ref["dest_ids"][ra:rb])
            seen_u[p] += 1
        assert info["num_edges"] == int(ref["bin_e"][hi]) - int(ref["bin_e"][lo])
        assert info["num_updates"] == int(ref["bin_u"][hi]) - int(ref["bin_u"][lo])
    assert np.all(seen_u == 1)  # every bin in exactly one shard


def run_shards(shards, n, bounds, iters, dangling, pr_init=None):
    """The sharded iteration in one process: the exchange done by hand."""
    pr = [[torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(2)] for _ in shards]
    sums = [torch.zeros(2, dtype=torch.float64, device="cuda") for _ in shards]
    for g, p, s in zip(shards, pr, sums):
        g.shard_init(p[0], s, pr_init)
    total = sum(s for s in sums)
    for s in sums:
        s.copy_(total)
    cur, xs, res = 0, [], []
    for _ in range(iters):
        for g, p, s in zip(shards, pr, sums):
            g.shard_step(p[cur], p[cur ^ 1], s, D, dangling)
        total = sum(s for s in sums)
        full = torch.empty(n, dtype=torch.float32, device="cuda")
        for r, p in enumerate(pr):
            full[bounds[r]:bounds[r + 1]] = p[cur ^ 1][bounds[r]:bounds[r + 1]]
        for p, s in zip(pr, sums):
            p[cur ^ 1].copy_(full)
            s.copy_(total)
        cur ^= 1
        xs.append(full.cpu().numpy())
        res.append(float(total[0]))
    for g in shards:
        g.sync_status()
    return xs, res


@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("nranks,dangling", [(2, "uniform"), (3, "uniform"), (2, "leak"), (5, "uniform")])
def test_shards_follow_oracle_every_iteration(name, nranks, dangling):
    (rp, col), q = GRAPHS[name]()
    n = rp.size - 1
    k = (n + q - 1) // q
    if nranks > k:
        pytest.skip("fewer partitions than ranks")
    ref = oracle.pagerank(rp, col, D, iters=20, dangling=dangling, history=True)
    d_rp, d_col, cuts = split(rp, col, q, nranks)
    bounds = node_bounds(cuts, n, q)
    shards = [pcpm.PNG.shard(d_rp, d_col, q, int(cuts[r]), int(cuts[r + 1])) for r in range(nranks)]
    xs, res = run_shards(shards, n, bounds, 20, dangling)
    for g in shards:
        g.close()
    for i in range(20):
        assert l1(xs[i], ref["hist"][i + 1]) <= L1_TOL, (i, l1(xs[i], ref["hist"][i + 1]))
        assert abs(res[i] - ref["resid"][i]) <= 2 * L1_TOL, (i, res[i], ref["resid"][i])


def test_shards_from_a_given_start_and_with_the_window_and_chunk_layouts():
    rp, col = graphgen.rmat(14, 16, seed=25)
    q, n = 2048, rp.size - 1
    x0 = graphgen.random_rank_vector(n, seed=26)
    ref = oracle.pagerank(rp, col, D, iters=6, x0=x0, history=True)
    d_rp, d_col, cuts = split(rp, col, q, 3)
    bounds = node_bounds(cuts, n, q)
    for opts in ({"gather_windows": 1}, {"gather_windows": 2}, {"canonical_gather": 1, "gather_windows": 2},
                 {"update_dtype": "f32", "gather_unit_chunks": 3}):
        shards = [pcpm.PNG.shard(d_rp, d_col, q, int(cuts[r]), int(cuts[r + 1]), **opts) for r in range(3)]
        xs, _ = run_shards(shards, n, bounds, 6, "uniform",
                           torch.from_numpy(x0.astype(np.float32)).cuda())
        for g in shards:
            g.close()
        for i in range(6):
            assert l1(xs[i], ref["hist"][i + 1]) <= L1_TOL, (opts, i)


def test_whole_graph_handle_is_its_own_shard():
    rp, col = graphgen.rmat(13, 16, seed=27)
    n, q = rp.size - 1, 1024
    ref = oracle.pagerank(rp, col, D, iters=5, history=True)
    with pcpm.PNG.from_host(rp, col, q) as g:
        xs, res = run_shards([g], n, [0, n], 5, "uniform")
        for i in range(5):
            assert l1(xs[i], ref["hist"][i + 1]) <= L1_TOL
        # and it still solves normally afterwards
        pr, its, _ = g.pagerank(D, max_iters=5)
        assert its == 5 and l1(pr.cpu().numpy(), ref["x"]) <= L1_TOL


def test_partial_shard_rejects_whole_graph_calls():
    rp, col = graphgen.rmat(12, 16, seed=28)
    d_rp, d_col = pcpm.to_device_csr(rp, col)
    g = pcpm.PNG.shard(d_rp, d_col, 512, 0, 3)
    for call in (lambda: g.reset(), lambda: g.iterate(D, 1), lambda: g.pagerank(D, 2),
                 lambda: g.spmv(torch.ones(g.n, device="cuda"))):
        with pytest.raises(pcpm.PcpmError) as e:
            call()
        assert e.value.code == -1
    with pytest.raises(pcpm.PcpmError):
        pcpm.PNG.shard(d_rp, d_col, 512, 3, 3)  # empty range
    with pytest.raises(pcpm.PcpmError):
        pcpm.PNG.shard(d_rp, d_col, 512, 0, 9)  # past k = 8
    g.close()


def test_shard_rejects_a_bad_column():
    rp = np.array([0, 2, 3, 3], np.uint32)
    col = np.array([1, 7, 0], np.uint32)  # 7 >= n = 3, outside every shard's range
    d_rp, d_col = pcpm.to_device_csr(rp, col)
    with pytest.raises(pcpm.PcpmError) as e:
        pcpm.PNG.shard(d_rp, d_col, 1, 0, 1)
    assert e.value.code == -6
    with pytest.raises(pcpm.PcpmError) as e:
        pcpm.dest_partition_counts(d_col, 3, 1)
    assert e.value.code == -6


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist

    import graphgen
    import paper_1709_07122_gb300 as pcpm
    from paper_1709_07122_gb300.sharded import ShardedPageRank

    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    pcpm.lib()
    rp, col = graphgen.rmat(16, 16, seed=1709)
    d_rp, d_col = pcpm.to_device_csr(rp, col)
    solver = ShardedPageRank(d_rp, d_col, 16384)
    x, its, hist = solver.pagerank(D, max_iters=20)
    x20 = x.cpu().numpy()
    x, its_tol, _ = solver.pagerank(D, max_iters=100, tol=1e-7)
    lo, hi = solver.own_nodes
    solver.close()
    dist.destroy_process_group()
    np.save(os.path.join(out_dir, f"x{rank}.npy"), x20)
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"iters": its, "hist": hist.tolist(), "own": [lo, hi], "iters_tol": its_tol}, f)


def test_two_processes_over_gloo_match_the_oracle(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    rp, col = graphgen.rmat(16, 16, seed=1709)
    ref = oracle.pagerank(rp, col, D, iters=20)
    owns = []
    for r in range(world):
        res = json.load(open(tmp_path / f"r{r}.json"))
        x = np.load(tmp_path / f"x{r}.npy")
        assert res["iters"] == 20
        assert l1(x, ref["x"]) <= L1_TOL
        assert np.all(np.abs(np.array(res["hist"]) - ref["resid"]) <= 2 * L1_TOL)
        # a solve to 1e-7 stops where the oracle's L1 change first drops below it
        assert res["iters_tol"] <= 100
        owns.append(res["own"])
    assert owns[0][0] == 0 and owns[0][1] == owns[1][0] and owns[1][1] == rp.size - 1
