"""Destination sharding without a GPU.

* pcpm_shard_split, the host-only cut of the partitions into contiguous
  ranges, against its rule written out by brute force and against the
  properties the sharded solve relies on.
* The per-iteration exchange of the sharded solve (sharded.Exchange) on two
  and three gloo ranks on 127.0.0.1: each rank applies Eq. 1 to its own
  destination range with the FP64 oracle, all-reduces the L1 change and the
  dangling mass and all-gathers the new vector. The result must be the
  oracle's single-process iteration, so a wrong range, a dropped slice or a
  dangling mass from the wrong iteration fails.
"""
import json
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import paper_1709_07122_gb300 as pcpm  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    pcpm.build()
    pcpm.lib()


def brute_split(ids, n, q, nranks):
    """The rule of pcpm_shard_split, exhaustively: cut r is the boundary
    whose prefix weight is nearest r/nranks of the total (ties to the lower),
    clamped so every rank keeps at least one partition."""
    k = len(ids)
    w = [int(ids[p]) + min(q, n - p * q) for p in range(k)]
    pre = [0]
    for x in w:
        pre.append(pre[-1] + x)
    W = pre[-1]
    cuts = [0]
    for r in range(1, nranks):
        # |pre[b] - r W / N| compared exactly as |N pre[b] - r W|
        best = min(range(k + 1), key=lambda b: (abs(nranks * pre[b] - r * W), b))
        cuts.append(min(max(best, cuts[-1] + 1), k - (nranks - r)))
    cuts.append(k)
    return cuts


@pytest.mark.parametrize("seed", range(12))
def test_split_matches_its_rule_and_balances(seed):
    rng = np.random.default_rng(seed)
    q = int(rng.integers(1, 50))
    k = int(rng.integers(1, 40))
    n = (k - 1) * q + int(rng.integers(1, q + 1))  # ragged last partition
    ids = rng.integers(0, 1000, size=k).astype(np.uint64)
    if seed % 3 == 0:
        ids[rng.integers(0, k)] = 10**6  # one hot partition
    for nranks in range(1, k + 1):
        cuts = pcpm.shard_split(ids, n, q, nranks)
        assert list(cuts) == brute_split(ids, n, q, nranks)
        assert cuts[0] == 0 and cuts[-1] == k
        assert np.all(np.diff(cuts.astype(np.int64)) >= 1)  # every rank holds a partition
        w = ids.astype(np.int64) + np.minimum(q, n - np.arange(k) * q)
        loads = [int(w[cuts[r]:cuts[r + 1]].sum()) for r in range(nranks)]
        if nranks == 1:
            assert loads == [int(w.sum())]


def test_split_edge_cases():
    ids = np.zeros(8, np.uint64)  # an edgeless graph splits by nodes
    assert list(pcpm.shard_split(ids, 8 * 16, 16, 4)) == [0, 2, 4, 6, 8]
    assert list(pcpm.shard_split(ids, 8 * 16, 16, 8)) == list(range(9))
    with pytest.raises(pcpm.PcpmError):
        pcpm.shard_split(ids, 8 * 16, 16, 9)  # more ranks than partitions
    with pytest.raises(pcpm.PcpmError):
        pcpm.shard_split(ids, 8 * 16, 16, 0)
    hot = np.array([0, 0, 10**9, 0], np.uint64)  # one partition holds nearly all edges
    cuts = pcpm.shard_split(hot, 4 * 8, 8, 3)
    assert cuts[0] == 0 and cuts[-1] == 4 and np.all(np.diff(cuts.astype(np.int64)) >= 1)
    assert cuts[1] <= 2 < cuts[2]  # the hot partition stays whole in one range


def test_node_bounds():
    from paper_1709_07122_gb300.sharded import node_bounds
    assert node_bounds([0, 2, 5], 70, 16) == [0, 32, 70]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir, dangling):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist

    import graphgen
    import oracle
    from paper_1709_07122_gb300.sharded import Exchange, node_bounds

    dist.init_process_group("gloo", rank=rank, world_size=world)
    # a graph with dangling nodes and a ragged last partition
    rp, col = graphgen.rmat(11, 6, seed=77)
    n, q = rp.size - 1, 160
    k = (n + q - 1) // q
    ids = np.bincount(col // q, minlength=k).astype(np.uint64)
    bounds = node_bounds(pcpm.shard_split(ids, n, q, world), n, q)
    lo, hi = bounds[rank], bounds[rank + 1]
    ex = Exchange(bounds)
    pull = oracle.Pull(rp, col)
    dang = pull.row_ptr[1:] == pull.row_ptr[:-1]
    x = torch.full((n,), 1.0 / n, dtype=torch.float64)
    own = np.zeros(n, bool)
    own[lo:hi] = True
    sums = torch.tensor([0.0, float(x.numpy()[own & dang].sum())], dtype=torch.float64)
    ex.all_reduce_sums(sums)
    hist = []
    for _ in range(20):
        y = torch.zeros(n, dtype=torch.float64)
        dm = float(sums[1]) if dangling == "uniform" else 0.0
        r = pull.step_all(x.numpy(), y.numpy(), 0.85, dangling, 1, lo, hi, dmass=dm)
        sums = torch.tensor([r, float(y.numpy()[own & dang].sum())], dtype=torch.float64)
        ex.all_reduce_sums(sums)
        ex.all_gather_slices(y)
        hist.append(float(sums[0]))
        x = y
    dist.destroy_process_group()
    np.save(os.path.join(out_dir, f"x{rank}.npy"), x.numpy())
    with open(os.path.join(out_dir, f"h{rank}.json"), "w") as f:
        json.dump(hist, f)


@pytest.mark.parametrize("world,dangling", [(2, "uniform"), (3, "uniform"), (2, "leak")])
def test_exchange_reproduces_the_single_process_iteration(tmp_path, world, dangling):
    import graphgen
    import oracle
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path), dangling), nprocs=world,
                       join=True, start_method="spawn")
    rp, col = graphgen.rmat(11, 6, seed=77)
    assert np.any(rp[1:] == rp[:-1])  # the graph has dangling nodes
    ref = oracle.pagerank(rp, col, 0.85, iters=20, dangling=dangling)
    for r in range(world):
        x = np.load(tmp_path / f"x{r}.npy")
        assert np.abs(x - ref["x"]).sum() < 1e-13
        hist = json.load(open(tmp_path / f"h{r}.json"))
        # the same sums up to FP64 reassociation of n terms (relative n * 2^-52)
        # and the last-ulp drift of the vectors (absolute 1e-14)
        ref_r = np.asarray(ref["resid"])
        assert np.all(np.abs(np.array(hist) - ref_r) <= rp.size * 2.0**-52 * ref_r + 1e-14)
