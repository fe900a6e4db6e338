"""Destination-sharded PCPM PageRank: one process per GPU.

Every destination partition is gathered and applied on its own (Sec. 3.1:
bin p' holds every update into partition p', and Algorithm 4 reads only that
bin), so the partitions split across ranks with no change to the method.
Rank r builds the bins of a contiguous range of destination partitions
(``pcpm_build_shard``), balanced by destination IDs plus nodes
(``pcpm_shard_split`` over ``pcpm_dest_partition_counts``), and owns the ranks
of their nodes. Its scatter (Algorithm 3) reads the ranks of every source, so
each iteration ends with one exchange:

* an all-reduce (sum) of two FP64 values, the L1 change and the dangling mass
  of the rank's own nodes, which gives the next iteration the whole graph's
  dangling mass and the caller the whole L1 change;
* an all-gather of the new rank vector: rank r broadcasts its own slice.

Everything here is orchestration: the library's kernels compute every value;
``torch.distributed`` moves them (NCCL between GPUs; any other backend, such
as gloo, through host copies). Kernels never wait on another GPU and never
read another GPU's memory.
"""
from __future__ import annotations

import numpy as np

from . import PNG, dest_partition_counts, shard_split


class Exchange:
    """The per-iteration exchange of a destination-sharded solve.

    node_bounds: the nodes each rank owns, rank r owning
    [node_bounds[r], node_bounds[r + 1]). Works on CUDA or CPU tensors; with
    a backend other than NCCL, CUDA tensors are staged through host memory."""

    def __init__(self, node_bounds, group=None, staged: bool | None = None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.bounds = [int(b) for b in node_bounds]
        if len(self.bounds) != self.world + 1:
            raise ValueError("node_bounds needs world_size + 1 entries")
        self.staged = (dist.get_backend(group) != "nccl") if staged is None else staged

    def _global_rank(self, r: int) -> int:
        return r if self.group is None else self.dist.get_global_rank(self.group, r)

    def all_reduce_sums(self, sums) -> None:
        """sums (float64 [2]) becomes the sum over ranks, in place."""
        if self.staged and sums.is_cuda:
            h = sums.cpu()
            self.dist.all_reduce(h, group=self.group)
            sums.copy_(h)
        else:
            self.dist.all_reduce(sums, group=self.group)

    def all_gather_slices(self, pr) -> None:
        """Every rank's own slice of pr (float32 [n]) reaches every rank."""
        for r in range(self.world):
            lo, hi = self.bounds[r], self.bounds[r + 1]
            if hi == lo:
                continue
            view = pr[lo:hi]
            if self.staged and pr.is_cuda:
                h = view.cpu() if r == self.rank else view.new_empty(hi - lo, device="cpu")
                self.dist.broadcast(h, src=self._global_rank(r), group=self.group)
                if r != self.rank:
                    view.copy_(h)
            else:
                self.dist.broadcast(view, src=self._global_rank(r), group=self.group)


def node_bounds(part_bounds, n: int, part_size: int) -> list[int]:
    """Owned node ranges of destination-partition cut points."""
    return [min(int(b) * part_size, n) for b in part_bounds]


class ShardedPageRank:
    """PCPM PageRank of one graph over the ranks of a process group.

    Every rank passes the same device CSR (row_ptr, col: CUDA 32-bit integer
    tensors, rows sorted) and part size; each builds only its own shard."""

    def __init__(self, row_ptr, col, part_size: int, group=None, stream=None, **options):
        import torch
        import torch.distributed as dist
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        n = row_ptr.numel() - 1
        self.n, self.part_size = n, part_size
        m = int(row_ptr[-1].item()) & 0xFFFFFFFF
        counts = dest_partition_counts(col, n, part_size, m, stream)
        self.part_bounds = shard_split(counts, n, part_size, self.world)
        self.node_bounds = node_bounds(self.part_bounds, n, part_size)
        lo, hi = int(self.part_bounds[self.rank]), int(self.part_bounds[self.rank + 1])
        self.png = PNG.shard(row_ptr, col, part_size, lo, hi, stream, **options)
        self.exchange = Exchange(self.node_bounds, group)
        self.pr = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(2)]
        self.sums = torch.zeros(2, dtype=torch.float64, device="cuda")
        self.cur = 0
        self.stream = stream

    @property
    def own_nodes(self) -> tuple[int, int]:
        return self.node_bounds[self.rank], self.node_bounds[self.rank + 1]

    def reset(self, pr_init=None) -> None:
        """PR_0 = pr_init (CUDA float32 [n], the same on every rank) or 1/n."""
        self.cur = 0
        self.png.shard_init(self.pr[0], self.sums, pr_init, self.stream)
        self.exchange.all_reduce_sums(self.sums)

    def step(self, d: float = 0.85, dangling: str = "uniform") -> None:
        """One iteration: own nodes in the kernels, then the exchange."""
        nxt = self.pr[self.cur ^ 1]
        self.png.shard_step(self.pr[self.cur], nxt, self.sums, d, dangling, self.stream)
        self.exchange.all_reduce_sums(self.sums)
        self.exchange.all_gather_slices(nxt)
        self.cur ^= 1

    @property
    def ranks(self):
        """The current rank vector (all n nodes, identical on every rank)."""
        return self.pr[self.cur]

    def pagerank(self, d: float = 0.85, max_iters: int = 20, tol: float = 0.0, pr_init=None,
                 dangling: str = "uniform"):
        """Returns (ranks tensor, iterations run, FP64 L1 changes per
        iteration as a numpy array). tol > 0 stops after the first iteration
        whose whole-graph L1 change is below tol (one host read per iteration)."""
        import torch
        self.reset(pr_init)
        hist = torch.empty(max(max_iters, 1), dtype=torch.float64, device="cuda")
        done = 0
        for i in range(max_iters):
            self.step(d, dangling)
            hist[i].copy_(self.sums[0])
            done = i + 1
            if tol > 0 and float(self.sums[0].item()) < tol:
                break
        self.png.sync_status()
        return self.ranks, done, hist[:done].cpu().numpy().astype(np.float64)

    def close(self) -> None:
        self.png.close()
