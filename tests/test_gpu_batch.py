"""Batched solves: many independent graphs in one captured CUDA graph launch.

Every handle of the batch ends exactly where pcpm_reset + pcpm_iterate
would leave it: ranks within L1 1e-6 of the FP64 oracle after the batch's
iterations and the L1 change of every iteration within 2e-6 of the oracle's,
for each graph, on every launch of the same batch.

With the window layout, each phase is one launch over the units of all
graphs of a (part size, cluster size, bin format) group: 2 + 3 iters kernels
per group for two-phase iterations, 3 + 2 iters for fused ones, plus the
history copy. A handle with another layout (the chunk layout here) sends the
batch to per-handle capture. Both are checked, with mixed part sizes and bin
formats, ragged and tiny graphs, and a history that grew (moved) between
launches; every handle also ends within L1 1e-6 of its own reset and
iterations."""
import numpy as np
import pytest

import graphgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1709_07122_gb300 as pcpm  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pcpm.build()
    pcpm.lib()


def small_graphs(count, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        s = int(rng.integers(6, 12))
        rp, col = graphgen.rmat(s, 8, seed=seed * 100 + i, relabel=str(rng.choice(["random", "bfs"])))
        q = int(rng.choice([64, 512, 4096, 32768]))
        out.append((rp, col, q))
    return out


def handle_options(mode, kind, i):
    # fused iterations need whole bins per gather unit: units large enough
    # that no bin of these graphs is cut
    o = {"gather_unit_chunks": 1 << 20} if mode == "fused" else {}
    if kind == "mixed" and i == 3:
        o["update_dtype"] = "bf16"
    if kind == "mixed" and i == 5:
        o["update_dtype"] = "f16"
    if kind == "chunks" and i == 2:
        o["gather_windows"] = 2  # the chunk layout: per-handle capture
    return o


@pytest.mark.parametrize("mode,kind", [("two_phase", "f32"), ("fused", "f32"), ("two_phase", "mixed"),
                                       ("fused", "mixed"), ("two_phase", "chunks")])
def test_batch_matches_oracle_on_every_graph(mode, kind):
    graphs = small_graphs(40, seed=5)
    graphs.append((np.array([0, 0], np.uint32), np.zeros(0, np.uint32), 64))  # one node, no edge
    iters = 12
    opts = [handle_options(mode, kind, i) for i in range(len(graphs))]
    handles = [pcpm.PNG.from_host(rp, col, q, **o) for (rp, col, q), o in zip(graphs, opts)]
    refs = [oracle.pagerank(rp, col, 0.85, iters=iters) for rp, col, _ in graphs]
    exact = [o.get("update_dtype", "f32") == "f32" for o in opts]
    infos = [h.info for h in handles]
    if mode == "fused":
        assert all(i["fused_ok"] for i in infos)
    one_launch = all(i["gather_windows"] == 1 for i in infos)
    with pcpm.Batch(handles, 0.85, iters, mode=mode) as b:
        kernels = b.kernel_launches
        if one_launch:
            groups = {(i["part_size"], i["gather_cluster"], i["update_dtype"]) for i in infos}
            per_group = 2 + 3 * iters if mode == "two_phase" else 3 + 2 * iters
            assert kernels == len(groups) * per_group + 1
        else:
            assert kind == "chunks"
            assert kernels >= len(graphs) * (2 + 2 * iters)  # per-handle work
        for launch in range(3):
            b.launch()
            torch.cuda.synchronize()
            got = [h.ranks().cpu().numpy().astype(np.float64) for h in handles]
            for h, x, ref, ex in zip(handles, got, refs, exact):
                assert float(np.abs(x - ref["x"]).sum()) <= (1e-6 if ex else 1e-3)
                hist = h.residual_history()
                assert hist.size == iters
                if ex:
                    assert np.all(np.abs(hist - np.asarray(ref["resid"])) <= 2e-6)
            # running something else on a handle between launches is fine,
            # also when its history grows (moves) past the batch's capture
            handles[0].reset()
            handles[0].iterate(0.85, 3 if launch == 0 else 1500)
    # every handle, 16-bit bins included, ends where its own reset and
    # iterations leave it
    for h, x in zip(handles, got):
        h.reset()
        h.iterate(0.85, iters, mode=mode)
        assert float(np.abs(h.ranks().cpu().numpy().astype(np.float64) - x).sum()) <= 1e-6
        h.close()


def test_batch_rejects_a_handle_twice_and_bad_arguments():
    rp, col = graphgen.rmat(8, 8, seed=1)
    h = pcpm.PNG.from_host(rp, col, 64)
    for args in (([h, h], 0.85, 5), ([h], 1.5, 5), ([h], 0.85, 0)):
        with pytest.raises(pcpm.PcpmError) as e:
            pcpm.Batch(*args)
        assert e.value.code == -1
    h.close()
