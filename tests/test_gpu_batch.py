"""Batched solves: many independent graphs in one captured CUDA graph launch.

Every handle of the batch ends exactly where pcpm_reset + pcpm_iterate
would leave it: ranks within L1 1e-6 of the FP64 oracle after the batch's
iterations and the L1 change of every iteration within 2e-6 of the oracle's,
for each graph, on every launch of the same batch.

With the window layout, FP32 bins and plain two-phase iterations, each phase
is one launch over the units of all graphs of a part size (2 + 3 iters
kernels per part size, plus the history copy); a handle that does not
qualify (16-bit bins here) sends the batch to per-handle capture. Both are
checked, with mixed part sizes, ragged and tiny graphs, and a history that
grew (moved) between launches."""
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


@pytest.mark.parametrize("mode,dtype", [("two_phase", "f32"), ("fused", "f32"), ("two_phase", "mixed")])
def test_batch_matches_oracle_on_every_graph(mode, dtype):
    graphs = small_graphs(40, seed=5)
    graphs.append((np.array([0, 0], np.uint32), np.zeros(0, np.uint32), 64))  # one node, no edge
    iters = 12
    dts = ["bf16" if (dtype == "mixed" and i == 3) else "f32" for i in range(len(graphs))]
    handles = [pcpm.PNG.from_host(rp, col, q, update_dtype=dt) for (rp, col, q), dt in zip(graphs, dts)]
    refs = [oracle.pagerank(rp, col, 0.85, iters=iters) for rp, col, _ in graphs]
    with pcpm.Batch(handles, 0.85, iters, mode=mode) as b:
        kernels = b.kernel_launches
        if mode == "two_phase" and dtype == "f32":
            groups = {(h.info["part_size"], h.info["gather_cluster"]) for h in handles}
            assert kernels == len(groups) * (2 + 3 * iters) + 1
        else:
            assert kernels >= len(graphs) * (2 + 2 * iters)  # per-handle work
        for launch in range(3):
            b.launch()
            torch.cuda.synchronize()
            for h, ref, dt in zip(handles, refs, dts):
                x = h.ranks().cpu().numpy().astype(np.float64)
                tol = 1e-6 if dt == "f32" else 1e-3
                assert float(np.abs(x - ref["x"]).sum()) <= tol
                hist = h.residual_history()
                assert hist.size == iters
                if dt == "f32":
                    assert np.all(np.abs(hist - np.asarray(ref["resid"])) <= 2e-6)
            # running something else on a handle between launches is fine,
            # also when its history grows (moves) past the batch's capture
            handles[0].reset()
            handles[0].iterate(0.85, 3 if launch == 0 else 1500)
    for h in handles:
        h.close()


def test_batch_rejects_a_handle_twice_and_bad_arguments():
    rp, col = graphgen.rmat(8, 8, seed=1)
    h = pcpm.PNG.from_host(rp, col, 64)
    for args in (([h, h], 0.85, 5), ([h], 1.5, 5), ([h], 0.85, 0)):
        with pytest.raises(pcpm.PcpmError) as e:
            pcpm.Batch(*args)
        assert e.value.code == -1
    h.close()
