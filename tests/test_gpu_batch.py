"""Batched solves: many independent graphs in one captured CUDA graph launch.

Every handle of the batch ends exactly where pcpm_reset + pcpm_iterate
would leave it: ranks within L1 1e-6 of the FP64 oracle after the batch's
iterations, for each graph, on every launch of the same batch."""
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


@pytest.mark.parametrize("mode", ["two_phase", "fused"])
def test_batch_matches_oracle_on_every_graph(mode):
    graphs = small_graphs(40, seed=5)
    iters = 12
    handles = [pcpm.PNG.from_host(rp, col, q) for rp, col, q in graphs]
    refs = [oracle.pagerank(rp, col, 0.85, iters=iters)["x"] for rp, col, _ in graphs]
    with pcpm.Batch(handles, 0.85, iters, mode=mode) as b:
        for launch in range(2):
            b.launch()
            torch.cuda.synchronize()
            for h, ref in zip(handles, refs):
                x = h.ranks().cpu().numpy().astype(np.float64)
                assert float(np.abs(x - ref).sum()) <= 1e-6
                assert h.residual_history().size == iters
            # running something else on a handle between launches is fine
            handles[0].reset()
            handles[0].iterate(0.85, 3)
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
