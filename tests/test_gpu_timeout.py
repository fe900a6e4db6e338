"""Bounded device-side waits, exercised without a fault.

The window-layout gather waits on mbarriers for its ring stages. A test hook
(pcpm_test_wait_limit) makes those waits for work give up at once, as if the
copies they wait for never completed. The call must return PCPM_ETIMEOUT (no
trap, no hang: the copies already in flight are still drained with the
normal bound before each CTA exits), and the same handle must then solve
normally and match the FP64 oracle.
"""
import numpy as np
import pytest

import graphgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1709_07122_gb300 as pcpm  # noqa: E402

PCPM_ETIMEOUT = -4


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pcpm.build()
    pcpm.lib()


@pytest.mark.parametrize("mode", ["two_phase", "fused"])
def test_wait_that_runs_out_reports_timeout_and_the_handle_recovers(mode):
    rp, col = graphgen.rmat(16, 16, seed=1709)
    ref = oracle.pagerank(rp, col, 0.85, iters=6)["x"]
    L = pcpm.lib()
    with pcpm.PNG.from_host(rp, col, 16384) as g:
        assert g.info["gather_windows"] == 1
        g.reset()
        assert L.pcpm_test_wait_limit(-1) == 0
        try:
            with pytest.raises(pcpm.PcpmError) as e:
                g.iterate(0.85, 2, mode=mode)
            assert e.value.code == PCPM_ETIMEOUT
        finally:
            assert L.pcpm_test_wait_limit(0) == 0
        torch.cuda.synchronize()  # the context is intact
        pr, its, _ = g.pagerank(0.85, max_iters=6, mode=mode)
        assert its == 6
        assert float(np.abs(pr.cpu().numpy().astype(np.float64) - ref).sum()) <= 1e-6
        # the status of the failed call does not stick to later solves
        g.sync_status()
