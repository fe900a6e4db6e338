"""The allocation-free entry point pcpm_rank_stats_noalloc, for callers that
cannot call cudaMalloc (for example code inside an allocator callback or a
process whose device memory is reserved up front). It must give the same L1
change and dangling mass as the solver's own reduction (pcpm_iterate's
residual and the state's dangling mass), call after call, although all calls
share one fixed scratch array in the library.

Kept in a file that pytest collects last, so a stop at the first failure has
already run every other test."""
import ctypes

import numpy as np
import pytest

import graphgen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1709_07122_gb300 as pcpm  # noqa: E402

# The solver sums |x - y| per thread in FP32 over at most 64 nodes before its
# FP64 reduction, so its total is within gamma_64 = 64 * 2^-24 (relative) of the
# FP64 sum this entry point computes; the dangling mass likewise.
RTOL = 64 * 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pcpm.build()
    pcpm.lib()


def noalloc(x, y, row_ptr, out):
    code = pcpm.lib().pcpm_rank_stats_noalloc(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                              ctypes.c_void_p(row_ptr.data_ptr()), row_ptr.numel() - 1,
                                              ctypes.c_void_p(out.data_ptr()), None)
    assert code == 0, pcpm.lib().pcpm_strerror(code)
    torch.cuda.synchronize()
    return out.cpu().numpy().copy()


def test_matches_solver_reduction_on_consecutive_calls():
    rp, col = graphgen.rmat(15, 16, seed=1709)
    d_rp, d_col = pcpm.to_device_csr(rp, col)
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pcpm.PNG(d_rp, d_col, 4096) as g:
        g.reset()
        prev = g.ranks()
        for call in range(2):  # two calls in a row, each against a fresh solver step
            _, res = g.iterate(0.85, 1)
            cur = g.ranks()
            dangling = g.export_state()["dangling"]
            got = noalloc(cur, prev, d_rp, out)
            np.testing.assert_allclose(got[0], res, rtol=RTOL)
            np.testing.assert_allclose(got[1], dangling, rtol=RTOL)
            prev = cur
    # the same call twice gives the same bits: nothing carries over
    again = noalloc(cur, prev, d_rp, out)
    np.testing.assert_array_equal(again, noalloc(cur, prev, d_rp, out))


def test_rejects_inputs_beyond_the_scratch():
    L = pcpm.lib()
    dummy = ctypes.c_void_p(16)  # never dereferenced: the size check comes first
    n = (1 << 16) * 4096 + 1
    assert L.pcpm_rank_stats_noalloc(dummy, dummy, dummy, n, dummy, None) == -7
    assert b"no-allocation" in L.pcpm_strerror(-7)
