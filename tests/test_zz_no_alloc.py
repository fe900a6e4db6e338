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

# The solver's apply adds |x - y| per thread in FP32 over at most 8 nodes at
# q = 4096 (768 threads per CTA, four nodes per 16-byte group) before its FP64
# reduction, so its total is within gamma_8 = 8 * 2^-24 (relative) of the FP64
# sum this entry point computes; the dangling mass likewise. 64 * 2^-24 leaves
# room for that.
RTOL = 64 * 2.0 ** -24
# Against numpy's FP64 sums of the same FP32 inputs: only the order of FP64
# additions differs.
EXACT_RTOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pcpm.build()
    pcpm.lib()


def noalloc(x, y, row_ptr, out, stream=None):
    code = pcpm.lib().pcpm_rank_stats_noalloc(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                              ctypes.c_void_p(row_ptr.data_ptr()), row_ptr.numel() - 1,
                                              ctypes.c_void_p(out.data_ptr()),
                                              None if stream is None else ctypes.c_void_p(stream.cuda_stream))
    assert code == 0, pcpm.lib().pcpm_strerror(code)
    torch.cuda.synchronize()
    return out.cpu().numpy().copy()


def dangling_csr(n, seed):
    """A CSR of n nodes where about a third of the nodes have no out-edges."""
    rng = np.random.default_rng(seed)
    deg = rng.integers(0, 4, size=n)
    deg[rng.random(n) < 0.33] = 0
    row_ptr = np.zeros(n + 1, np.uint32)
    row_ptr[1:] = np.cumsum(deg)
    col = np.concatenate([np.sort(rng.choice(n, size=min(int(d), n), replace=False)) for d in deg]
                         + [np.zeros(0, np.int64)]).astype(np.uint32)
    return row_ptr, col


@pytest.mark.parametrize("n", [1, 4095, 4096, 3 * 4096 + 17])
def test_exact_sums_on_ragged_sizes(n):
    # n = 1 and 4095: one block; 3 * 4096 + 17: a clamped last block
    rp, col = dangling_csr(n, seed=n)
    d_rp, _ = pcpm.to_device_csr(rp, col)
    rng = np.random.default_rng(7 + n)
    x = rng.random(n).astype(np.float32)
    y = rng.random(n).astype(np.float32)
    want_l1 = np.abs(x.astype(np.float64) - y.astype(np.float64)).sum()
    want_dg = x.astype(np.float64)[rp[1:] == rp[:-1]].sum()
    dx, dy = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    side = torch.cuda.Stream()
    for stream in (None, side):  # the default stream, then a caller's stream
        got = noalloc(dx, dy, d_rp, out, stream)
        np.testing.assert_allclose(got[0], want_l1, rtol=EXACT_RTOL)
        np.testing.assert_allclose(got[1], want_dg, rtol=EXACT_RTOL, atol=0 if want_dg else 1e-300)


def test_wrapper_with_preallocated_out():
    # callers that cannot allocate pass `out`; the wrapper then allocates nothing
    rp, col = dangling_csr(5000, seed=3)
    d_rp, _ = pcpm.to_device_csr(rp, col)
    rng = np.random.default_rng(11)
    x = rng.random(5000).astype(np.float32)
    y = rng.random(5000).astype(np.float32)
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    ret = pcpm.rank_stats_noalloc(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), d_rp, out=out)
    assert ret.data_ptr() == out.data_ptr()
    torch.cuda.synchronize()
    np.testing.assert_allclose(out.cpu().numpy()[0], np.abs(x.astype(np.float64) - y).sum(), rtol=EXACT_RTOL)
    np.testing.assert_allclose(out.cpu().numpy()[1], x.astype(np.float64)[rp[1:] == rp[:-1]].sum(), rtol=EXACT_RTOL)


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
