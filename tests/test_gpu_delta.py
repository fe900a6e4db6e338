"""Delta iterations (PCPM_DELTA) on the GPU, against the FP64 oracle.

By linearity of Eq. 1, PR_{i+1} = PR_i + d (A^T dSPR + dD / n) with dSPR the
change of SPR since the previous iteration and dD that of the dangling mass.
The bins then carry changes, which shrink as the iteration converges.

* Bins: the stored changes equal, bit for bit, the format (FP32, BF16, or
  FP16 of the change times 2^E, E = floor(log2(65504 / r)), r the last L1
  change) applied to the change of SPR computed on the host in FP32 from the
  exported ranks.
* Steps: each delta step from the GPU's own two last rank vectors matches the
  FP64 delta step from the same vectors within the rounding the formats allow.
  With 16-bit bins each node's stored change also carries what the rounding
  of its previous one left out (error feedback), so a step applies
  dSPR_i + e_{i-1} - e_i, each e within one rounding of its change.
* Solves: run to L1 change 1e-7, the delta form with 16-bit bins ends within
  L1 1e-6 of the FP64 fixed point, the FP32 path's bar, which the plain 16-bit
  forms do not reach.
"""
import numpy as np
import pytest

import graphgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1709_07122_gb300 as pcpm  # noqa: E402

D = 0.85
U32 = 2.0 ** -24
UNIT = {"f32": U32, "f16": 2.0 ** -11, "bf16": 2.0 ** -8}


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pcpm.build()
    pcpm.lib()


GRAPHS = {
    "rmat14_q2048": lambda: (graphgen.rmat(14, 16, seed=41), 2048),
    "rmat12_bfs_q512": lambda: (graphgen.rmat(12, 16, seed=42, relabel="bfs"), 512),
    "random1000_q7": lambda: (graphgen.random_graph(1000, 5000, seed=43), 7),
}


def inv_outdeg(rp):
    deg = np.diff(rp.astype(np.int64))
    inv = np.where(deg > 0, np.float32(1) / np.maximum(deg, 1).astype(np.float32), np.float32(0))
    return inv.astype(np.float32), deg


def f16_exponent(r):
    return 100 if not r > 0 else max(-100, min(100, int(np.floor(np.log2(65504.0 / r)))))


@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_delta_bins_bit_exact(name, dtype):
    (rp, col), q = GRAPHS[name]()
    n = rp.size - 1
    x0 = graphgen.random_rank_vector(n, seed=45).astype(np.float32)
    ref = oracle.png(rp, col, q)
    with pcpm.PNG.from_host(rp, col, q, update_dtype=dtype) as g:
        g.reset(torch.from_numpy(x0).cuda())
        g.iterate(D, 1, mode="two_phase")
        x1 = g.ranks().cpu().numpy()
        r1 = float(g.residual_history()[0])
        g.iterate(D, 1, mode="delta")
        st = g.export_state()
    inv, _ = inv_outdeg(rp)
    change = (x1 - x0) * inv  # FP32, in the kernel's order
    if dtype == "f16":
        change = change * np.float32(2.0 ** (f16_exponent(r1) - 15))
    want = oracle.store_updates(change[ref["src_idx"]], dtype)
    np.testing.assert_array_equal(st["updates"].view(np.uint32 if dtype == "f32" else np.uint16),
                                  want.view(np.uint32 if dtype == "f32" else np.uint16))


def delta_step_fp64(pull, x, xp, dangling_rows):
    """x + d (A^T ((x - xp) / outdeg) + (D(x) - D(xp)) / n) in FP64."""
    n = x.size
    dx = x.astype(np.float64) - xp.astype(np.float64)
    y = np.empty(n)
    pull.step_all(dx, y, 1.0, "leak", 1)  # y = A^T (dx / outdeg)
    dD = float(dx[dangling_rows].sum())
    return x.astype(np.float64) + D * (y + dD / n)


@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("name", ["rmat14_q2048", "rmat12_bfs_q512"])
@pytest.mark.parametrize("opts", [{}, {"gather_windows": 2}, {"gather_unit_chunks": 1, "gather_cluster": 1}],
                         ids=["windows", "chunks", "cut_bins"])
def test_each_delta_step_within_rounding_bound(name, dtype, opts):
    (rp, col), q = GRAPHS[name]()
    n, m = rp.size - 1, int(rp[-1])
    pull = oracle.Pull(rp, col)
    dangling = np.diff(rp) == 0
    with pcpm.PNG.from_host(rp, col, q, update_dtype=dtype, **opts) as g:
        g.reset()
        xp = g.ranks().cpu().numpy()
        g.iterate(D, 1, mode="two_phase")
        x = g.ranks().cpu().numpy()
        r_prev, sub_prev = 0.0, 0.0  # the first delta step carries no earlier rounding
        for i in range(6):
            r = float(np.abs(x.astype(np.float64) - xp.astype(np.float64)).sum())
            g.iterate(D, 1, mode="delta")
            y = g.ranks().cpu().numpy()
            want = delta_step_fp64(pull, x, xp, dangling)
            # Each node's stored change is its change of SPR plus the previous
            # rounding left-over e_{i-1}, rounded: the step applies
            # dSPR + e_{i-1} - e_i, each e within u (of the format) of its
            # change; summed over out-edges: d u (r_i + r_{i-1}) (1.01 for the
            # carried terms). FP16 changes below the normal range: 2^-25 2^-E
            # per edge. FP32 staging and sums: 68 u32 d r_i; the addition to
            # the ranks: 2 u32 sum(y).
            sub = m * 2.0 ** -25 * 2.0 ** -f16_exponent(r) if dtype == "f16" else 0.0
            fb = 0.0 if dtype == "f32" else 1.0  # FP32 bins store changes exactly: no feedback
            bound = (D * UNIT[dtype] * 1.01 * (r + fb * r_prev) + D * 68 * U32 * r + sub + fb * sub_prev
                     + 2 * U32 * float(np.abs(want).sum()) + 1e-12)
            err = float(np.abs(y.astype(np.float64) - want).sum())
            assert err <= bound, (i, err, bound)
            xp, x = x, y
            r_prev, sub_prev = r, sub


@pytest.mark.parametrize("dtype", ["f16", "bf16", "f32"])
@pytest.mark.parametrize("name", ["rmat14_q2048", "rmat12_bfs_q512", "random1000_q7"])
def test_delta_solve_reaches_fp32_accuracy(name, dtype):
    # The plain 16-bit forms stop near the rounding of SPR itself (their L1
    # distance to the FP64 fixed point stays around 1e-4); the delta form with
    # error feedback reaches L1 change 1e-7 and the FP32 path's 1e-6 bar. It
    # needs more iterations than FP32: what the roundings leave in the slowest
    # modes of the changes (their total mass among them) decays only at rate d.
    (rp, col), q = GRAPHS[name]()
    tol = 1e-7
    with pcpm.PNG.from_host(rp, col, q, update_dtype=dtype) as g:
        x, it, res = g.pagerank(D, max_iters=300, tol=tol, mode="delta")
        x = x.cpu().numpy().astype(np.float64)
    assert res < tol and it < 300, (it, res)
    ref = oracle.pagerank(rp, col, D, iters=400)["x"]
    err = float(np.abs(x - ref).sum())
    assert err <= 1e-6, err
