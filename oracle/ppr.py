"""FP64 reference of batched personalized PageRank (test infrastructure only).

Not in the paper's experiments: the paper computes one PageRank vector (Eq. 1).
Personalized PageRank replaces its uniform teleport (1 - d)/|V| with a
per-column teleport distribution t_j; c columns are iterated together as an
[n, c] block, so the scatter-gather of Eq. 2 becomes a sparse-times-dense
product. Reading: the mass of dangling nodes returns to t_j (the column's own
teleport distribution), so every column keeps summing to 1:

    R'[:, j] = (1 - d) * t_j + d * (A^T (R[:, j] * w) + D_j * t_j)
    w(u) = 1 / |N_o(u)|  (0 for dangling u),   D_j = sum over dangling u of R[u, j]

Column j of the teleport block is uniform over its seed nodes S_j (distinct).
The iteration starts from R = T. Only the tests and the benchmark may import
this module; it shares no code with the CUDA path.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def teleport(n: int, seed_ptr, seed_idx) -> np.ndarray:
    """Dense [n, c] FP64 teleport block: column j uniform over seeds
    seed_idx[seed_ptr[j]:seed_ptr[j+1]]."""
    seed_ptr = np.asarray(seed_ptr, dtype=np.int64)
    seed_idx = np.asarray(seed_idx, dtype=np.int64)
    c = seed_ptr.size - 1
    t = np.zeros((n, c), dtype=np.float64)
    for j in range(c):
        s = seed_idx[seed_ptr[j]:seed_ptr[j + 1]]
        if s.size == 0:
            raise ValueError("every column needs at least one seed")
        if np.unique(s).size != s.size or s.min() < 0 or s.max() >= n:
            raise ValueError("seeds of a column must be distinct node IDs")
        t[s, j] = 1.0 / s.size
    return t


def step(row_ptr, col, r, t, d: float) -> np.ndarray:
    """One iteration of the block recurrence above, in FP64."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    n = row_ptr.size - 1
    outdeg = np.diff(row_ptr)
    w = np.where(outdeg > 0, 1.0 / np.maximum(outdeg, 1), 0.0)
    a = sp.csr_matrix((np.ones(col.size), col, row_ptr), shape=(n, n))  # row u: out-edges u -> v
    spr = r * w[:, None]
    y = a.T @ spr  # y[v] = sum over in-edges (u, v) of spr[u]
    dang = r[outdeg == 0].sum(axis=0)
    return (1.0 - d) * t + d * (y + t * dang[None, :])


def ppr(row_ptr, col, seed_ptr, seed_idx, d: float = 0.85, iters: int = 20, history: bool = False):
    """Iterates from R = T. Returns a dict with ``r`` ([n, c] FP64), ``resid``
    ([iters, c]: L1 change of each column per iteration) and, if ``history``,
    ``hist`` ([iters+1, n, c])."""
    n = np.asarray(row_ptr).size - 1
    t = teleport(n, seed_ptr, seed_idx)
    r = t.copy()
    resid = np.zeros((iters, t.shape[1]))
    hist = [r.copy()] if history else None
    for i in range(iters):
        r2 = step(row_ptr, col, r, t, d)
        resid[i] = np.abs(r2 - r).sum(axis=0)
        r = r2
        if history:
            hist.append(r.copy())
    out = {"r": r, "resid": resid}
    if history:
        out["hist"] = np.stack(hist)
    return out


def fixed_point(row_ptr, col, seed_ptr, seed_idx, d: float = 0.85) -> np.ndarray:
    """The exact fixed point by a dense linear solve, per column:
    (I - d (A^T W + t_j 1_dangling^T)) r_j = (1 - d) t_j. Small graphs only."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    n = row_ptr.size - 1
    t = teleport(n, seed_ptr, seed_idx)
    outdeg = np.diff(row_ptr)
    m = np.zeros((n, n))
    for u in range(n):
        for v in col[row_ptr[u]:row_ptr[u + 1]]:
            m[v, u] += 1.0 / outdeg[u]
    dang = (outdeg == 0).astype(np.float64)
    r = np.empty_like(t)
    for j in range(t.shape[1]):
        mj = m + np.outer(t[:, j], dang)
        r[:, j] = np.linalg.solve(np.eye(n) - d * mj, (1.0 - d) * t[:, j])
    return r
