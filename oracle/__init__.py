"""FP64 CPU oracle for PCPM PageRank (arXiv 1709.07122).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference arm may import this; the product path
(``paper_1709_07122_gb300``) never does, and this package never imports it.

The arithmetic lives in ``pcpm_oracle.c`` (plain sequential C, FP64), compiled
with gcc on first use; this file only marshals numpy arrays. Functions and the
passages they follow:

* :func:`pagerank` - Eq. 1 / Algorithm 1 (pull direction), plus the dangling
  reading (uniform redistribution by default, or leak).
* :class:`Pull` - the same step over a range of destination nodes, with the
  in-neighbour lists built once (used to time bounded samples).
* :func:`png` - Partition-Node Graph of Sec. 3.3: per (source partition,
  destination partition) update and edge counts, the write offsets of Sec. 3.1,
  and the bins in canonical order (source partitions in ID order, nodes in ID
  order, destination IDs in adjacency order; MSB marks a message's first ID).
* :func:`scatter_gather` - Algorithm 3 followed by Algorithm 4 in FP64.
* :func:`bin_weights`, :func:`spmv`, :func:`weighted_scatter_gather` -
  weighted graphs and SpMV (Sec. 3.5): weights stored beside the destination
  IDs in bin order; y = A^T_w x by its definition and through the bins.
* :func:`store_updates` / :func:`load_updates` - the storage formats of
  reduced-precision update bins. Not in the paper (it keeps 4-byte updates,
  Sec. 3.2): IEEE 754 binary16 of SPR * 2^15 and bfloat16 (binary32's upper
  16 bits), both rounded to nearest, ties to even.

Parity of :func:`pagerank` is pinned by closed forms, a dense linear solve and
invariants; :func:`png` by brute-force enumeration and the paper's offset
example; :func:`scatter_gather` by a dense matrix product (see tests/).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pcpm_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_pcpm_oracle.so")
_lib = None
_lock = threading.Lock()

_u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compiles pcpm_oracle.c into a shared library next to it."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread", "-o", tmp, _SRC, "-lm"],
                       check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            vp = ctypes.c_void_p
            lib.oracle_pagerank.argtypes = [ctypes.c_uint32, _u32p, _u32p, ctypes.c_double, ctypes.c_int,
                                            ctypes.c_int, vp, vp, vp, vp]
            lib.oracle_pagerank.restype = ctypes.c_int
            lib.oracle_pagerank_mt.argtypes = [ctypes.c_uint32, _u32p, _u32p, ctypes.c_double, ctypes.c_int,
                                               ctypes.c_int, vp, vp, vp, vp, ctypes.c_int]
            lib.oracle_pagerank_mt.restype = ctypes.c_int
            lib.oracle_pull_step_mt.argtypes = [ctypes.c_uint32, _u32p, _u32p, _u32p, ctypes.c_double,
                                                ctypes.c_double, ctypes.c_uint32, ctypes.c_uint32, _f64p, _f64p,
                                                ctypes.c_int]
            lib.oracle_pull_step_mt.restype = ctypes.c_double
            lib.oracle_in_adjacency.argtypes = [ctypes.c_uint32, _u32p, _u32p, _u32p, _u32p]
            lib.oracle_in_adjacency.restype = None
            lib.oracle_dangling_mass.argtypes = [ctypes.c_uint32, _u32p, _f64p]
            lib.oracle_dangling_mass.restype = ctypes.c_double
            lib.oracle_pull_step.argtypes = [ctypes.c_uint32, _u32p, _u32p, _u32p, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_uint32, ctypes.c_uint32, _f64p, _f64p]
            lib.oracle_pull_step.restype = ctypes.c_double
            lib.oracle_png_count.argtypes = [ctypes.c_uint32, _u32p, _u32p, ctypes.c_uint32, _u32p, _u32p]
            lib.oracle_png_count.restype = None
            lib.oracle_png_fill.argtypes = [ctypes.c_uint32, _u32p, _u32p, ctypes.c_uint32, _u32p, _u32p,
                                            _u32p, _u32p, _u32p, _u32p, _u32p, _u32p]
            lib.oracle_png_fill.restype = None
            lib.oracle_png_fill_weights.argtypes = [ctypes.c_uint32, _u32p, _u32p, ctypes.c_uint32, _u32p, _u32p,
                                                    _f64p, _f64p]
            lib.oracle_png_fill_weights.restype = None
            lib.oracle_spmv.argtypes = [ctypes.c_uint32, _u32p, _u32p, _f64p, _f64p, _f64p]
            lib.oracle_spmv.restype = None
            lib.oracle_spmv_rect.argtypes = [ctypes.c_uint32, ctypes.c_uint32, _u32p, _u32p, _f64p, _f64p, _f64p]
            lib.oracle_spmv_rect.restype = None
            lib.oracle_weighted_gather.argtypes = [ctypes.c_uint32, ctypes.c_uint32, _u32p, _u32p, _u32p, _u32p,
                                                   _f64p, _f64p, _f64p]
            lib.oracle_weighted_gather.restype = None
            lib.oracle_scatter_gather.argtypes = [ctypes.c_uint32, ctypes.c_uint32, _u32p, _u32p, _u32p, _u32p,
                                                  _f64p, _f64p]
            lib.oracle_scatter_gather.restype = None
            _lib = lib
    return _lib


def _csr(row_ptr, col):
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.uint32)
    col = np.ascontiguousarray(col, dtype=np.uint32)
    if col.size == 0:
        col = np.zeros(1, dtype=np.uint32)  # valid pointer; row_ptr[n] = 0 says no edges
    return row_ptr, col


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def host_threads() -> int:
    """Host threads the oracle uses when asked for all cores."""
    return max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1))


def pagerank(row_ptr, col, d: float = 0.85, iters: int = 20, x0=None, dangling: str = "uniform",
             history: bool = False, threads: int = 1):
    """Iterates Eq. 1 ``iters`` times from ``x0`` (uniform 1/n if None).

    Returns a dict with ``x`` (final vector), ``resid`` (L1 change per
    iteration) and, if ``history``, ``hist`` of shape (iters+1, n). With
    ``threads`` > 1 each step runs on that many threads over contiguous
    destination ranges: the same vectors, residuals up to FP64 reassociation."""
    if dangling not in ("uniform", "leak"):
        raise ValueError("dangling must be 'uniform' or 'leak'")
    lib = _load()
    row_ptr, col = _csr(row_ptr, col)
    n = row_ptr.size - 1
    x0a = None if x0 is None else np.ascontiguousarray(x0, dtype=np.float64)
    if x0a is not None and x0a.size != n:
        raise ValueError("x0 has the wrong length")
    hist = np.empty((iters + 1, n), dtype=np.float64) if history else None
    x = np.empty(n, dtype=np.float64)
    resid = np.empty(max(iters, 1), dtype=np.float64)
    rc = lib.oracle_pagerank_mt(n, row_ptr, col, float(d), 1 if dangling == "uniform" else 0, int(iters),
                                _ptr(x0a), _ptr(hist), _ptr(x), _ptr(resid), int(threads))
    if rc != 0:
        raise MemoryError("oracle_pagerank could not allocate")
    out = {"x": x, "resid": resid[:iters]}
    if history:
        out["hist"] = hist
    return out


class Pull:
    """In-neighbour lists of a graph, for single Eq. 1 steps over node ranges."""

    def __init__(self, row_ptr, col):
        lib = _load()
        self.row_ptr, self.col = _csr(row_ptr, col)
        self.n = self.row_ptr.size - 1
        m = int(self.row_ptr[self.n])
        self.in_start = np.empty(self.n + 1, dtype=np.uint32)
        self.in_src = np.empty(max(m, 1), dtype=np.uint32)
        lib.oracle_in_adjacency(self.n, self.row_ptr, self.col, self.in_start, self.in_src)

    def in_edges(self, v_begin: int, v_end: int) -> int:
        return int(self.in_start[v_end]) - int(self.in_start[v_begin])

    def dangling_mass(self, x) -> float:
        return _load().oracle_dangling_mass(self.n, self.row_ptr, np.ascontiguousarray(x, dtype=np.float64))

    def step(self, x, y, d: float = 0.85, dangling: str = "uniform", v_begin: int = 0, v_end=None) -> float:
        """y[v] = Eq. 1 applied to x for v in [v_begin, v_end); returns the L1
        change over that range. x and y are float64 arrays of length n."""
        lib = _load()
        v_end = self.n if v_end is None else v_end
        dmass = self.dangling_mass(x) if dangling == "uniform" else 0.0
        return lib.oracle_pull_step(self.n, self.row_ptr, self.in_start, self.in_src, float(d), dmass,
                                    int(v_begin), int(v_end), x, y)

    def step_all(self, x, y, d: float = 0.85, dangling: str = "uniform", threads: int = 1, v_begin: int = 0,
                 v_end=None, dmass=None) -> float:
        """y[v] = Eq. 1 applied to x for v in [v_begin, v_end) (all nodes by
        default) on ``threads`` threads over contiguous pieces of the range;
        returns the L1 change over it. ``dmass``: the dangling mass of x, if
        already known."""
        v_end = self.n if v_end is None else v_end
        if dmass is None:
            dmass = self.dangling_mass(x) if dangling == "uniform" else 0.0
        return _load().oracle_pull_step_mt(self.n, self.row_ptr, self.in_start, self.in_src, float(d), float(dmass),
                                           int(v_begin), int(v_end), x, y, int(threads))


def png(row_ptr, col, q: int):
    """Partition-Node Graph for partition size ``q`` (nodes per partition)."""
    lib = _load()
    row_ptr, col = _csr(row_ptr, col)
    n = row_ptr.size - 1
    k = (n + q - 1) // q
    cnt_u = np.empty(k * k, dtype=np.uint32)
    cnt_e = np.empty(k * k, dtype=np.uint32)
    lib.oracle_png_count(n, row_ptr, col, int(q), cnt_u, cnt_e)
    ne = int(cnt_u.sum(dtype=np.uint64))
    m = int(row_ptr[n])
    off_u = np.empty(k * k, dtype=np.uint32)
    off_e = np.empty(k * k, dtype=np.uint32)
    bin_u = np.empty(k + 1, dtype=np.uint32)
    bin_e = np.empty(k + 1, dtype=np.uint32)
    src_idx = np.empty(max(ne, 1), dtype=np.uint32)
    dest_ids = np.empty(max(m, 1), dtype=np.uint32)
    lib.oracle_png_fill(n, row_ptr, col, int(q), cnt_u, cnt_e, off_u, off_e, bin_u, bin_e, src_idx, dest_ids)
    return {
        "n": n, "q": int(q), "k": k, "m": m, "ne": ne,
        "cnt_u": cnt_u.reshape(k, k), "cnt_e": cnt_e.reshape(k, k),
        "off_u": off_u.reshape(k, k), "off_e": off_e.reshape(k, k),
        "bin_u": bin_u, "bin_e": bin_e,
        "src_idx": src_idx[:ne], "dest_ids": dest_ids[:m],
    }


def scatter_gather(g: dict, spr) -> np.ndarray:
    """Algorithm 3 + Algorithm 4 in FP64 over the bins of :func:`png`:
    returns y[v] = sum of spr[u] over in-neighbours u of v."""
    lib = _load()
    spr = np.ascontiguousarray(spr, dtype=np.float64)
    y = np.empty(g["n"], dtype=np.float64)
    src = g["src_idx"] if g["ne"] else np.zeros(1, dtype=np.uint32)
    dst = g["dest_ids"] if g["m"] else np.zeros(1, dtype=np.uint32)
    lib.oracle_scatter_gather(g["n"], g["k"], g["bin_u"], g["bin_e"], np.ascontiguousarray(src),
                              np.ascontiguousarray(dst), spr, y)
    return y


# ------------------------------------------------------------------ formats
F16_SCALE_LOG2 = 15
_F16_MAX = 65504.0


def store_updates(values_f32, dtype: str) -> np.ndarray:
    """Stored form of FP32 update values. f32: unchanged. f16: binary16 of
    value * 2^15 (an exact power-of-two scaling), rounded to nearest even,
    saturating at +-the largest finite half (numpy's float32 -> float16 cast
    rounds to nearest even). bf16: the 16-bit pattern of binary32 rounded to
    nearest even at bit 16, returned as uint16."""
    v = np.ascontiguousarray(values_f32, dtype=np.float32)
    if dtype == "f32":
        return v.copy()
    if dtype == "f16":
        scaled = v * np.float32(2.0 ** F16_SCALE_LOG2)
        return np.clip(scaled, np.float32(-_F16_MAX), np.float32(_F16_MAX)).astype(np.float16)
    if dtype == "bf16":
        bits = v.view(np.uint32).astype(np.uint64)
        # round to nearest, ties to even: add 0x7FFF plus the lowest kept bit
        rounded = (bits + 0x7FFF + ((bits >> 16) & 1)) >> 16
        return rounded.astype(np.uint16)
    raise ValueError("dtype must be f32, f16 or bf16")


def load_updates(stored, dtype: str) -> np.ndarray:
    """FP64 values of stored updates (inverse of the format, scale removed)."""
    if dtype == "f32":
        return np.asarray(stored, dtype=np.float64)
    if dtype == "f16":
        return np.asarray(stored, dtype=np.float16).astype(np.float64) * 2.0 ** -F16_SCALE_LOG2
    if dtype == "bf16":
        bits = np.asarray(stored, dtype=np.uint16).astype(np.uint32) << 16
        return bits.view(np.float32).astype(np.float64)
    raise ValueError("dtype must be f32, f16 or bf16")


def bin_weights(row_ptr, col, q: int, weights, g: dict | None = None) -> np.ndarray:
    """Edge weights (CSR order) placed beside their destination IDs in bin
    order (Sec. 3.5)."""
    lib = _load()
    row_ptr, col = _csr(row_ptr, col)
    g = png(row_ptr, col, q) if g is None else g
    w = np.ascontiguousarray(weights, dtype=np.float64)
    out = np.empty(max(g["m"], 1), dtype=np.float64)
    off_e = np.ascontiguousarray(g["off_e"].ravel())
    lib.oracle_png_fill_weights(g["n"], row_ptr, col, int(q), off_e, g["bin_e"], w if w.size else np.zeros(1), out)
    return out[:g["m"]]


def spmv(row_ptr, col, weights, x) -> np.ndarray:
    """y(v) = sum over edges (u, v) of w(u, v) * x(u), FP64."""
    lib = _load()
    row_ptr, col = _csr(row_ptr, col)
    n = row_ptr.size - 1
    w = np.ascontiguousarray(weights, dtype=np.float64)
    y = np.empty(n, dtype=np.float64)
    lib.oracle_spmv(n, row_ptr, col if col.size else np.zeros(1, np.uint32), w if w.size else np.zeros(1),
                    np.ascontiguousarray(x, dtype=np.float64), y)
    return y


def spmv_rect(row_ptr, col, weights, x, n_cols: int) -> np.ndarray:
    """Non-square A (rows = row_ptr.size - 1, n_cols columns) in CSR:
    y(c) = sum over entries (r, c) of w * x(r), FP64 (Sec. 3.5)."""
    lib = _load()
    row_ptr, col = _csr(row_ptr, col)
    n_rows = row_ptr.size - 1
    w = np.ascontiguousarray(weights, dtype=np.float64)
    y = np.empty(max(n_cols, 1), dtype=np.float64)
    lib.oracle_spmv_rect(n_rows, int(n_cols), row_ptr, col if col.size else np.zeros(1, np.uint32),
                         w if w.size else np.zeros(1), np.ascontiguousarray(x, dtype=np.float64), y)
    return y[:n_cols]


def weighted_scatter_gather(g: dict, wbin, x) -> np.ndarray:
    """Algorithm 3 + Algorithm 4 over the bins of :func:`png` with the weights
    applied in the gather (Sec. 3.5), FP64."""
    lib = _load()
    y = np.empty(g["n"], dtype=np.float64)
    src = g["src_idx"] if g["ne"] else np.zeros(1, dtype=np.uint32)
    dst = g["dest_ids"] if g["m"] else np.zeros(1, dtype=np.uint32)
    wb = np.ascontiguousarray(wbin, dtype=np.float64) if g["m"] else np.zeros(1)
    lib.oracle_weighted_gather(g["n"], g["k"], g["bin_u"], g["bin_e"], np.ascontiguousarray(src),
                               np.ascontiguousarray(dst), wb, np.ascontiguousarray(x, dtype=np.float64), y)
    return y
