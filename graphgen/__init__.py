"""Seeded synthetic graph inputs shared by the tests, the benchmark, the oracle
and the CUDA path.

This module holds none of the PageRank or partition-centric arithmetic. It
draws RMAT and Erdos-Renyi edge lists with a counter-based generator
(SplitMix64's output function over (seed, stream, counter)), relabels nodes
(random permutation, optionally followed by breadth-first order) and returns a
CSR out-adjacency: ``row_ptr`` uint32[n+1], ``col`` uint32[m], every row sorted
ascending, duplicates and self-loops removed. The heavy lifting is in
``graphgen.c`` (plain C, pthreads), compiled on first use.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB_PATH = os.path.join(_HERE, "_graphgen.so")
_lib = None
_lock = threading.Lock()

RELABEL = {"none": 0, "random": 1, "bfs": 2}


def build(force: bool = False) -> str:
    """Compiles graphgen.c into a shared library next to it; returns its path."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread", "-o", tmp, _SRC],
                       check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            p32 = ctypes.POINTER(ctypes.POINTER(ctypes.c_uint32))
            lib.gg_rmat.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                    p32, p32, ctypes.POINTER(ctypes.c_uint64)]
            lib.gg_er.argtypes = [ctypes.c_uint64, ctypes.c_double, ctypes.c_uint64, ctypes.c_int,
                                  ctypes.c_int, p32, p32, ctypes.POINTER(ctypes.c_uint64)]
            lib.gg_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double)]
            lib.gg_free.argtypes = [ctypes.c_void_p]
            _lib = lib
    return _lib


def _threads(threads):
    return int(threads) if threads else max(1, min(64, os.cpu_count() or 1))


def _take(lib, ptr, count):
    arr = np.ctypeslib.as_array(ptr, shape=(max(count, 1),))[:count].copy()
    lib.gg_free(ptr)
    return arr


def _call(fn, *args):
    lib = _load()
    rp = ctypes.POINTER(ctypes.c_uint32)()
    cp = ctypes.POINTER(ctypes.c_uint32)()
    m = ctypes.c_uint64(0)
    rc = fn(*args, ctypes.byref(rp), ctypes.byref(cp), ctypes.byref(m))
    if rc != 0:
        raise RuntimeError(f"graphgen failed with code {rc}")
    return rp, cp, m.value


def rmat(scale: int, edge_factor: float = 16.0, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 1709, relabel: str = "random", threads: int | None = None):
    """RMAT graph with 2**scale nodes and edge_factor * 2**scale drawn edges
    (fewer after duplicates and self-loops are removed). Returns (row_ptr, col)."""
    lib = _load()
    n = 1 << scale
    rp, cp, m = _call(lib.gg_rmat, int(scale), float(edge_factor), float(a), float(b), float(c),
                      int(seed), RELABEL[relabel], _threads(threads))
    return _take(lib, rp, n + 1), _take(lib, cp, m)


def erdos_renyi(n: int, mean_degree: float = 16.0, seed: int = 1709, relabel: str = "random",
                threads: int | None = None):
    """Erdos-Renyi style graph: mean_degree * n uniformly random (u, v) draws,
    duplicates and self-loops removed. Returns (row_ptr, col)."""
    lib = _load()
    rp, cp, m = _call(lib.gg_er, int(n), float(mean_degree), int(seed), RELABEL[relabel],
                      _threads(threads))
    return _take(lib, rp, n + 1), _take(lib, cp, m)


def uniform(count: int, seed: int) -> np.ndarray:
    """Seeded uniform doubles in [0, 1)."""
    lib = _load()
    out = np.empty(count, dtype=np.float64)
    lib.gg_uniform(int(count), int(seed), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


def random_rank_vector(n: int, seed: int) -> np.ndarray:
    """A seeded positive vector with entries in [0.5, 1.5)/n rescaled to sum 1,
    used as a non-uniform starting vector."""
    x = 0.5 + uniform(n, seed)
    return x / x.sum()


def csr_from_edges(n: int, src, dst, dedupe: bool = True, drop_self_loops: bool = True):
    """CSR (row_ptr uint32[n+1], col uint32[m]) from an explicit edge list, rows
    sorted ascending. Used for small hand-made graphs."""
    src = np.asarray(src, dtype=np.int64).ravel()
    dst = np.asarray(dst, dtype=np.int64).ravel()
    if src.shape != dst.shape:
        raise ValueError("src and dst differ in length")
    if src.size and (src.min() < 0 or dst.min() < 0 or src.max() >= n or dst.max() >= n):
        raise ValueError("edge endpoint out of range")
    if drop_self_loops:
        keep = src != dst
        src, dst = src[keep], dst[keep]
    order = np.lexsort((dst, src))
    src, dst = src[order], dst[order]
    if dedupe and src.size:
        keep = np.ones(src.size, dtype=bool)
        keep[1:] = (src[1:] != src[:-1]) | (dst[1:] != dst[:-1])
        src, dst = src[keep], dst[keep]
    row_ptr = np.zeros(n + 1, dtype=np.uint32)
    np.cumsum(np.bincount(src, minlength=n), out=row_ptr[1:])
    return row_ptr, dst.astype(np.uint32)


def random_graph(n: int, m_draws: int, seed: int, dedupe: bool = True, drop_self_loops: bool = True):
    """Small uniformly random digraph from m_draws seeded (u, v) draws."""
    r = uniform(2 * m_draws, seed)
    src = np.minimum((r[0::2] * n).astype(np.int64), n - 1)
    dst = np.minimum((r[1::2] * n).astype(np.int64), n - 1)
    return csr_from_edges(n, src, dst, dedupe=dedupe, drop_self_loops=drop_self_loops)
