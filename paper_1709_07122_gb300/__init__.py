"""Partition-Centric PageRank (PCPM, arXiv 1709.07122) on GB300 (sm_103a).

Thin Python binding over the C ABI of ``include/pcpm.h`` (``libpcpm.so``,
built in-tree by :func:`build`). Everything here is argument marshalling:
PyTorch provides device memory and the current CUDA stream; every step of the
method (PNG construction, scatter, gather/apply, reductions) runs in the
library's own kernels. There is no CPU fallback: if the library is missing the
calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

__all__ = ["build", "lib", "PNG", "pagerank_host", "PcpmError", "DANGLING_LEAK", "TWO_PHASE"]

PCPM_OK = 0
PCPM_NOT_CONVERGED = 1
DANGLING_LEAK = 0x1
TWO_PHASE = 0x2
DELTA = 0x4
NUM_PHASES = 3
PHASES = ("scatter", "gather_apply", "reduce")

_lib = None
_lock = threading.Lock()


class PcpmError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = lib().pcpm_strerror(code).decode() if _lib is not None else str(code)
        if code == -2 and _lib is not None:  # PCPM_ECUDA: name the CUDA error
            msg += " [" + lib().pcpm_last_cuda_error().decode() + "]"
        super().__init__(f"{where} failed: {msg} (status {code})")


class _Info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint32), ("part_size", ctypes.c_uint32), ("num_partitions", ctypes.c_uint32),
                ("shard_part_lo", ctypes.c_uint32), ("num_edges", ctypes.c_uint64), ("num_updates", ctypes.c_uint64),
                ("compression_ratio", ctypes.c_double), ("device_bytes", ctypes.c_uint64),
                ("iterations_done", ctypes.c_int32), ("gather_units", ctypes.c_uint32),
                ("scatter_units", ctypes.c_uint32), ("gather_cluster", ctypes.c_uint32),
                ("fused_ok", ctypes.c_uint32), ("canonical_gather", ctypes.c_uint32),
                ("gather_runs", ctypes.c_uint32), ("merged_adds", ctypes.c_uint64),
                ("update_dtype", ctypes.c_uint32), ("update_bytes", ctypes.c_uint32),
                ("gather_windows", ctypes.c_uint32), ("shard_part_hi", ctypes.c_uint32),
                ("num_windows", ctypes.c_uint64)]


class _Options(ctypes.Structure):
    _fields_ = [("gather_unit_chunks", ctypes.c_uint32), ("scatter_unit_groups", ctypes.c_uint32),
                ("gather_cluster", ctypes.c_uint32), ("canonical_gather", ctypes.c_uint32),
                ("gather_runs", ctypes.c_uint32), ("update_dtype", ctypes.c_uint32),
                ("gather_windows", ctypes.c_uint32)]

# Storage of the update bins (PCPM_UPDATE_* in pcpm.h).
UPDATE_DTYPES = {"f32": 0, "f16": 1, "bf16": 2}
F16_SCALE_LOG2 = 15


def build(force: bool = False, verbose: bool = False) -> str:
    """Compiles libpcpm.so for sm_103a (no-op when up to date)."""
    return _build.build(force=force, verbose=verbose)


def lib(path: str | None = None):
    """Loads libpcpm.so and declares its signatures; raises if it is absent."""
    global _lib
    with _lock:
        if _lib is None:
            path = path or _build.LIB_PATH
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library not built: {path} is missing (run __graft_entry__.build())")
            L = ctypes.CDLL(path)
            vp, u32, u64, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
            f32, f64 = ctypes.c_float, ctypes.c_double
            pi, pd, pf = ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_float)
            sig = {
                "pcpm_build": (i32, [vp, vp, u32, u64, u32, vp, ctypes.POINTER(vp)]),
                "pcpm_build_ex": (i32, [vp, vp, u32, u64, u32, ctypes.POINTER(_Options), vp, ctypes.POINTER(vp)]),
                "pcpm_free": (None, [vp]),
                "pcpm_png_get_info": (i32, [vp, ctypes.POINTER(_Info)]),
                "pcpm_png_export": (i32, [vp] + [vp] * 8),
                "pcpm_reset": (i32, [vp, vp, vp]),
                "pcpm_iterate": (i32, [vp, f32, i32, f64, u32, pi, pd, vp]),
                "pcpm_iterate_timed": (i32, [vp, f32, i32, u32, pf, vp]),
                "pcpm_ranks": (i32, [vp, vp, vp]),
                "pcpm_residual_history": (i32, [vp, vp, i32]),
                "pcpm_pagerank": (i32, [vp, f32, i32, f64, u32, vp, vp, pi, pd, vp]),
                "pcpm_pagerank_host": (i32, [vp, vp, u32, u64, u32, f32, i32, f64, u32, vp, pi, pd]),
                "pcpm_scatter_only": (i32, [vp, vp]),
                "pcpm_export_state": (i32, [vp, vp, vp, vp, pd]),
                "pcpm_rank_stats_noalloc": (i32, [vp, vp, vp, u32, vp, vp]),
                "pcpm_strerror": (ctypes.c_char_p, [i32]),
                "pcpm_last_cuda_error": (ctypes.c_char_p, []),
                "pcpm_release_cached_memory": (i32, []),
                "pcpm_autotune": (i32, [vp, vp, u32, u64, vp, i32, f32, i32, i32, u32, vp, ctypes.POINTER(u32),
                                        vp]),
                "pcpm_autotune_ex": (i32, [vp, vp, u32, u64, vp, i32, ctypes.POINTER(_Options), i32, f32, i32,
                                           i32, u32, vp, ctypes.POINTER(u32), pi, vp]),
                "pcpm_ppr_create": (i32, [vp, vp, vp, vp, ctypes.POINTER(vp)]),
                "pcpm_ppr_run": (i32, [vp, f32, i32, vp]),
                "pcpm_ppr_residuals": (i32, [vp, vp, i32]),
                "pcpm_ppr_ranks": (i32, [vp, vp, vp]),
                "pcpm_ppr_info": (i32, [vp, ctypes.POINTER(u64), ctypes.POINTER(u32)]),
                "pcpm_ppr_free": (None, [vp]),
                "pcpm_build_weighted": (i32, [vp, vp, vp, u32, u64, u32, ctypes.POINTER(_Options), vp,
                                              ctypes.POINTER(vp)]),
                "pcpm_spmv": (i32, [vp, vp, vp, vp]),
                "pcpm_batch_create": (i32, [vp, i32, f32, i32, u32, ctypes.POINTER(vp)]),
                "pcpm_batch_launch": (i32, [vp, vp]),
                "pcpm_batch_free": (None, [vp]),
                "pcpm_batch_kernel_launches": (i32, [vp, ctypes.POINTER(i32)]),
                "pcpm_export_weights": (i32, [vp, vp]),
                "pcpm_ws_features": (i32, [vp, vp, vp, vp, vp]),
                "pcpm_ws_predict": (i32, [vp, vp, u32, vp, vp]),
                "pcpm_ws_targets": (i32, [vp, u32, vp, vp]),
                "pcpm_ws_loss_grad": (i32, [vp, vp, vp, u32, vp, vp, vp]),
                "pcpm_ws_adam": (i32, [vp, vp, vp, vp, i32, f32, f32, f32, f32, vp]),
                "pcpm_ws_init_ranks": (i32, [vp, u32, vp, vp]),
                "pcpm_ws_degree_sums": (i32, [vp, vp, vp, vp]),
                "pcpm_ws_feature_moments": (i32, [vp, u32, vp, vp]),
                "pcpm_ws_standardisation": (i32, [vp, vp, vp]),
                "pcpm_dest_partition_counts": (i32, [vp, u64, u32, u32, vp, vp]),
                "pcpm_shard_split": (i32, [vp, u32, u32, u32, vp]),
                "pcpm_build_shard": (i32, [vp, vp, u32, u64, u32, u32, u32, ctypes.POINTER(_Options), vp,
                                           ctypes.POINTER(vp)]),
                "pcpm_shard_init": (i32, [vp, vp, vp, vp, vp]),
                "pcpm_shard_step": (i32, [vp, f32, u32, vp, vp, vp, vp]),
                "pcpm_sync_status": (i32, [vp]),
                "pcpm_build_rect": (i32, [vp, vp, vp, u32, u32, u64, u32, ctypes.POINTER(_Options), vp,
                                          ctypes.POINTER(vp)]),
                "pcpm_spmv_rect": (i32, [vp, vp, vp, vp]),
                "pcpm_test_wait_limit": (i32, [ctypes.c_longlong]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(code: int, where: str, allow=(PCPM_OK,)) -> int:
    if code not in allow:
        raise PcpmError(code, where)
    return code


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev_u32(t):
    """A CUDA tensor of 32-bit integers (int32 or uint32) viewed for the ABI."""
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda):
        raise TypeError("expected a CUDA tensor")
    if t.dtype not in (torch.int32, getattr(torch, "uint32", torch.int32)):
        raise TypeError("expected a 32-bit integer tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _flags(dangling: str, mode: str = "fused") -> int:
    """mode: "fused", "two_phase", or "delta" (two-phase iterations that
    scatter the change of SPR, PCPM_DELTA)."""
    if dangling not in ("uniform", "leak"):
        raise ValueError("dangling must be 'uniform' or 'leak'")
    if mode not in ("fused", "two_phase", "delta"):
        raise ValueError("mode must be 'fused', 'two_phase' or 'delta'")
    return ((DANGLING_LEAK if dangling == "leak" else 0) | (TWO_PHASE if mode != "fused" else 0)
            | (DELTA if mode == "delta" else 0))


def autotune(row_ptr, col, part_sizes=(2048, 4096, 8192, 16384, 32768), d: float = 0.85, warmup: int = 2,
             iters: int = 5, dangling: str = "uniform", mode: str = "two_phase", stream=None):
    """Partition-size autotuner (pcpm_autotune) on a device CSR: returns
    (best part size, {part size: ms per iteration, or None if rejected})."""
    cand = np.ascontiguousarray(part_sizes, dtype=np.uint32)
    ms = np.empty(cand.size, np.float32)
    best = ctypes.c_uint32(0)
    n = row_ptr.numel() - 1
    m = int(row_ptr[-1].item()) & 0xFFFFFFFF
    _check(lib().pcpm_autotune(_dev_u32(row_ptr), _dev_u32(col), n, m, cand.ctypes.data_as(ctypes.c_void_p),
                               int(cand.size), float(d), int(warmup), int(iters), _flags(dangling, mode),
                               _stream(stream), ctypes.byref(best), ms.ctypes.data_as(ctypes.c_void_p)),
           "pcpm_autotune")
    return best.value, {int(q): (float(t) if t >= 0 else None) for q, t in zip(cand, ms)}


# Tile shapes the autotuner tries by default: the automatic decomposition,
# one gather CTA per unit, four-CTA clusters, small and large gather units,
# and the chunk layout.
TILE_SHAPES = ({}, {"gather_cluster": 1}, {"gather_cluster": 4}, {"gather_unit_chunks": 64},
               {"gather_unit_chunks": 1024}, {"scatter_unit_groups": 4096}, {"gather_windows": 2})


def autotune_tiles(row_ptr, col, part_sizes=(8192, 16384, 32768), tile_shapes=TILE_SHAPES, d: float = 0.85,
                   warmup: int = 2, iters: int = 5, dangling: str = "uniform", mode: str = "two_phase",
                   stream=None):
    """Partition size and tile shape (pcpm_autotune_ex) on a device CSR:
    returns (best part size, best build options dict, {(part size, shape
    index): ms per iteration, or None if rejected})."""
    cand = np.ascontiguousarray(part_sizes, dtype=np.uint32)
    shapes = list(tile_shapes)
    opts = (_Options * len(shapes))(*[_Options(**{k: int(v) for k, v in o.items()}) for o in shapes])
    ms = np.empty(cand.size * len(shapes), np.float32)
    best_q, best_o = ctypes.c_uint32(0), ctypes.c_int(0)
    n = row_ptr.numel() - 1
    m = int(row_ptr[-1].item()) & 0xFFFFFFFF
    _check(lib().pcpm_autotune_ex(_dev_u32(row_ptr), _dev_u32(col), n, m, cand.ctypes.data_as(ctypes.c_void_p),
                                  int(cand.size), opts, len(shapes), float(d), int(warmup), int(iters),
                                  _flags(dangling, mode), _stream(stream), ctypes.byref(best_q),
                                  ctypes.byref(best_o), ms.ctypes.data_as(ctypes.c_void_p)), "pcpm_autotune_ex")
    table = {(int(q), j): (float(ms[i * len(shapes) + j]) if ms[i * len(shapes) + j] >= 0 else None)
             for i, q in enumerate(cand) for j in range(len(shapes))}
    return best_q.value, dict(shapes[best_o.value]), table


def release_cached_memory() -> None:
    """Returns device memory that the library's pool keeps for later builds,
    but that no live handle uses, to the driver (pcpm_release_cached_memory)."""
    _check(lib().pcpm_release_cached_memory(), "pcpm_release_cached_memory")


def to_device_csr(row_ptr: np.ndarray, col: np.ndarray, device="cuda"):
    """Copies a host CSR (uint32 arrays) to CUDA int32 tensors (same bits)."""
    import torch
    rp = torch.from_numpy(np.ascontiguousarray(row_ptr, dtype=np.uint32).view(np.int32)).to(device)
    c = np.ascontiguousarray(col, dtype=np.uint32)
    ct = torch.from_numpy((c if c.size else np.zeros(1, np.uint32)).view(np.int32)).to(device)
    return rp, ct


class PNG:
    """A device-resident Partition-Node Graph and its solver state."""

    def __init__(self, row_ptr, col, part_size: int, stream=None, **options):
        """row_ptr, col: CUDA int32/uint32 tensors (CSR out-adjacency, rows sorted).
        options: gather_unit_chunks, scatter_unit_groups, gather_cluster (0 = automatic),
        canonical_gather (1 = gather from the canonical bins), gather_runs (1 = sum runs of
        equal destinations in registers, 2 = never, 0 = automatic), update_dtype ("f32", "f16",
        "bf16" or the PCPM_UPDATE_* value)."""
        L = lib()
        n = row_ptr.numel() - 1
        m = int(row_ptr[-1].item()) & 0xFFFFFFFF
        h = ctypes.c_void_p()
        if isinstance(options.get("update_dtype"), str):
            options = dict(options, update_dtype=UPDATE_DTYPES[options["update_dtype"]])
        opt = _Options(**{k: int(v) for k, v in options.items()})
        _check(L.pcpm_build_ex(_dev_u32(row_ptr), _dev_u32(col), n, m, int(part_size), ctypes.byref(opt),
                               _stream(stream), ctypes.byref(h)), "pcpm_build")
        self._h = h
        self.n = n

    @classmethod
    def shard(cls, row_ptr, col, part_size: int, part_lo: int, part_hi: int, stream=None, **options):
        """The bins of destination partitions [part_lo, part_hi) only
        (pcpm_build_shard); driven by shard_init / shard_step."""
        if isinstance(options.get("update_dtype"), str):
            options = dict(options, update_dtype=UPDATE_DTYPES[options["update_dtype"]])
        n = row_ptr.numel() - 1
        m = int(row_ptr[-1].item()) & 0xFFFFFFFF
        opt = _Options(**{k: int(v) for k, v in options.items()})
        h = ctypes.c_void_p()
        _check(lib().pcpm_build_shard(_dev_u32(row_ptr), _dev_u32(col), n, m, int(part_size), int(part_lo),
                                      int(part_hi), ctypes.byref(opt), _stream(stream), ctypes.byref(h)),
               "pcpm_build_shard")
        obj = cls.__new__(cls)
        obj._h = h
        obj.n = n
        return obj

    @classmethod
    def rect(cls, row_ptr, col, n_cols: int, part_size: int, weights=None, stream=None, **options):
        """A non-square matrix (rows = row_ptr.numel() - 1, n_cols columns)
        for pcpm_spmv_rect (Sec. 3.5); weights: CUDA float32 per entry or None."""
        if isinstance(options.get("update_dtype"), str):
            options = dict(options, update_dtype=UPDATE_DTYPES[options["update_dtype"]])
        n_rows = row_ptr.numel() - 1
        m = int(row_ptr[-1].item()) & 0xFFFFFFFF
        opt = _Options(**{k: int(v) for k, v in options.items()})
        w = None
        if weights is not None and m:
            w = ctypes.c_void_p(_f32(weights, m, "weights").value)
        h = ctypes.c_void_p()
        _check(lib().pcpm_build_rect(_dev_u32(row_ptr), _dev_u32(col) if m else None, w, n_rows, int(n_cols), m,
                                     int(part_size), ctypes.byref(opt), _stream(stream), ctypes.byref(h)),
               "pcpm_build_rect")
        obj = cls.__new__(cls)
        obj._h = h
        obj.n = max(n_rows, int(n_cols))
        obj.n_rows, obj.n_cols = n_rows, int(n_cols)
        return obj

    def spmv_rect(self, x, out=None, stream=None):
        """y = A^T_w x of a non-square handle (pcpm_spmv_rect)."""
        import torch
        out = torch.empty(self.n_cols, dtype=torch.float32, device="cuda") if out is None else out
        _check(lib().pcpm_spmv_rect(self._h, _f32(x, self.n_rows, "x"), _f32(out, self.n_cols, "out"),
                                    _stream(stream)), "pcpm_spmv_rect")
        return out

    def shard_init(self, pr_out, sums, pr_init=None, stream=None):
        """pcpm_shard_init: PR_0 into pr_out (all n), sums = {0, own dangling mass}."""
        p = None if pr_init is None else ctypes.c_void_p(_f32_dev(pr_init, self.n).data_ptr())
        _check(lib().pcpm_shard_init(self._h, p, ctypes.c_void_p(_f32_dev(pr_out, self.n).data_ptr()),
                                     ctypes.c_void_p(_f64_dev(sums, 2).data_ptr()), _stream(stream)),
               "pcpm_shard_init")

    def shard_step(self, pr_in, pr_out, sums, d: float = 0.85, dangling: str = "uniform", stream=None):
        """pcpm_shard_step: PR_{i+1} of the shard's own nodes into pr_out;
        sums[1] must hold the whole graph's dangling mass of pr_in."""
        _check(lib().pcpm_shard_step(self._h, float(d), _flags(dangling, "two_phase"),
                                     ctypes.c_void_p(_f32_dev(pr_in, self.n).data_ptr()),
                                     ctypes.c_void_p(_f32_dev(pr_out, self.n).data_ptr()),
                                     ctypes.c_void_p(_f64_dev(sums, 2).data_ptr()), _stream(stream)),
               "pcpm_shard_step")

    def sync_status(self) -> None:
        """Waits for the handle's stream; raises on a device-side error."""
        _check(lib().pcpm_sync_status(self._h), "pcpm_sync_status")

    @classmethod
    def weighted(cls, row_ptr, col, weights, part_size: int, stream=None, **options):
        """Weighted graph (Sec. 3.5): weights is a CUDA float32 tensor of one
        value per column index (CSR order); see pcpm_build_weighted."""
        if isinstance(options.get("update_dtype"), str):
            options = dict(options, update_dtype=UPDATE_DTYPES[options["update_dtype"]])
        L = lib()
        n = row_ptr.numel() - 1
        m = int(row_ptr[-1].item()) & 0xFFFFFFFF
        opt = _Options(**{k: int(v) for k, v in options.items()})
        h = ctypes.c_void_p()
        w = ctypes.c_void_p(weights.data_ptr()) if m else ctypes.c_void_p(1)
        if m:
            _f32(weights, m, "weights")
        _check(L.pcpm_build_weighted(_dev_u32(row_ptr), _dev_u32(col), w, n, m, int(part_size), ctypes.byref(opt),
                                     _stream(stream), ctypes.byref(h)), "pcpm_build_weighted")
        obj = cls.__new__(cls)
        obj._h = h
        obj.n = n
        return obj

    def spmv(self, x, out=None, stream=None):
        """y = A^T_w x over the PNG (pcpm_spmv): y(v) = sum of w(u, v) x(u)."""
        import torch
        out = torch.empty(self.n, dtype=torch.float32, device="cuda") if out is None else out
        _check(lib().pcpm_spmv(self._h, _f32(x, self.n, "x"), _f32(out, self.n, "out"), _stream(stream)), "pcpm_spmv")
        return out

    def export_weights(self) -> np.ndarray:
        """Weights in canonical bin order (pcpm_export_weights)."""
        m = self.info["num_edges"]
        w = np.empty(max(m, 1), np.float32)
        _check(lib().pcpm_export_weights(self._h, w.ctypes.data_as(ctypes.c_void_p)), "pcpm_export_weights")
        return w[:m]

    @classmethod
    def from_host(cls, row_ptr: np.ndarray, col: np.ndarray, part_size: int, stream=None, **options):
        rp, c = to_device_csr(row_ptr, col)
        return cls(rp, c, part_size, stream, **options)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().pcpm_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def info(self) -> dict:
        i = _Info()
        _check(lib().pcpm_png_get_info(self._h, ctypes.byref(i)), "pcpm_png_get_info")
        return {f: getattr(i, f) for f, _ in _Info._fields_ if not f.startswith("reserved")}

    def export(self) -> dict:
        """Host copies of counts, offsets, bin starts and bins (see pcpm.h)."""
        inf = self.info
        k, ne, m = inf["num_partitions"], inf["num_updates"], inf["num_edges"]
        out = {key: np.empty(k * k, np.uint32) for key in ("cnt_u", "cnt_e", "off_u", "off_e")}
        out["bin_u"] = np.empty(k + 1, np.uint32)
        out["bin_e"] = np.empty(k + 1, np.uint32)
        out["src_idx"] = np.empty(max(ne, 1), np.uint32)
        out["dest_ids"] = np.empty(max(m, 1), np.uint32)
        order = ("cnt_u", "cnt_e", "off_u", "off_e", "bin_u", "bin_e", "src_idx", "dest_ids")
        _check(lib().pcpm_png_export(self._h, *[out[x].ctypes.data_as(ctypes.c_void_p) for x in order]),
               "pcpm_png_export")
        for key in ("cnt_u", "cnt_e", "off_u", "off_e"):
            out[key] = out[key].reshape(k, k)
        out["src_idx"] = out["src_idx"][:ne]
        out["dest_ids"] = out["dest_ids"][:m]
        out.update(k=k, ne=ne, m=m, n=inf["n"], q=inf["part_size"])
        return out

    def reset(self, pr_init=None, stream=None):
        p = None if pr_init is None else ctypes.c_void_p(_f32_dev(pr_init, self.n).data_ptr())
        _check(lib().pcpm_reset(self._h, p, _stream(stream)), "pcpm_reset")

    def iterate(self, d: float = 0.85, iters: int = 1, tol: float = 0.0, dangling: str = "uniform",
                stream=None, sync: bool = True, mode: str = "fused"):
        """Advances the state; returns (iterations run, last L1 change) when sync."""
        it, res = ctypes.c_int(0), ctypes.c_double(0.0)
        code = lib().pcpm_iterate(self._h, float(d), int(iters), float(tol), _flags(dangling, mode),
                                  ctypes.byref(it) if sync else None, ctypes.byref(res) if sync else None,
                                  _stream(stream))
        _check(code, "pcpm_iterate", allow=(PCPM_OK, PCPM_NOT_CONVERGED))
        return (it.value, res.value) if sync else None

    def iterate_timed(self, d: float = 0.85, iters: int = 1, dangling: str = "uniform", stream=None,
                      mode: str = "fused") -> dict:
        ms = (ctypes.c_float * (NUM_PHASES + 1))()
        _check(lib().pcpm_iterate_timed(self._h, float(d), int(iters), _flags(dangling, mode), ms, _stream(stream)),
               "pcpm_iterate_timed")
        return dict(zip(PHASES + ("span",), list(ms)))

    def ranks(self, out=None, stream=None):
        import torch
        out = torch.empty(self.n, dtype=torch.float32, device="cuda") if out is None else _f32_dev(out, self.n)
        _check(lib().pcpm_ranks(self._h, ctypes.c_void_p(out.data_ptr()), _stream(stream)), "pcpm_ranks")
        return out

    def residual_history(self) -> np.ndarray:
        cnt = self.info["iterations_done"]
        buf = np.empty(max(cnt, 1), np.float64)
        got = lib().pcpm_residual_history(self._h, buf.ctypes.data_as(ctypes.c_void_p), cnt)
        if got < 0:
            raise PcpmError(got, "pcpm_residual_history")
        return buf[:got]

    def pagerank(self, d: float = 0.85, max_iters: int = 20, tol: float = 0.0, pr_init=None,
                 dangling: str = "uniform", out=None, stream=None, mode: str = "fused"):
        """Full solve; returns (ranks tensor, iterations run, last L1 change)."""
        import torch
        out = torch.empty(self.n, dtype=torch.float32, device="cuda") if out is None else _f32_dev(out, self.n)
        p = None if pr_init is None else ctypes.c_void_p(_f32_dev(pr_init, self.n).data_ptr())
        it, res = ctypes.c_int(0), ctypes.c_double(0.0)
        code = lib().pcpm_pagerank(self._h, float(d), int(max_iters), float(tol), _flags(dangling, mode), p,
                                   ctypes.c_void_p(out.data_ptr()), ctypes.byref(it), ctypes.byref(res),
                                   _stream(stream))
        _check(code, "pcpm_pagerank", allow=(PCPM_OK, PCPM_NOT_CONVERGED))
        return out, it.value, res.value

    def scatter_only(self, stream=None):
        _check(lib().pcpm_scatter_only(self._h, _stream(stream)), "pcpm_scatter_only")

    def export_state(self) -> dict:
        inf = self.info
        pr = np.empty(self.n, np.float32)
        spr = np.empty(self.n, np.float32)
        # raw update bins: float32, float16 (SPR * 2^15) or bfloat16 bits as uint16
        utype = {0: np.float32, 1: np.float16, 2: np.uint16}[inf["update_dtype"]]
        upd = np.empty(max(inf["num_updates"], 1), utype)
        dang = ctypes.c_double(0.0)
        _check(lib().pcpm_export_state(self._h, pr.ctypes.data_as(ctypes.c_void_p),
                                       spr.ctypes.data_as(ctypes.c_void_p), upd.ctypes.data_as(ctypes.c_void_p),
                                       ctypes.byref(dang)), "pcpm_export_state")
        return {"pr": pr, "spr": spr, "updates": upd[:inf["num_updates"]], "dangling": dang.value}


def _f32_dev(t, n):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise TypeError("expected a contiguous CUDA float32 tensor")
    if t.numel() != n:
        raise ValueError(f"expected {n} elements, got {t.numel()}")
    return t


def _f64_dev(t, n):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous CUDA float64 tensor")
    if t.numel() != n:
        raise ValueError(f"expected {n} elements, got {t.numel()}")
    return t


def dest_partition_counts(col, n: int, part_size: int, m: int | None = None, stream=None) -> np.ndarray:
    """Edges per destination partition of a device CSR's columns
    (pcpm_dest_partition_counts): uint64 [ceil(n / part_size)]. m: the edge
    count (default col.numel())."""
    k = (n + part_size - 1) // part_size
    out = np.zeros(k, np.uint64)
    m = col.numel() if m is None else int(m)
    _check(lib().pcpm_dest_partition_counts(_dev_u32(col) if m else None, m, n, int(part_size),
                                            out.ctypes.data_as(ctypes.c_void_p), _stream(stream)),
           "pcpm_dest_partition_counts")
    return out


def shard_split(ids_per_part, n: int, part_size: int, nranks: int) -> np.ndarray:
    """Contiguous destination-partition ranges of near-equal weight
    (pcpm_shard_split, host only): uint32 [nranks + 1] cut points."""
    ids = np.ascontiguousarray(ids_per_part, dtype=np.uint64)
    if ids.size != (n + part_size - 1) // part_size:
        raise ValueError("ids_per_part needs one count per partition")
    out = np.zeros(nranks + 1, np.uint32)
    _check(lib().pcpm_shard_split(ids.ctypes.data_as(ctypes.c_void_p), int(n), int(part_size), int(nranks),
                                  out.ctypes.data_as(ctypes.c_void_p)), "pcpm_shard_split")
    return out


def pagerank_host(row_ptr: np.ndarray, col: np.ndarray, part_size: int, d: float = 0.85, max_iters: int = 20,
                  tol: float = 0.0, dangling: str = "uniform", pr_out: np.ndarray | None = None,
                  mode: str = "fused"):
    """End-to-end solve from host arrays through pcpm_pagerank_host.
    Returns (ranks float32 array, iterations run, last L1 change)."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.uint32)
    c = np.ascontiguousarray(col, dtype=np.uint32)
    n = rp.size - 1
    out = np.empty(n, np.float32) if pr_out is None else pr_out
    it, res = ctypes.c_int(0), ctypes.c_double(0.0)
    code = lib().pcpm_pagerank_host(rp.ctypes.data_as(ctypes.c_void_p),
                                    c.ctypes.data_as(ctypes.c_void_p) if c.size else None, n, int(rp[-1]),
                                    int(part_size), float(d), int(max_iters), float(tol), _flags(dangling, mode),
                                    out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(it), ctypes.byref(res))
    _check(code, "pcpm_pagerank_host", allow=(PCPM_OK, PCPM_NOT_CONVERGED))
    return out, it.value, res.value


def rank_stats_noalloc(x, y, row_ptr, out=None, stream=None):
    """(L1 change between x and y, dangling mass of x) in FP64 through the
    allocation-free entry point. x, y: CUDA float32 [n]; row_ptr: CUDA 32-bit
    integer [n+1]; out: CUDA float64 [2].

    The entry point itself allocates nothing. With out=None this wrapper
    allocates the result through torch, so a caller that must not allocate
    (inside an allocator callback, or with all device memory reserved up
    front) passes a preallocated `out`."""
    import torch
    n = row_ptr.numel() - 1
    _f32_dev(x, n)
    _f32_dev(y, n)
    if out is None:
        out = torch.empty(2, dtype=torch.float64, device="cuda")
    elif not (isinstance(out, torch.Tensor) and out.is_cuda and out.dtype == torch.float64
              and out.is_contiguous() and out.numel() >= 2):
        raise TypeError("out: expected a contiguous CUDA float64 tensor of at least 2 elements")
    _check(lib().pcpm_rank_stats_noalloc(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                         _dev_u32(row_ptr), n, ctypes.c_void_p(out.data_ptr()), _stream(stream)),
           "pcpm_rank_stats_noalloc")
    return out


# ----------------------------------------------------------- warm start
# Learned warm start (pcpm_warmstart.h): features, network inference and
# training steps, and the initial rank vector. Shapes: features [n, 5],
# params [WS_PARAMS] (mu, inv_sigma, W1, b1, W2, b2, w3, b3), all float32 CUDA.
WS_FEATURES, WS_HIDDEN, WS_TRAINABLE = 5, 64, 10
WS_PARAMS = 2 * 5 + 64 * 5 + 64 + 64 * 64 + 64 + 64 + 1


def _f32(t, numel=None, name="tensor"):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise TypeError(f"{name}: expected a contiguous CUDA float32 tensor")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name}: expected {numel} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def ws_features(png: "PNG", row_ptr, col, out=None, stream=None):
    """Features of every node (pcpm_ws_features); resets the handle's state."""
    import torch
    out = torch.empty((png.n, WS_FEATURES), dtype=torch.float32, device="cuda") if out is None else out
    _check(lib().pcpm_ws_features(png._h, _dev_u32(row_ptr), _dev_u32(col),
                                  _f32(out, png.n * WS_FEATURES, "features"), _stream(stream)), "pcpm_ws_features")
    return out


def ws_degree_sums(png: "PNG", row_ptr, out=None, stream=None):
    """Exact in-degree, sum of in-neighbours' in-degrees and sum of their
    out-degrees (pcpm_ws_degree_sums): CUDA int32 [3, n] holding uint32 bits."""
    import torch
    out = torch.empty((3, png.n), dtype=torch.int32, device="cuda") if out is None else out
    if not (out.is_cuda and out.dtype == torch.int32 and out.is_contiguous() and out.numel() == 3 * png.n):
        raise TypeError("out: expected a contiguous CUDA int32 tensor of 3 * n elements")
    _check(lib().pcpm_ws_degree_sums(png._h, _dev_u32(row_ptr), ctypes.c_void_p(out.data_ptr()), _stream(stream)),
           "pcpm_ws_degree_sums")
    return out


def ws_feature_moments(features, moments, stream=None):
    """Adds the FP64 row count, column sums and sums of squares of the
    features [n, 5] to moments (CUDA float64 [11]) (pcpm_ws_feature_moments)."""
    n = features.shape[0]
    _check(lib().pcpm_ws_feature_moments(_f32(features, n * WS_FEATURES, "features"), n,
                                         ctypes.c_void_p(_f64_dev(moments, 11).data_ptr()), _stream(stream)),
           "pcpm_ws_feature_moments")


def ws_standardisation(moments, params, stream=None):
    """mu and inv_sigma from accumulated moments into params[0:10]
    (pcpm_ws_standardisation)."""
    _check(lib().pcpm_ws_standardisation(ctypes.c_void_p(_f64_dev(moments, 11).data_ptr()),
                                         _f32(params, WS_PARAMS, "params"), _stream(stream)),
           "pcpm_ws_standardisation")


def ws_targets(pr, out=None, stream=None):
    """Training targets log(n * pr) (pcpm_ws_targets)."""
    import torch
    n = pr.numel()
    out = torch.empty(n, dtype=torch.float32, device="cuda") if out is None else out
    _check(lib().pcpm_ws_targets(_f32(pr, n, "pr"), n, _f32(out, n, "out"), _stream(stream)), "pcpm_ws_targets")
    return out


def ws_predict(params, features, out=None, stream=None):
    """Network output per row, BF16-rounded weights (pcpm_ws_predict)."""
    import torch
    n = features.shape[0]
    out = torch.empty(n, dtype=torch.float32, device="cuda") if out is None else out
    _check(lib().pcpm_ws_predict(_f32(params, WS_PARAMS, "params"), _f32(features, n * WS_FEATURES, "features"), n,
                                 _f32(out, n, "out"), _stream(stream)), "pcpm_ws_predict")
    return out


def ws_loss_grad(params, features, target, grad, loss, stream=None):
    """Mean squared error and its gradient into grad [WS_PARAMS] and loss
    (float64 [1]) on the device (pcpm_ws_loss_grad); does not synchronise."""
    import torch
    n = features.shape[0]
    if not (isinstance(loss, torch.Tensor) and loss.is_cuda and loss.dtype == torch.float64 and loss.numel() == 1):
        raise TypeError("loss: expected a CUDA float64 tensor of one element")
    _check(lib().pcpm_ws_loss_grad(_f32(params, WS_PARAMS, "params"), _f32(features, n * WS_FEATURES, "features"),
                                   _f32(target, n, "target"), n, _f32(grad, WS_PARAMS, "grad"),
                                   ctypes.c_void_p(loss.data_ptr()), _stream(stream)), "pcpm_ws_loss_grad")


def ws_adam(params, grad, m, v, step: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
            eps: float = 1e-8, stream=None):
    """One Adam step on the trainable parameters (pcpm_ws_adam)."""
    _check(lib().pcpm_ws_adam(_f32(params, WS_PARAMS, "params"), _f32(grad, WS_PARAMS, "grad"),
                              _f32(m, WS_PARAMS, "m"), _f32(v, WS_PARAMS, "v"), int(step), float(lr), float(beta1),
                              float(beta2), float(eps), _stream(stream)), "pcpm_ws_adam")


def ws_init_ranks(pred, out=None, stream=None):
    """Initial ranks softmax(pred) (pcpm_ws_init_ranks)."""
    import torch
    n = pred.numel()
    out = torch.empty(n, dtype=torch.float32, device="cuda") if out is None else out
    _check(lib().pcpm_ws_init_ranks(_f32(pred, n, "pred"), n, _f32(out, n, "out"), _stream(stream)),
           "pcpm_ws_init_ranks")
    return out


class Batch:
    """Independent graphs solved by one CUDA graph launch (pcpm_batch_*):
    every handle is reset to the uniform start and iterated `iters` times."""

    def __init__(self, handles, d: float = 0.85, iters: int = 20, dangling: str = "uniform",
                 mode: str = "two_phase"):
        self.handles = list(handles)  # the handles must outlive the batch
        arr = (ctypes.c_void_p * len(self.handles))(*[h._h.value for h in self.handles])
        b = ctypes.c_void_p()
        _check(lib().pcpm_batch_create(arr, len(self.handles), float(d), int(iters), _flags(dangling, mode),
                                       ctypes.byref(b)), "pcpm_batch_create")
        self._b = b

    def launch(self, stream=None):
        _check(lib().pcpm_batch_launch(self._b, _stream(stream)), "pcpm_batch_launch")

    @property
    def kernel_launches(self) -> int:
        """Kernels one launch runs (pcpm_batch_kernel_launches)."""
        k = ctypes.c_int32()
        _check(lib().pcpm_batch_kernel_launches(self._b, ctypes.byref(k)), "pcpm_batch_kernel_launches")
        return int(k.value)

    def close(self):
        if getattr(self, "_b", None) is not None and self._b.value:
            lib().pcpm_batch_free(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


PPR_COLS = 64


class PPR:
    """Batched personalized PageRank over a PNG (pcpm_ppr_*): PPR_COLS columns,
    column j teleporting uniformly to its seeds seed_idx[seed_ptr[j]:seed_ptr[j+1]].
    The PNG must outlive the solver."""

    def __init__(self, png: "PNG", seed_ptr, seed_idx, stream=None):
        sp = np.ascontiguousarray(seed_ptr, dtype=np.uint32)
        si = np.ascontiguousarray(seed_idx, dtype=np.uint32)
        if sp.size != PPR_COLS + 1:
            raise ValueError(f"seed_ptr needs {PPR_COLS + 1} entries")
        self.png = png
        self.n = png.n
        h = ctypes.c_void_p()
        _check(lib().pcpm_ppr_create(png._h, sp.ctypes.data_as(ctypes.c_void_p),
                                     si.ctypes.data_as(ctypes.c_void_p) if si.size else None, _stream(stream),
                                     ctypes.byref(h)), "pcpm_ppr_create")
        self._h = h
        self.iters = 0

    def run(self, d: float = 0.85, iters: int = 20, stream=None):
        """From R = T, `iters` iterations on the stream (no synchronisation)."""
        _check(lib().pcpm_ppr_run(self._h, float(d), int(iters), _stream(stream)), "pcpm_ppr_run")
        self.iters = int(iters)

    def residuals(self, iters: int | None = None) -> np.ndarray:
        """L1 change per column of each iteration of the last run: [iters, PPR_COLS]."""
        it = self.iters if iters is None else int(iters)
        out = np.empty((max(it, 1), PPR_COLS), np.float64)
        _check(lib().pcpm_ppr_residuals(self._h, out.ctypes.data_as(ctypes.c_void_p), it), "pcpm_ppr_residuals")
        return out[:it]

    def ranks(self, out=None, stream=None):
        """The current ranks as a CUDA float32 tensor [n, PPR_COLS]."""
        import torch
        out = torch.empty((self.n, PPR_COLS), dtype=torch.float32, device="cuda") if out is None else out
        if not (out.is_cuda and out.dtype == torch.float32 and out.is_contiguous()
                and tuple(out.shape) == (self.n, PPR_COLS)):
            raise ValueError(f"out must be a contiguous CUDA float32 tensor of shape ({self.n}, {PPR_COLS})")
        _check(lib().pcpm_ppr_ranks(self._h, ctypes.c_void_p(out.data_ptr()), _stream(stream)), "pcpm_ppr_ranks")
        return out

    @property
    def info(self) -> dict:
        b, sd = ctypes.c_uint64(0), ctypes.c_uint32(0)
        _check(lib().pcpm_ppr_info(self._h, ctypes.byref(b), ctypes.byref(sd)), "pcpm_ppr_info")
        return {"device_bytes": b.value, "split_destinations": sd.value}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().pcpm_ppr_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
